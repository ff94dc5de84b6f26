// Level sweeps of Alg. 1 (generate, v = L xi) and the inverse application
// and log-determinant of Sec. 3 (whiten, xi = L^-1 v; logdet; NLL).
//
// generate: v_0 = L0 xi_0 for the dense block, then batch by batch
// (Sec. 2.2: points of one depth level are conditionally independent)
// v_i = b_i . v_c(i) + sigma_i xi_i; every neighbour lies in an earlier level.
// One cooperative launch walks the levels with a grid-wide barrier between
// consecutive levels (sweepsync.cuh).  Rows, sigma and xi do not depend on
// the field: each lane group loads those of its next step before gathering
// the current one, and those of a level's first step before the barrier, so
// the row stream overlaps both the gathers and the barrier.  The depth levels
// at both ends of the sweep hold a few dozen to a few hundred points (about
// 90 levels at any N); each of those runs is done by a single block that
// synchronises with __syncthreads, since a grid barrier per level costs
// more than the level's work there.
//
// whiten: xi_i = (v_i - b_i . v_c(i)) / sigma_i has no dependencies.  Blocks
// walk spatial tiles through every level (plus xi_0 = L0^-1 v_0 for the
// dense block), so the gathered v lines of a tile stay in L1; rows are
// streamed without L1 allocation, v is kept in L2 (evict-last).
#include <algorithm>

#include "sweepsync.cuh"

namespace ggp {
namespace {

// y[i] = sum_{m <= i} M[i][m] x[m] for the n0 x n0 lower-triangular M; one
// warp per row.  Optionally accumulates sum y_i^2 in FP64.
__global__ void dense_lower_matvec_kernel(const float* __restrict__ M, const float* __restrict__ x,
                                          float* __restrict__ y, int n0, double* __restrict__ sq) {
  int warps = (gridDim.x * blockDim.x) >> 5;
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int i = w; i < n0; i += warps) {
    const float* r = M + (int64_t)i * n0;
    float s = 0.0f;
    for (int m = lane; m <= i; m += 32) s = fmaf(r[m], x[m], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      y[i] = s;
      if (sq) atomicAdd(sq, (double)s * (double)s);
    }
  }
}

template <int KP>
struct Row {
  int4 n[KP / 4];
  float4 w[KP / 4];
};

template <int KP>
__device__ __forceinline__ void load_row(Row<KP>& r, const int32_t* __restrict__ nbr,
                                         const float* __restrict__ b, int64_t row, uint64_t pol) {
  const int4* np = reinterpret_cast<const int4*>(nbr + row * KP);
  const float4* bp = reinterpret_cast<const float4*>(b + row * KP);
#pragma unroll
  for (int q = 0; q < KP / 4; q++) {
    r.n[q] = ld_stream_i4(np + q, pol);
    r.w[q] = ld_stream_f4(bp + q, pol);
  }
}


// The same row, loaded without allocating in L1 (the whiten sweep keeps L1
// for the gathered field values of its tile).
template <int KP>
__device__ __forceinline__ void load_row_na(Row<KP>& r, const int32_t* __restrict__ nbr,
                                            const float* __restrict__ b, int64_t row,
                                            uint64_t pol) {
  const int4* np = reinterpret_cast<const int4*>(nbr + row * KP);
  const float4* bp = reinterpret_cast<const float4*>(b + row * KP);
#pragma unroll
  for (int q = 0; q < KP / 4; q++) {
    r.n[q] = ld_stream_na_i4(np + q, pol);
    r.w[q] = ld_stream_na_f4(bp + q, pol);
  }
}

// sum_a b_a v[c_a].  LEVEL: v is written level by level in the same launch;
// the gathered entries belong to earlier levels, published by the barrier.
template <int KP, bool LEVEL>
__device__ __forceinline__ float gather_dot(const Row<KP>& r, const float* __restrict__ v,
                                            uint64_t pol) {
  float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
  for (int q = 0; q < KP / 4; q++) {
    float v0, v1, v2, v3;
    if (LEVEL) {
      v0 = ld_level_f(v + r.n[q].x, pol); v1 = ld_level_f(v + r.n[q].y, pol);
      v2 = ld_level_f(v + r.n[q].z, pol); v3 = ld_level_f(v + r.n[q].w, pol);
    } else {
      v0 = ld_keep_f(v + r.n[q].x, pol); v1 = ld_keep_f(v + r.n[q].y, pol);
      v2 = ld_keep_f(v + r.n[q].z, pol); v3 = ld_keep_f(v + r.n[q].w, pol);
    }
    acc0 = fmaf(r.w[q].x, v0, acc0);
    acc1 = fmaf(r.w[q].y, v1, acc1);
    acc0 = fmaf(r.w[q].z, v2, acc0);
    acc1 = fmaf(r.w[q].w, v3, acc1);
  }
  return acc0 + acc1;
}

constexpr int kSweepThreads = 256;


// Positions per lane group and step of generate_kernel: as many as keep the
// two row buffers below about 64 registers.
__host__ __device__ constexpr int gen_steps(int hp) { return hp <= 4 ? 4 : (hp <= 8 ? 2 : 1); }

// Levels [l_first, l_end) of generate.  LANES threads share one position:
// lane h holds entries [h HP, (h+1) HP) of the row (HP = KP / LANES) and the
// partial sums meet in shuffles.  A lane group takes U positions per step,
// and the rows, sigma and xi of its next step are loaded before the gathers
// of the current one, so their DRAM latency hides under the gathers.  The
// first step of a level is loaded before the level's wait (rows do not depend
// on the field).
//   GRID: a cooperative launch; block b takes the b-th of gridDim.x equal
//         slices of every level and waits at the grid-wide level barrier.
//   !GRID: one block takes whole levels and waits at __syncthreads (levels
//         of a few hundred points, where the grid barrier would dominate).
template <int KP, int LANES, int U, int NT, bool GRID>
__device__ __forceinline__ void gen_levels(const int32_t* __restrict__ nbr,
                                           const float* __restrict__ b,
                                           const float* __restrict__ sigma,
                                           const float* __restrict__ xi, float* v,
                                           const int64_t* __restrict__ level_off, int l_first,
                                           int l_end, int64_t n0, const LevelBarrier& lb,
                                           int* s_flag) {
  constexpr int HP = KP / LANES;   // row entries per lane
  constexpr int GPB = NT / LANES;  // lane groups per block
  constexpr int PPB = U * GPB;     // positions per block step
  const uint64_t pol_rows = l2_evict_first();
  const uint64_t pol_v = l2_evict_last();
  const int h = threadIdx.x % LANES;
  const int slot = threadIdx.x / LANES;
  const int32_t* nb = nbr + h * HP;
  const float* bw = b + h * HP;
  Row<HP> rn[U];
  float sgn[U], xn[U];
  for (int l = l_first; l < l_end; l++) {
    const int64_t lo = level_off[l], n = level_off[l + 1] - lo;
    int64_t b0 = lo, hi = lo + n;
    if (GRID) {
      const int64_t per = (n + gridDim.x - 1) / gridDim.x;
      b0 = lo + min((int64_t)blockIdx.x * per, n);
      hi = lo + min((int64_t)(blockIdx.x + 1) * per, n);
    }
    int64_t p = b0 + slot;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t q = p + u * GPB;
      sgn[u] = xn[u] = 0.0f;
      if (q < hi) {
        load_row<HP>(rn[u], nb, bw, (q - n0) * LANES, pol_rows);
        if (h == 0) {
          sgn[u] = ld_stream_f(sigma + q, pol_rows);
          xn[u] = ld_stream_f(xi + q, pol_rows);
        }
      }
    }
    if (l > l_first) {
      if (GRID) {
        if (lb.wait(l - 1, gridDim.x, s_flag)) return;
      } else {
        __syncthreads();
      }
    }
    const int64_t steps = (hi - b0 + PPB - 1) / PPB;
    for (int64_t st = 0; st < steps; st++) {
      Row<HP> r[U];
      float sg[U], x[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        r[u] = rn[u];
        sg[u] = sgn[u];
        x[u] = xn[u];
      }
      const int64_t pn = p + PPB;
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t qn = pn + u * GPB;
        if (qn < hi) {
          load_row<HP>(rn[u], nb, bw, (qn - n0) * LANES, pol_rows);
          if (h == 0) {
            sgn[u] = ld_stream_f(sigma + qn, pol_rows);
            xn[u] = ld_stream_f(xi + qn, pol_rows);
          }
        }
      }
      float acc[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t q = p + u * GPB;
        acc[u] = q < hi ? gather_dot<HP, true>(r[u], v, pol_v) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (LANES >= 4) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 2);
        if (LANES >= 2) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 1);
        const int64_t q = p + u * GPB;
        if (q < hi && h == 0) st_keep_f(v + q, fmaf(sg[u], x[u], acc[u]), pol_v);
      }
      p = pn;
    }
    if (GRID) {
      __syncthreads();
      lb.arrive(l);
    }
  }
}

template <int KP, int LANES, int U>
__global__ void __launch_bounds__(kSweepThreads) generate_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ xi, float* v, const int64_t* __restrict__ level_off, int l_first,
    int l_end, int64_t n0, LevelBarrier lb) {
  __shared__ int s_flag;
  gen_levels<KP, LANES, U, kSweepThreads, true>(nbr, b, sigma, xi, v, level_off, l_first, l_end,
                                                n0, lb, &s_flag);
}

// One block of small_threads(KP) threads for runs of small levels.
__host__ __device__ constexpr int small_threads(int hp) { return hp <= 4 ? 1024 : (hp <= 8 ? 512 : 256); }
__host__ __device__ constexpr int small_steps(int hp) { return hp <= 8 ? 2 : 1; }

template <int KP, int LANES>
__global__ void __launch_bounds__(small_threads(KP / LANES), 1) generate_small_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ xi, float* v, const int64_t* __restrict__ level_off, int l_first,
    int l_end, int64_t n0) {
  constexpr int HP = KP / LANES;
  LevelBarrier none{nullptr, nullptr, 0};
  gen_levels<KP, LANES, small_steps(HP), small_threads(HP), false>(
      nbr, b, sigma, xi, v, level_off, l_first, l_end, n0, none, nullptr);
}

template <int KP>
__global__ void __launch_bounds__(256) whiten_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ v, float* __restrict__ xi, int64_t N, int64_t n0,
    double* __restrict__ sq) {
  const uint64_t pol_rows = l2_policy<0>();  // whiten: rows evict-normal (measured best)
  const uint64_t pol_v = l2_evict_last();
  double local = 0.0;
  for (int64_t pos = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < N;
       pos += (int64_t)gridDim.x * blockDim.x) {
    Row<KP> r;
    load_row<KP>(r, nbr, b, pos - n0, pol_rows);
    float sg = ld_stream_f(sigma + pos, pol_rows);
    float vi = ld_keep_f(v + pos, pol_v);
    float acc = gather_dot<KP, false>(r, v, pol_v);
    float out = (vi - acc) / sg;
    st_stream_f(xi + pos, out, pol_rows);
    if (sq) local += (double)out * (double)out;
  }
  if (sq) {
    __shared__ double red[8];
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
      atomicAdd(sq, s);
    }
  }
}

// whiten over spatial tiles: a block takes one tile (a k-d in-order rank range
// of kTileR points) and walks its positions in every level >= 1.  The gathers
// of a tile land mostly on the same tile's v values, which stay in L1.
template <int KP>
__global__ void __launch_bounds__(256) whiten_tiles_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ v, float* __restrict__ xi, int64_t n0,
    const int32_t* __restrict__ tile_start, int64_t n_tiles, int num_levels,
    double* __restrict__ sq) {
  extern __shared__ int32_t sm[];
  int32_t* s_start = sm;               // [num_levels]
  int32_t* s_pref = sm + num_levels;   // [num_levels + 1]
  __shared__ int32_t s_carry;
  const uint64_t pol_rows = l2_policy<0>();  // whiten: rows evict-normal (measured best)
  const uint64_t pol_v = l2_evict_last();
  double local = 0.0;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int32_t* ts = tile_start + t * num_levels;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    // exclusive prefix of the tile's counts over levels 1..L-1 (level 0 is dense)
    for (int base = 1; base < num_levels; base += blockDim.x) {
      int l = base + threadIdx.x;
      int32_t c = 0;
      if (l < num_levels) {
        int32_t a0 = ts[l];
        c = ts[num_levels + l] - a0;
        s_start[l] = a0;
      }
      // block-wide inclusive scan of c
      int32_t x = c;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
      }
      __shared__ int32_t wsum[8];
      if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
      __syncthreads();
      int32_t wpre = 0;
      for (int w = 0; w < (int)(threadIdx.x >> 5); w++) wpre += wsum[w];
      int32_t carry = s_carry;
      if (l < num_levels) s_pref[l] = carry + wpre + x - c;
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) s_carry = carry + wpre + x;
      __syncthreads();
    }
    const int32_t total = s_carry;
    // LANES lanes share a position; lane h holds row entries [h HP, (h+1) HP),
    // so a warp reads 32/LANES consecutive rows as whole sectors
    constexpr int LANES = gen_lanes(KP), HP = KP / LANES, GPB = 256 / LANES;
    const int h = threadIdx.x % LANES;
    const int32_t steps = (total + GPB - 1) / GPB;
    for (int32_t st = 0; st < steps; st++) {
      const int32_t vi = st * GPB + (int32_t)threadIdx.x / LANES;
      const bool act = vi < total;
      int64_t pos = 0;
      float acc = 0.0f;
      if (act) {
        // level of vi: last l >= 1 with s_pref[l] <= vi
        int lo = 1, hi = num_levels - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (s_pref[mid] <= vi) lo = mid; else hi = mid - 1;
        }
        pos = (int64_t)s_start[lo] + (vi - s_pref[lo]);
        Row<HP> r;
        load_row_na<HP>(r, nbr + h * HP, b + h * HP, (pos - n0) * LANES, pol_rows);
        acc = gather_dot<HP, false>(r, v, pol_v);
      }
      if (LANES >= 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (LANES >= 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (act && h == 0) {
        float sg = ld_stream_na_f(sigma + pos, pol_rows);
        float vv = ld_keep_f(v + pos, pol_v);
        float out = (vv - acc) / sg;
        st_stream_f(xi + pos, out, pol_rows);
        if (sq) local += (double)out * (double)out;
      }
    }
    __syncthreads();
  }
  if (sq) {
    __shared__ double red[8];
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
      atomicAdd(sq, s);
    }
  }
}

__global__ void nll_finish_kernel(const double* __restrict__ sq, const double* __restrict__ logdet,
                                  double* __restrict__ out) {
  out[0] = 0.5 * sq[0] + 0.5 * logdet[0];
}

template <int KP>
int launch_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi, float* v,
                    cudaStream_t s) {
  const int L = g->num_levels;
  if (L <= 1) return GRAPHGP_OK;
  constexpr int LANES = gen_lanes(KP), HP = KP / LANES, U = gen_steps(HP);
  // Runs of small levels at both ends of the sweep (a level that one block
  // covers in two steps) go to one block; the levels between them to the
  // cooperative grid.  Levels [1, a) and [z, L) are small.
  constexpr int64_t kSmall = 2 * small_steps(HP) * (small_threads(HP) / LANES);
  const std::vector<int64_t>& lo = g->level_off_h;
  int a = 1;
  while (a < L && lo[a + 1] - lo[a] <= kSmall) a++;
  int z = L;
  while (z > a && lo[z] - lo[z - 1] <= kSmall) z--;
  const int64_t* lod = g->level_off_d;
  int64_t n0 = g->n0;
  constexpr int NTS = small_threads(HP);
  if (a > 1) {
    generate_small_kernel<KP, LANES><<<1, NTS, 0, s>>>(g->nbr, f->b, f->sigma, xi, v, lod, 1, a,
                                                       n0);
    GGP_CUDA(cudaGetLastError());
  }
  if (a < z) {
    GGP_CUDA(cudaMemsetAsync(g->level_bar, 0, L * sizeof(uint32_t), s));
    auto kern = generate_kernel<KP, LANES, U>;
    static int max_grid_dev[kMaxDevices] = {};
    const int max_grid = coop_grid_cached(max_grid_dev, kern, kSweepThreads);
    int64_t want = (g->max_level_size + kSweepThreads - 1) / kSweepThreads;
    int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(want, 1));
    LevelBarrier lb{g->level_bar, g->err, g->max_spin};
    const int32_t* nbr = g->nbr;
    const float* bw = f->b;
    const float* sg = f->sigma;
    void* args[] = {(void*)&nbr, (void*)&bw, (void*)&sg, (void*)&xi, (void*)&v,
                    (void*)&lod, (void*)&a,  (void*)&z,  (void*)&n0, (void*)&lb};
    GGP_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kSweepThreads), args,
                                         0, s));
  }
  if (z < L) {
    generate_small_kernel<KP, LANES><<<1, NTS, 0, s>>>(g->nbr, f->b, f->sigma, xi, v, lod, z, L,
                                                       n0);
    GGP_CUDA(cudaGetLastError());
  }
  return GRAPHGP_OK;
}

template <int KP>
int launch_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
                  cudaStream_t s) {
  int64_t n = g->N - g->n0;
  if (n <= 0) return GRAPHGP_OK;
  if (g->tile_start && g->num_levels <= 8192) {
    size_t smem = (2 * (size_t)g->num_levels + 1) * sizeof(int32_t);
    GGP_CUDA(allow_dyn_smem(whiten_tiles_kernel<KP>, smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, whiten_tiles_kernel<KP>, 256, smem);
    int64_t grid = std::min<int64_t>(g->n_tiles, (int64_t)std::max(per_sm, 1) * num_sms());
    whiten_tiles_kernel<KP><<<(unsigned)grid, 256, smem, s>>>(
        g->nbr, f->b, f->sigma, v, xi, g->n0, g->tile_start, g->n_tiles, g->num_levels, sq);
  } else {
    whiten_kernel<KP><<<grid_for(n, 256, 8), 256, 0, s>>>(g->nbr, f->b, f->sigma, v, xi, g->N,
                                                          g->n0, sq);
  }
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

#define GGP_KP_DISPATCH(kp, call)            \
  switch (kp) {                              \
    case 4: call(4); break;                  \
    case 8: call(8); break;                  \
    case 12: call(12); break;                \
    case 16: call(16); break;                \
    case 20: call(20); break;                \
    case 24: call(24); break;                \
    case 28: call(28); break;                \
    case 32: call(32); break;                \
    case 48: call(48); break;                \
    default: call(64); break;                \
  }

}  // namespace

int dense_matvec(const float* M, const float* x, float* y, int n0, double* sq, cudaStream_t s) {
  dense_lower_matvec_kernel<<<(n0 + 7) / 8, 256, 0, s>>>(M, x, y, n0, sq);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

int run_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi, float* v,
                 cudaStream_t s) {
  int n0 = g->n0;
  dense_lower_matvec_kernel<<<(n0 + 7) / 8, 256, 0, s>>>(f->L0, xi, v, n0, nullptr);
  GGP_CUDA(cudaGetLastError());
  int rc = GRAPHGP_OK;
#define GGP_GEN(KP) rc = launch_generate<KP>(g, f, xi, v, s)
  GGP_KP_DISPATCH(g->kp, GGP_GEN)
#undef GGP_GEN
  return rc;
}

int run_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
               cudaStream_t s) {
  int n0 = g->n0;
  dense_lower_matvec_kernel<<<(n0 + 7) / 8, 256, 0, s>>>(f->L0inv, v, xi, n0, sq);
  GGP_CUDA(cudaGetLastError());
  int rc = GRAPHGP_OK;
#define GGP_WH(KP) rc = launch_whiten<KP>(g, f, v, xi, sq, s)
  GGP_KP_DISPATCH(g->kp, GGP_WH)
#undef GGP_WH
  return rc;
}

}  // namespace ggp

using namespace ggp;

static bool same_graph(graphgp_graph_t g, graphgp_factor_t f) {
  return g && f && f->g == g && f->row_end < 0;  // whole-graph factors only
}

extern "C" int graphgp_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi_d,
                                float* v_d, void* stream) {
  if (!same_graph(g, f) || !xi_d || !v_d) return GRAPHGP_ERR_INVALID;
  if (xi_d < v_d + g->N && v_d < xi_d + g->N) return GRAPHGP_ERR_INVALID;  // overlap
  return run_generate(g, f, xi_d, v_d, (cudaStream_t)stream);
}

extern "C" int graphgp_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                              float* xi_d, void* stream) {
  if (!same_graph(g, f) || !xi_d || !v_d) return GRAPHGP_ERR_INVALID;
  return run_whiten(g, f, v_d, xi_d, nullptr, (cudaStream_t)stream);
}

extern "C" int graphgp_logdet(graphgp_factor_t f, double* out_d, void* stream) {
  if (!f || !out_d) return GRAPHGP_ERR_INVALID;
  GGP_CUDA(cudaMemcpyAsync(out_d, f->logdet, sizeof(double), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return GRAPHGP_OK;
}

extern "C" int graphgp_nll(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                           double* out_d, void* stream) {
  if (!same_graph(g, f) || !v_d || !out_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* sq = nullptr;
  GGP_TRY(sc.alloc(&sq, 1));
  GGP_CUDA(cudaMemsetAsync(sq, 0, 8, s));
  GGP_TRY(run_whiten(g, f, v_d, g->tmp_vec, sq, s));
  nll_finish_kernel<<<1, 1, 0, s>>>(sq, f->logdet, out_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

extern "C" int graphgp_sync_status(graphgp_graph_t g, graphgp_factor_t f, void* stream,
                                   int64_t* n_not_pd) {
  GGP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  uint32_t err = 0;
  unsigned long long bad = 0;
  if (g) GGP_CUDA(cudaMemcpy(&err, g->err, 4, cudaMemcpyDeviceToHost));
  if (f) GGP_CUDA(cudaMemcpy(&bad, f->not_pd, 8, cudaMemcpyDeviceToHost));
  if (n_not_pd) *n_not_pd = (int64_t)bad;
  if (err & ERRBIT_TIMEOUT) return GRAPHGP_ERR_TIMEOUT;
  if (err & ERRBIT_INDEX) return GRAPHGP_ERR_INVALID;
  if (bad) return GRAPHGP_WARN_NOT_PD;
  return GRAPHGP_OK;
}

extern "C" const char* graphgp_status_string(int status) {
  switch (status) {
    case GRAPHGP_OK: return "ok";
    case GRAPHGP_ERR_INVALID: return "invalid argument";
    case GRAPHGP_ERR_OOM: return "device out of memory";
    case GRAPHGP_ERR_CUDA: return "CUDA runtime error";
    case GRAPHGP_ERR_TIMEOUT: return "bounded device wait timed out";
    case GRAPHGP_ERR_NAN: return "non-finite input";
    case GRAPHGP_ERR_IO: return "file error";
    case GRAPHGP_WARN_NOT_PD: return "pivots clamped (matrix not positive definite)";
  }
  return "unknown status";
}
