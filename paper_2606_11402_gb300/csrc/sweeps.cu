// Level sweeps of Alg. 1 (generate, v = L xi) and the inverse application
// and log-determinant of Sec. 3 (whiten, xi = L^-1 v; logdet; NLL).
//
// generate: v_0 = L0 xi_0 for the dense block, then for every position i of
// depth >= 1: v_i = b_i . v_c(i) + sigma_i xi_i, where every neighbour lies in
// an earlier depth level.  One persistent launch walks all levels without a
// grid barrier: blocks take chunks of 256 consecutive positions in order from
// a ticket counter, issue the loads of their rows (neighbour indices,
// weights, sigma, xi) at once, then wait until every chunk their rows depend
// on is complete -- a watermark W counts the leading complete chunks -- and
// then gather.  Chunks are claimed in increasing order and each depends only
// on earlier chunks, so the lowest unfinished chunk can always run.  Every
// wait is bounded; on expiry the kernel records ERR_TIMEOUT and all blocks
// leave.
//
// whiten: xi_i = (v_i - b_i . v_c(i)) / sigma_i has no dependencies; one
// streaming launch (plus xi_0 = L0^-1 v_0 for the dense block).
#include "common.cuh"

namespace ggp {
namespace {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_sc() { asm volatile("fence.sc.gpu;" ::: "memory"); }

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
                                         const float* __restrict__ b, int64_t row) {
  const int4* np = reinterpret_cast<const int4*>(nbr + row * KP);
  const float4* bp = reinterpret_cast<const float4*>(b + row * KP);
#pragma unroll
  for (int q = 0; q < KP / 4; q++) {
    r.n[q] = __ldcs(np + q);
    r.w[q] = __ldcs(bp + q);
  }
}

// sum_a b_a v[c_a]; gathered through L2 (.cg) because v is written by other
// blocks during the sweep.
template <int KP, bool COHERENT>
__device__ __forceinline__ float gather_dot(const Row<KP>& r, const float* __restrict__ v) {
  float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
  for (int q = 0; q < KP / 4; q++) {
    float v0, v1, v2, v3;
    if (COHERENT) {
      v0 = __ldcg(v + r.n[q].x); v1 = __ldcg(v + r.n[q].y);
      v2 = __ldcg(v + r.n[q].z); v3 = __ldcg(v + r.n[q].w);
    } else {
      v0 = __ldg(v + r.n[q].x); v1 = __ldg(v + r.n[q].y);
      v2 = __ldg(v + r.n[q].z); v3 = __ldg(v + r.n[q].w);
    }
    acc0 = fmaf(r.w[q].x, v0, acc0);
    acc1 = fmaf(r.w[q].y, v1, acc1);
    acc0 = fmaf(r.w[q].z, v2, acc0);
    acc1 = fmaf(r.w[q].w, v3, acc1);
  }
  return acc0 + acc1;
}

constexpr int kSweepThreads = kSweepChunk;  // one position per thread

template <int KP>
__global__ void __launch_bounds__(kSweepThreads) generate_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ xi, float* v, const int32_t* __restrict__ chunk_lo,
    const int32_t* __restrict__ chunk_hi, const int32_t* __restrict__ chunk_need,
    int64_t n_chunks, int64_t n0, uint32_t* sync, uint32_t* err, int64_t max_spin) {
  __shared__ int s_chunk;
  __shared__ int s_abort;
  uint32_t* ticket = sync;
  uint32_t* water = sync + 1;
  uint32_t* done = sync + 2;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) s_chunk = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t c = s_chunk;
    if (c >= n_chunks) break;
    const int32_t lo = chunk_lo[c], hi = chunk_hi[c];
    const uint32_t need = (uint32_t)chunk_need[c];
    const int64_t pos = (int64_t)lo + tid;
    const bool act = pos < hi;
    Row<KP> r;
    float sg = 0.0f, x = 0.0f;
    if (act) {
      load_row<KP>(r, nbr, b, pos - n0);
      sg = __ldcs(sigma + pos);
      x = __ldcs(xi + pos);
    }
    if (tid == 0) {
      int abort = 0;
      if (ld_acquire(water) < need) {
        int64_t spins = 0;
        while (ld_acquire(water) < need) {
          if (ld_acquire(err) & ERRBIT_TIMEOUT) {
            abort = 1;
            break;
          }
          if (++spins > max_spin) {
            atomicOr(err, ERRBIT_TIMEOUT);
            abort = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      s_abort = abort;
    }
    __syncthreads();
    if (s_abort) break;
    if (act) {
      float acc = gather_dot<KP, true>(r, v);
      __stcg(v + pos, fmaf(sg, x, acc));
    }
    __syncthreads();
    if (tid == 0) {
      fence_sc();
      st_release(done + c, 1u);
      fence_sc();
      // advance the watermark over the leading complete chunks
      uint32_t w = ld_acquire(water);
      uint32_t w0 = w;
      while (w < (uint32_t)n_chunks && ld_acquire(done + w)) w++;
      if (w > w0) atomicMax(water, w);
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(256) whiten_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ v, float* __restrict__ xi, int64_t N, int64_t n0,
    double* __restrict__ sq) {
  double local = 0.0;
  for (int64_t pos = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < N;
       pos += (int64_t)gridDim.x * blockDim.x) {
    Row<KP> r;
    load_row<KP>(r, nbr, b, pos - n0);
    float sg = __ldcs(sigma + pos);
    float vi = __ldcs(v + pos);
    float acc = gather_dot<KP, false>(r, v);
    float out = (vi - acc) / sg;
    __stcs(xi + pos, out);
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

__global__ void nll_finish_kernel(const double* __restrict__ sq, const double* __restrict__ logdet,
                                  double* __restrict__ out) {
  out[0] = 0.5 * sq[0] + 0.5 * logdet[0];
}

template <int KP>
int launch_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi, float* v,
                    cudaStream_t s) {
  if (g->n_chunks == 0) return GRAPHGP_OK;
  GGP_CUDA(cudaMemsetAsync(g->sweep_sync, 0, (2 + g->n_chunks) * sizeof(uint32_t), s));
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, generate_kernel<KP>,
                                                  kSweepThreads, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  int64_t grid = (int64_t)num_sms() * blocks_per_sm;
  if (grid > g->n_chunks) grid = g->n_chunks;
  generate_kernel<KP><<<(unsigned)grid, kSweepThreads, 0, s>>>(
      g->nbr, f->b, f->sigma, xi, v, g->chunk_lo, g->chunk_hi, g->chunk_need, g->n_chunks, g->n0,
      g->sweep_sync, g->err, g->max_spin);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int KP>
int launch_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
                  cudaStream_t s) {
  int64_t n = g->N - g->n0;
  if (n <= 0) return GRAPHGP_OK;
  whiten_kernel<KP><<<grid_for(n, 256, 8), 256, 0, s>>>(g->nbr, f->b, f->sigma, v, xi, g->N,
                                                        g->n0, sq);
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
    default: call(32); break;                \
  }

}  // namespace

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

static bool same_graph(graphgp_graph_t g, graphgp_factor_t f) { return g && f && f->g == g; }

extern "C" int graphgp_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi_d,
                                float* v_d, void* stream) {
  if (!same_graph(g, f) || !xi_d || !v_d) return GRAPHGP_ERR_INVALID;
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
