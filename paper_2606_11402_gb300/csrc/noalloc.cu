// graphgp_nll_noalloc: the negative log-likelihood of graphgp_nll computed
// without allocating any device memory during the call.
//
// graphgp_nll allocates an FP64 accumulator on every call and writes the
// whitened field into the graph's work vector.  Some callers cannot allocate
// while they run: a serving loop that reserved all device memory for resident
// graphs and factors up front, or code that must not pay cudaMalloc's
// device-wide synchronisation on a latency-critical path.  This variant keeps
// its reduction scratch in a file-scope device array instead: one FP64 slot
// per block of eight dense rows (up to 256) and one per whiten tile.  Every
// slot that is summed is written first in the same call, so nothing needs
// clearing, and the final sum runs in a fixed order (the result does not
// depend on block scheduling).
//
// The array is loaded with the library and held by every GPU that loads it
// until the process exits.  Its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) on the first call made on
// that device; make that first call before any stream capture.  All calls
// share the one array, so calls that overlap on the GPU race on it: do not
// run two of them concurrently (on different streams) on the same device.
#include <algorithm>
#include <mutex>

#include "sweepsync.cuh"

// Up to 256 slots for the dense block (eight rows each, n0 <= 2048) and one
// per whiten tile (at most 65536 tiles of 4096 points, i.e. N <= 2^28):
// 514 KiB.
static constexpr int kDenseSlots = 256;
static constexpr int kNllSlots = kDenseSlots + 65536;
static __device__ __align__(256) double g_nll_scratch[kNllSlots];

namespace ggp {
namespace {

std::mutex g_addr_mu;
double* g_addr[64] = {};

// Device address of g_nll_scratch on the current device (set up on first use).
int nll_scratch(double** out) {
  int dev = 0;
  GGP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GRAPHGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_nll_scratch);
    if (e != cudaSuccess) {
      std::fprintf(stderr, "graphgp_nll_noalloc: cudaGetSymbolAddress failed: %s\n",
                   cudaGetErrorString(e));
      return GRAPHGP_ERR_CUDA;
    }
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return GRAPHGP_OK;
}

// Fixed-order block sum of one double per thread (blockDim.x == 256).
__device__ double block_sum_fixed(double x) {
  __shared__ double red[256];
  red[threadIdx.x] = x;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// Dense block: slot[b] = sum over rows 8b..8b+7 of (L0^-1 v_0)_i^2; block b
// of 256 threads, one warp per row.
__global__ void nll_dense_slot_kernel(const float* __restrict__ W, const float* __restrict__ v,
                                      int n0, double* __restrict__ slot) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double local = 0.0;
  for (int i = blockIdx.x * 8 + w; i < n0 && i < (int)(blockIdx.x + 1) * 8; i += 8) {
    const float* r = W + (int64_t)i * n0;
    float s = 0.0f;
    for (int m = lane; m <= i; m += 32) s = fmaf(r[m], v[m], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) local += (double)s * (double)s;
  }
  double t = block_sum_fixed(local);
  if (threadIdx.x == 0) slot[blockIdx.x] = t;
}

// One tile per block iteration: slot[t] = sum over the tile's positions of
// xi_i^2, xi_i = (v_i - b_i . v_c(i)) / sigma_i.
template <int KP>
__global__ void __launch_bounds__(256) nll_tiles_slot_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ v, int64_t n0, const int32_t* __restrict__ tile_start,
    int64_t n_tiles, int num_levels, double* __restrict__ slot) {
  extern __shared__ int32_t sm[];
  int32_t* s_start = sm;
  int32_t* s_pref = sm + num_levels;
  __shared__ int32_t s_total;
  __shared__ int32_t wsum[8];
  const uint64_t pol_rows = l2_evict_first();
  const uint64_t pol_v = l2_evict_last();
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int32_t* ts = tile_start + t * num_levels;
    if (threadIdx.x == 0) s_total = 0;
    __syncthreads();
    // the tile's positions, level by level (levels >= 1; level 0 is dense):
    // exclusive prefix of the per-level counts, 256 levels per round
    for (int base = 1; base < num_levels; base += blockDim.x) {
      int l = base + threadIdx.x;
      int32_t c = 0;
      if (l < num_levels) {
        s_start[l] = ts[l];
        c = ts[num_levels + l] - ts[l];
      }
      int32_t x = c;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
      }
      if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
      __syncthreads();
      int32_t wpre = 0;
      for (int w = 0; w < (int)(threadIdx.x >> 5); w++) wpre += wsum[w];
      int32_t carry = s_total;
      if (l < num_levels) s_pref[l] = carry + wpre + x - c;
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) s_total = carry + wpre + x;
      __syncthreads();
    }
    const int32_t total = s_total;
    double local = 0.0;
    // the same lane split and summation order as the whiten sweep, so the
    // whitened values are bit-identical to graphgp_nll's
    constexpr int LANES = KP % 16 == 0 ? 4 : (KP % 8 == 0 ? 2 : 1);
    constexpr int HP = KP / LANES, GPB = 256 / LANES;
    const int h = threadIdx.x % LANES;
    const int32_t steps = (total + GPB - 1) / GPB;
    for (int32_t st = 0; st < steps; st++) {
      const int32_t vi = st * GPB + (int32_t)threadIdx.x / LANES;
      const bool act = vi < total;
      int64_t pos = 0;
      float acc = 0.0f;
      if (act) {
        int lo = 1, hi = num_levels - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (s_pref[mid] <= vi) lo = mid; else hi = mid - 1;
        }
        pos = (int64_t)s_start[lo] + (vi - s_pref[lo]);
        const int4* np = reinterpret_cast<const int4*>(nbr + (pos - n0) * KP + h * HP);
        const float4* bp = reinterpret_cast<const float4*>(b + (pos - n0) * KP + h * HP);
        int4 c[HP / 4];
        float4 w[HP / 4];
#pragma unroll
        for (int q = 0; q < HP / 4; q++) {
          c[q] = ld_stream_i4(np + q, pol_rows);
          w[q] = ld_stream_f4(bp + q, pol_rows);
        }
        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
        for (int q = 0; q < HP / 4; q++) {
          acc0 = fmaf(w[q].x, ld_keep_f(v + c[q].x, pol_v), acc0);
          acc1 = fmaf(w[q].y, ld_keep_f(v + c[q].y, pol_v), acc1);
          acc0 = fmaf(w[q].z, ld_keep_f(v + c[q].z, pol_v), acc0);
          acc1 = fmaf(w[q].w, ld_keep_f(v + c[q].w, pol_v), acc1);
        }
        acc = acc0 + acc1;
      }
      if (LANES >= 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (LANES >= 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (act && h == 0) {
        float sg = ld_stream_f(sigma + pos, pol_rows);
        float vv = ld_keep_f(v + pos, pol_v);
        float out = (vv - acc) / sg;
        local += (double)out * (double)out;
      }
    }
    double tsum = block_sum_fixed(local);
    if (threadIdx.x == 0) slot[t] = tsum;
  }
}

// out = 0.5 (sum of the nd dense slots and the nt tile slots) + 0.5 logdet,
// summed in a fixed order.
__global__ void nll_noalloc_finish_kernel(const double* __restrict__ slot, int nd, int64_t nt,
                                          const double* __restrict__ logdet,
                                          double* __restrict__ out) {
  double local = 0.0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) local += slot[i];
  for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) local += slot[kDenseSlots + i];
  double t = block_sum_fixed(local);
  if (threadIdx.x == 0) out[0] = 0.5 * t + 0.5 * logdet[0];
}

template <int KP>
int launch_tiles(graphgp_graph_t g, graphgp_factor_t f, const float* v, double* slot,
                 cudaStream_t s) {
  size_t smem = (2 * (size_t)g->num_levels + 1) * sizeof(int32_t);
  GGP_CUDA(allow_dyn_smem(nll_tiles_slot_kernel<KP>, smem));
  int per_sm = 0;
  GGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nll_tiles_slot_kernel<KP>, 256,
                                                         smem));
  int64_t grid = std::min<int64_t>(g->n_tiles, (int64_t)std::max(per_sm, 1) * num_sms());
  nll_tiles_slot_kernel<KP><<<(unsigned)grid, 256, smem, s>>>(
      g->nbr, f->b, f->sigma, v, g->n0, g->tile_start, g->n_tiles, g->num_levels, slot);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace
}  // namespace ggp

using namespace ggp;

extern "C" int graphgp_nll_noalloc(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                                   double* out_d, void* stream) {
  if (!g || !f || f->g != g || f->row_end >= 0 || !v_d || !out_d) return GRAPHGP_ERR_INVALID;
  if (!g->tile_start || g->num_levels > 8192) {
    std::fprintf(stderr, "graphgp_nll_noalloc: graph has %d depth levels; at most 8192 are "
                         "supported without allocation\n", g->num_levels);
    return GRAPHGP_ERR_INVALID;
  }
  const int64_t nt = g->N > g->n0 ? g->n_tiles : 0;
  const int nd = (g->n0 + 7) / 8;
  if (nt > kNllSlots - kDenseSlots || nd > kDenseSlots) {
    std::fprintf(stderr, "graphgp_nll_noalloc: N=%lld needs %lld tile slots; the static "
                         "scratch holds %d (N <= 2^28)\n",
                 (long long)g->N, (long long)nt, kNllSlots - kDenseSlots);
    return GRAPHGP_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* slot = nullptr;
  GGP_TRY(nll_scratch(&slot));
  nll_dense_slot_kernel<<<nd, 256, 0, s>>>(f->L0inv, v_d, g->n0, slot);
  GGP_CUDA(cudaGetLastError());
  if (nt > 0) {
    int rc = GRAPHGP_OK;
    double* tslot = slot + kDenseSlots;
    switch (g->kp) {
      case 4: rc = launch_tiles<4>(g, f, v_d, tslot, s); break;
      case 8: rc = launch_tiles<8>(g, f, v_d, tslot, s); break;
      case 12: rc = launch_tiles<12>(g, f, v_d, tslot, s); break;
      case 16: rc = launch_tiles<16>(g, f, v_d, tslot, s); break;
      case 20: rc = launch_tiles<20>(g, f, v_d, tslot, s); break;
      case 24: rc = launch_tiles<24>(g, f, v_d, tslot, s); break;
      case 28: rc = launch_tiles<28>(g, f, v_d, tslot, s); break;
      case 32: rc = launch_tiles<32>(g, f, v_d, tslot, s); break;
      case 48: rc = launch_tiles<48>(g, f, v_d, tslot, s); break;
      default: rc = launch_tiles<64>(g, f, v_d, tslot, s); break;
    }
    if (rc < 0) return rc;
  }
  nll_noalloc_finish_kernel<<<1, 256, 0, s>>>(slot, nd, nt, f->logdet, out_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}
