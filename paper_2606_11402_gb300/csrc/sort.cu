// Device-wide exclusive scan and stable LSD radix sort of (key, value) pairs.
// Used by the k-d tree build (per-dimension presort, Sec. 2.3 "sort-based
// tree build") and the depth sort (Sec. 2.2 "Batch construction").  Stability makes every result deterministic: equal keys
// keep their input order.
#include "common.cuh"

namespace ggp {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 elements per block

__device__ __forceinline__ int pad(int x) { return x + (x >> 5); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kThreads / 32) warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  uint32_t warp_prefix = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kThreads / 32 - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                   uint32_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t idx = base + i * kThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_apply_kernel(const uint32_t* __restrict__ in,
                                  uint32_t* __restrict__ out, int64_t n,
                                  const uint32_t* __restrict__ block_off) {
  __shared__ uint32_t tile[kTile + kTile / 32];
  int64_t base = (int64_t)blockIdx.x * kTile;
  int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t idx = base + i * kThreads + t;
    tile[pad(i * kThreads + t)] = idx < n ? in[idx] : 0u;
  }
  __syncthreads();
  uint32_t v[kItems];
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    v[i] = run;
    run += tile[pad(t * kItems + i)];
  }
  uint32_t total;
  uint32_t pre = block_exclusive_scan(run, &total);
  uint32_t off = block_off ? block_off[blockIdx.x] : 0u;
#pragma unroll
  for (int i = 0; i < kItems; i++) tile[pad(t * kItems + i)] = v[i] + pre + off;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t idx = base + i * kThreads + t;
    if (idx < n) out[idx] = tile[pad(i * kThreads + t)];
  }
}

__global__ void rs_hist_kernel(const uint32_t* __restrict__ keys, int64_t n,
                               int shift, uint32_t* __restrict__ hist,
                               int64_t nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t idx = base + i * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: element order inside a tile is (round, warp, lane), which is
// the input order, and ranks are assigned in that order.
__global__ void rs_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                  const uint32_t* __restrict__ vals_in,
                                  uint32_t* __restrict__ keys_out,
                                  uint32_t* __restrict__ vals_out, int64_t n,
                                  int shift,
                                  const uint32_t* __restrict__ offs,
                                  int64_t nblocks) {
  __shared__ uint32_t base_off[256];
  __shared__ uint32_t running[256];
  __shared__ uint32_t cnt[kThreads / 32][256];
  __shared__ uint32_t pre[kThreads / 32][256];
  int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  base_off[t] = offs[(int64_t)t * nblocks + blockIdx.x];
  running[t] = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; w++) cnt[w][t] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t lt = lanemask_lt();
  for (int i = 0; i < kItems; i++) {
    int64_t idx = base + i * kThreads + t;
    bool valid = idx < n;
    uint32_t key = valid ? keys_in[idx] : 0u;
    uint32_t val = valid ? vals_in[idx] : 0u;
    uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    if (valid && lane == leader) cnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = running[t];
#pragma unroll
      for (int w = 0; w < kThreads / 32; w++) {
        uint32_t c = cnt[w][t];
        pre[w][t] = run;
        cnt[w][t] = 0;
        run += c;
      }
      running[t] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base_off[d] + pre[warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
  }
}

}  // namespace

int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n,
                       cudaStream_t s) {
  if (n <= 0) return GRAPHGP_OK;
  int64_t nb = (n + kTile - 1) / kTile;
  if (nb == 1) {
    scan_apply_kernel<<<1, kThreads, 0, s>>>(in, out, n, nullptr);
    GGP_CUDA(cudaGetLastError());
    return GRAPHGP_OK;
  }
  Scratch sc(s);
  uint32_t *sums = nullptr, *offs = nullptr;
  GGP_TRY(sc.alloc(&sums, nb));
  GGP_TRY(sc.alloc(&offs, nb));
  scan_reduce_kernel<<<(unsigned)nb, kThreads, 0, s>>>(in, n, sums);
  GGP_CUDA(cudaGetLastError());
  GGP_TRY(scan_exclusive_u32(sums, offs, nb, s));
  scan_apply_kernel<<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, offs);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

int radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in,
                     uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                     int bits, cudaStream_t s) {
  if (n <= 0) return GRAPHGP_OK;
  if (n >= (int64_t)1 << 32) return GRAPHGP_ERR_INVALID;
  int passes = (bits + 7) / 8;
  if (passes <= 0) {
    GGP_CUDA(cudaMemcpyAsync(keys_out, keys_in, n * 4, cudaMemcpyDeviceToDevice, s));
    GGP_CUDA(cudaMemcpyAsync(vals_out, vals_in, n * 4, cudaMemcpyDeviceToDevice, s));
    return GRAPHGP_OK;
  }
  int64_t nb = (n + kTile - 1) / kTile;
  Scratch sc(s);
  uint32_t *tk = nullptr, *tv = nullptr, *hist = nullptr, *offs = nullptr;
  GGP_TRY(sc.alloc(&tk, n));
  GGP_TRY(sc.alloc(&tv, n));
  GGP_TRY(sc.alloc(&hist, 256 * nb));
  GGP_TRY(sc.alloc(&offs, 256 * nb));
  const uint32_t* sk = keys_in;
  const uint32_t* sv = vals_in;
  for (int p = 0; p < passes; p++) {
    bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* dk = to_out ? keys_out : tk;
    uint32_t* dv = to_out ? vals_out : tv;
    rs_hist_kernel<<<(unsigned)nb, kThreads, 0, s>>>(sk, n, 8 * p, hist, nb);
    GGP_CUDA(cudaGetLastError());
    GGP_TRY(scan_exclusive_u32(hist, offs, 256 * nb, s));
    rs_scatter_kernel<<<(unsigned)nb, kThreads, 0, s>>>(sk, sv, dk, dv, n, 8 * p, offs, nb);
    GGP_CUDA(cudaGetLastError());
    sk = dk;
    sv = dv;
  }
  return GRAPHGP_OK;
}

}  // namespace ggp
