// On-the-fly sweeps (Alg. 1 as printed: the conditioning factor of every point
// recomputed inside the pass, nothing stored) for 16 < k <= 32: one warp per
// point, the factor of the 32-lane group form (point_factor_group, the same
// routine and rescue decision as the factor kernel for these k), so b and
// sigma are bit-identical to the stored factor's.  The dot b . v_c follows
// the stored sweeps' summation order: the row of kp entries cut into
// gen_lanes(kp) slices of HP entries, two alternating accumulators per slice
// over whole groups of four, slices combined as the stored sweep's xor
// shuffles do.  Lane h of the warp forms slice h from the weights of lanes
// h HP .. (h+1) HP - 1 (shuffled) and the row's neighbour indices (loaded),
// padding entries included (weight 0, index 0), exactly as the stored sweep
// reads the padded row.
//
// generate: one cooperative launch over the depth levels with the level
// barrier of the stored sweep; a warp factors its first point of a level
// before waiting at the barrier.  whiten: warps stride over the positions,
// optionally reducing xi.xi and sum log sigma_i^2 in FP64.
#include "pointfactor.cuh"
#include "sweepsync.cuh"

namespace ggp {
namespace {

constexpr int kGW = 4;  // warps per block
constexpr size_t kGWSmem = (size_t)kGW * 32 * 33 * sizeof(double);  // FP64 rescue workspaces

struct WarpFactor {
  float b;      // weight of this lane's neighbour (0 for lanes >= k)
  float sigma;  // same on every lane
  bool clamped;
};

// Factor of position i for the warp (lane a owns neighbour a), with the
// factor kernel's FP64 rescue decision and routine; Lg: the warp's
// shared-memory rows, W: its FP64 rescue workspace (32 x 33 doubles).
template <int KT>
__device__ __forceinline__ WarpFactor warp_factor(const float4* __restrict__ xs,
                                                  const int32_t* __restrict__ row, int64_t i,
                                                  int k, const KernF& kf, float* Lg, double* W) {
  const int a = threadIdx.x & 31;
  const int32_t ca = a < k ? __ldg(row + a) : 0;
  PointState<32> st;
  point_factor_group<32, KT>(st, a, k, kf, __ldg(xs + ca), __ldg(xs + i), Lg);
  __syncwarp();
  const bool lane_bad = a < k && !isfinite(st.b_own);
  const bool rescue = st.clamped || row_error_too_large(st.max_ratio, st.varw, st.sigma, kf) ||
                      !isfinite(st.sigma) || __ballot_sync(0xffffffffu, lane_bad);
  WarpFactor out{a < k ? st.b_own : 0.0f, st.sigma, st.clamped};
  if (rescue) {
    const WarpRow64 w = warp_row_factor64<32, KT>(xs, row, k, __ldg(xs + i), kf, W);
    out.b = a < k ? (float)w.b : 0.0f;
    out.sigma = (float)w.sigma;
    out.clamped = w.clamped;
  }
  return out;
}

__device__ inline void block_count(unsigned long long c, unsigned long long* out) {
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

template <int KP, int KT>
__global__ void __launch_bounds__(32 * kGW) whiten_fused_group_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, const float* __restrict__ v, float* __restrict__ xi, double* __restrict__ sq,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd) {
  __shared__ __align__(16) float Ls[kGW * PFLayout<32>::GS];
  extern __shared__ __align__(16) double gws[];  // kGW x 32 x 33 doubles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* Lg = Ls + warp * PFLayout<32>::GS;
  double* W = gws + warp * (32 * 33);
  const uint64_t pol_v = l2_evict_last();
  LogAcc lacc;
  double local = 0.0;
  unsigned long long clamped = 0;
  const int64_t npts = N - n0;
  for (int64_t t = (int64_t)blockIdx.x * kGW + warp; t < npts; t += (int64_t)gridDim.x * kGW) {
    const int64_t i = n0 + t;
    const int32_t* row = nbr + t * KP;
    const WarpFactor wf = warp_factor<KT>(xs, row, i, k, kf, Lg, W);
    const float acc = warp_dot_stored_order<KP, false>(wf.b, row, v, pol_v);
    if (lane == 0) {
      const float out = (ld_keep_f(v + i, pol_v) - acc) / wf.sigma;
      xi[i] = out;
      local += (double)out * (double)out;
      lacc.mul(wf.sigma);
      clamped += wf.clamped ? 1 : 0;
    }
  }
  if (sq) block_add_double(lane == 0 ? local : 0.0, sq);
  if (logdet) block_add_double(lane == 0 ? lacc.log_value() : 0.0, logdet);
  block_count(clamped, not_pd);
}

template <int KP, int KT>
__global__ void __launch_bounds__(32 * kGW) generate_fused_group_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int64_t n0, KernF kf,
    const float* __restrict__ xi, float* v, const int64_t* __restrict__ level_off,
    int num_levels, LevelBarrier lb, unsigned long long* __restrict__ not_pd) {
  __shared__ int s_flag;
  __shared__ __align__(16) float Ls[kGW * PFLayout<32>::GS];
  extern __shared__ __align__(16) double gws[];  // kGW x 32 x 33 doubles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* Lg = Ls + warp * PFLayout<32>::GS;
  double* W = gws + warp * (32 * 33);
  const uint64_t pol_v = l2_evict_last();
  unsigned long long clamped = 0;
  for (int l = 1; l < num_levels; l++) {
    const int64_t lo = level_off[l], n = level_off[l + 1] - lo;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = lo + min((int64_t)blockIdx.x * per, n);
    const int64_t hi = lo + min((int64_t)(blockIdx.x + 1) * per, n);
    const int64_t steps = (hi - b0 + kGW - 1) / kGW;
    if (steps == 0 && l > 1 && lb.wait(l - 1, gridDim.x, &s_flag)) return;
    for (int64_t st = 0; st < steps; st++) {
      const int64_t q = b0 + st * kGW + warp;
      const bool active = q < hi;  // uniform over the warp
      const int32_t* row = nbr + (active ? q - n0 : 0) * KP;
      WarpFactor wf{0.0f, 1.0f, false};
      if (active) wf = warp_factor<KT>(xs, row, active ? q : n0, k, kf, Lg, W);
      // the level's inputs are complete once every block arrived at l - 1
      if (st == 0 && l > 1 && lb.wait(l - 1, gridDim.x, &s_flag)) return;
      if (active) {
        const float acc = warp_dot_stored_order<KP, true>(wf.b, row, v, pol_v);
        if (lane == 0) {
          st_keep_f(v + q, fmaf(wf.sigma, xi[q], acc), pol_v);
          clamped += wf.clamped ? 1 : 0;
        }
      }
    }
    __syncthreads();
    lb.arrive(l);
  }
  block_count(clamped, not_pd);
}

template <int KP>
int whiten_group_kp(graphgp_graph_t g, int type, const KernF& kf, const float* v, float* xi,
                    double* sq, double* logdet, unsigned long long* not_pd, cudaStream_t s) {
  const int64_t npts = g->N - g->n0;
  if (npts <= 0) return GRAPHGP_OK;
  const unsigned grid = grid_for((npts + kGW - 1) / kGW * 32 * kGW, 32 * kGW, 16);
#define GGP_WG(KT)                                                                          \
  GGP_CUDA(cudaFuncSetAttribute(whiten_fused_group_kernel<KP, KT>,                          \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGWSmem)); \
  whiten_fused_group_kernel<KP, KT><<<grid, 32 * kGW, kGWSmem, s>>>(                        \
      g->xs, g->nbr, g->N, g->k, g->n0, kf, v, xi, sq, logdet, not_pd)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_WG(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_WG(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_WG(GRAPHGP_MATERN52); break;
    default: GGP_WG(GRAPHGP_SQEXP); break;
  }
#undef GGP_WG
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int KP, int KT>
int generate_group_kt(graphgp_graph_t g, const KernF& kf, const float* xi, float* v,
                      unsigned long long* not_pd, cudaStream_t s) {
  GGP_CUDA(cudaFuncSetAttribute(generate_fused_group_kernel<KP, KT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGWSmem));
  static int max_grid_dev[kMaxDevices] = {};
  const int max_grid =
      coop_grid_cached(max_grid_dev, generate_fused_group_kernel<KP, KT>, 32 * kGW, kGWSmem);
  const int64_t want = (g->max_level_size + kGW - 1) / kGW;
  const int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(want, 1));
  GGP_CUDA(cudaMemsetAsync(g->level_bar, 0, g->num_levels * sizeof(uint32_t), s));
  LevelBarrier lb{g->level_bar, g->err, g->max_spin};
  const float4* xs = g->xs;
  const int32_t* nbr = g->nbr;
  int k = g->k;
  int64_t n0 = g->n0;
  const int64_t* lo = g->level_off_d;
  int nl = g->num_levels;
  void* args[] = {(void*)&xs, (void*)&nbr, (void*)&k, (void*)&n0, (void*)&kf, (void*)&xi,
                  (void*)&v,  (void*)&lo,  (void*)&nl, (void*)&lb, (void*)&not_pd};
  GGP_CUDA(cudaLaunchCooperativeKernel((const void*)generate_fused_group_kernel<KP, KT>,
                                       dim3(grid), dim3(32 * kGW), args, kGWSmem, s));
  return GRAPHGP_OK;
}

template <int KP>
int generate_group_kp(graphgp_graph_t g, int type, const KernF& kf, const float* xi, float* v,
                      unsigned long long* not_pd, cudaStream_t s) {
  if (g->num_levels <= 1) return GRAPHGP_OK;
  switch (type) {
    case GRAPHGP_MATERN12: return generate_group_kt<KP, GRAPHGP_MATERN12>(g, kf, xi, v, not_pd, s);
    case GRAPHGP_MATERN32: return generate_group_kt<KP, GRAPHGP_MATERN32>(g, kf, xi, v, not_pd, s);
    case GRAPHGP_MATERN52: return generate_group_kt<KP, GRAPHGP_MATERN52>(g, kf, xi, v, not_pd, s);
    default: return generate_group_kt<KP, GRAPHGP_SQEXP>(g, kf, xi, v, not_pd, s);
  }
}

}  // namespace

// 16 < k <= 32 (row lengths 20, 24, 28, 32).
int whiten_fused_group(graphgp_graph_t g, int type, const KernF& kf, const float* v, float* xi,
                       double* sq, double* logdet, unsigned long long* not_pd, cudaStream_t s) {
  switch (g->kp) {
    case 20: return whiten_group_kp<20>(g, type, kf, v, xi, sq, logdet, not_pd, s);
    case 24: return whiten_group_kp<24>(g, type, kf, v, xi, sq, logdet, not_pd, s);
    case 28: return whiten_group_kp<28>(g, type, kf, v, xi, sq, logdet, not_pd, s);
    default: return whiten_group_kp<32>(g, type, kf, v, xi, sq, logdet, not_pd, s);
  }
}

int generate_fused_group(graphgp_graph_t g, int type, const KernF& kf, const float* xi, float* v,
                         unsigned long long* not_pd, cudaStream_t s) {
  switch (g->kp) {
    case 20: return generate_group_kp<20>(g, type, kf, xi, v, not_pd, s);
    case 24: return generate_group_kp<24>(g, type, kf, xi, v, not_pd, s);
    case 28: return generate_group_kp<28>(g, type, kf, xi, v, not_pd, s);
    default: return generate_group_kp<32>(g, type, kf, xi, v, not_pd, s);
  }
}

}  // namespace ggp
