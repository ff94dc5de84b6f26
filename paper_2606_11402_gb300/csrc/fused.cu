// On-the-fly sweeps: Alg. 1 as printed, with the conditioning factor of
// every point (Sec. 2.1 Eq. 2) recomputed inside the pass from the
// coordinates and the kernel parameters and never stored.  No factor handle
// exists, so the device holds the graph alone (k + 4 words per point instead
// of 2k + 5 with stored weights); this is the form for kernel parameters that
// change at every step.
//
// Each thread owns one point and runs point_factor_thread (k <= 16; 16 < k
// <= 32 in fused_group.cu) with the same FP64 rescue decision as the factor
// kernel, so b and sigma are bit-identical to the stored factor's; the dot b . v_c then
// follows the stored sweeps' summation order (the row cut into gen_lanes(K)
// slices, two alternating accumulators per slice, slices combined as their
// xor-shuffle tree does), so the fused sweeps return the same bits as
// factor + generate / whiten.
//
// generate: one cooperative launch over the depth levels with the level
// barrier of the stored sweep; a thread computes the factor of its first
// point of a level before waiting at the barrier, so the factor work of
// level l overlaps the end of level l - 1.  whiten: one grid-stride launch in
// position order (no dependencies), optionally reducing xi.xi and
// sum log sigma_i^2 in FP64.
#include "pointfactor.cuh"
#include "sweepsync.cuh"

namespace ggp {
namespace {

template <int K, int KT>
__device__ __forceinline__ void factor_at(PointRegs<K>& p, const ThreadStage<K>& st,
                                          const float4* __restrict__ xs, const int32_t* row,
                                          int64_t i, int k, const KernF& kf) {
  const float4 xq = __ldg(xs + i);
  stage_coords<K>(st, xs, row, k);
  point_factor_thread<K, KT>(p, k, kf, st, xq);
}

__device__ inline void block_add_count(unsigned long long c, unsigned long long* out) {
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

template <int K, int KT>
__global__ void __launch_bounds__(128) whiten_fused_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, const float* __restrict__ v, float* __restrict__ xi, double* __restrict__ sq,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd) {
  extern __shared__ __align__(16) unsigned char tstage[];
  const ThreadStage<K> stg(tstage);
  double* W = fused_rescue_ws<K>(tstage);
  const uint64_t pol_v = l2_evict_last();
  LogAcc lacc;
  double local = 0.0;
  unsigned long long clamped = 0;
  const int64_t npts = N - n0;
  const int64_t total = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (npts + total - 1) / total;  // the same on every lane
  for (int64_t it = 0; it < iters; it++) {
    const int64_t t = it * total + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = t < npts;
    const int64_t i = n0 + (valid ? t : 0);
    const int32_t* row = nbr + (valid ? t : 0) * K;
    PointRegs<K> p;
    if (valid) factor_at<K, KT>(p, stg, xs, row, i, k, kf);
    warp_rescue<K, KT>(p, valid && needs_rescue(p, k, kf), xs, row, k, __ldg(xs + i), kf, W);
    if (!valid) continue;
    const float acc = dot_stored_order<K, false>(p.y, row, v, pol_v);
    const float out = (ld_keep_f(v + i, pol_v) - acc) / p.sigma;
    xi[i] = out;
    local += (double)out * (double)out;
    lacc.mul(p.sigma);
    clamped += p.clamped ? 1 : 0;
  }
  if (sq) block_add_double(local, sq);
  if (logdet) block_add_double(lacc.log_value(), logdet);
  block_add_count(clamped, not_pd);
}

template <int K, int KT>
__global__ void __launch_bounds__(128) generate_fused_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int64_t n0, KernF kf,
    const float* __restrict__ xi, float* v, const int64_t* __restrict__ level_off,
    int num_levels, LevelBarrier lb, unsigned long long* __restrict__ not_pd) {
  __shared__ int s_flag;
  extern __shared__ __align__(16) unsigned char tstage[];
  const ThreadStage<K> stg(tstage);
  double* W = fused_rescue_ws<K>(tstage);
  const uint64_t pol_v = l2_evict_last();
  unsigned long long clamped = 0;
  for (int l = 1; l < num_levels; l++) {
    const int64_t lo = level_off[l], n = level_off[l + 1] - lo;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = lo + min((int64_t)blockIdx.x * per, n);
    const int64_t hi = lo + min((int64_t)(blockIdx.x + 1) * per, n);
    const int64_t steps = (hi - b0 + blockDim.x - 1) / blockDim.x;
    if (steps == 0 && l > 1 && lb.wait(l - 1, gridDim.x, &s_flag)) return;
    for (int64_t st = 0; st < steps; st++) {
      const int64_t q = b0 + st * blockDim.x + threadIdx.x;
      const bool active = q < hi;
      const int32_t* row = nbr + (active ? q - n0 : 0) * K;
      PointRegs<K> p;
      if (active) factor_at<K, KT>(p, stg, xs, row, q, k, kf);
      warp_rescue<K, KT>(p, active && needs_rescue(p, k, kf), xs, row, k,
                         __ldg(xs + (active ? q : n0)), kf, W);
      // the level's inputs are complete once every block arrived at l - 1
      if (st == 0 && l > 1 && lb.wait(l - 1, gridDim.x, &s_flag)) return;
      if (active) {
        const float acc = dot_stored_order<K, true>(p.y, row, v, pol_v);
        st_keep_f(v + q, fmaf(p.sigma, xi[q], acc), pol_v);
        clamped += p.clamped ? 1 : 0;
      }
    }
    __syncthreads();
    lb.arrive(l);
  }
  block_add_count(clamped, not_pd);
}

__global__ void nll_fused_finish_kernel(const double* __restrict__ sq,
                                        const double* __restrict__ logdet,
                                        double* __restrict__ out) {
  out[0] = 0.5 * sq[0] + 0.5 * logdet[0];
}

}  // namespace

bool valid_kernel(const graphgp_kernel* kern) {
  return kern && kern->type >= 0 && kern->type <= 3 && kern->sigma2 > 0 &&
         kern->lengthscale > 0 && kern->nugget >= 0 && std::isfinite(kern->rescue_tol);
}

// Dense block of the fused forms into a temporary handle whose arrays live in
// the call's scratch: L0, L0^-1, sigma_0..n0-1; the block's log-determinant
// is added to *logdet and its floored pivots to *not_pd.
int dense_into(graphgp_graph_t g, const graphgp_kernel* kern, Scratch& sc, double* logdet,
               unsigned long long* not_pd, graphgp_factor_s& f, cudaStream_t s) {
  const int64_t nn = (int64_t)g->n0 * g->n0;
  f.g = g;
  f.kern = *kern;
  GGP_TRY(sc.alloc(&f.L0, nn));
  GGP_TRY(sc.alloc(&f.L0inv, nn));
  GGP_TRY(sc.alloc(&f.sigma, g->n0));
  f.logdet = logdet;
  f.not_pd = not_pd;
  return dense_factor(g, &f, make_kernf(*kern), kern->type, s);
}

namespace {

template <int K>
int launch_whiten_fused(graphgp_graph_t g, int type, const KernF& kf, const float* v, float* xi,
                        double* sq, double* logdet, unsigned long long* not_pd, cudaStream_t s) {
  const int64_t npts = g->N - g->n0;
  if (npts <= 0) return GRAPHGP_OK;
  const unsigned grid = grid_for(npts, kThreadBlock, 8);
  constexpr size_t smem = fused_smem<K>();
#define GGP_WF(KT)                                                                            \
  GGP_CUDA(allow_dyn_smem(whiten_fused_kernel<K, KT>, smem));                                 \
  whiten_fused_kernel<K, KT><<<grid, kThreadBlock, smem, s>>>(g->xs, g->nbr, g->N, g->k, g->n0, \
                                                              kf, v, xi, sq, logdet, not_pd)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_WF(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_WF(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_WF(GRAPHGP_MATERN52); break;
    default: GGP_WF(GRAPHGP_SQEXP); break;
  }
#undef GGP_WF
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int K, int KT>
int launch_generate_fused_kt(graphgp_graph_t g, const KernF& kf, const float* xi, float* v,
                             unsigned long long* not_pd, cudaStream_t s) {
  constexpr size_t smem = fused_smem<K>();
  GGP_CUDA(allow_dyn_smem(generate_fused_kernel<K, KT>, smem));
  static int max_grid_dev[kMaxDevices] = {};
  const int max_grid = coop_grid_cached(max_grid_dev, generate_fused_kernel<K, KT>, kThreadBlock, smem);
  const int64_t want = (g->max_level_size + 127) / 128;
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
  GGP_CUDA(cudaLaunchCooperativeKernel((const void*)generate_fused_kernel<K, KT>, dim3(grid),
                                       dim3(kThreadBlock), args, smem, s));
  return GRAPHGP_OK;
}

template <int K>
int launch_generate_fused(graphgp_graph_t g, int type, const KernF& kf, const float* xi, float* v,
                          unsigned long long* not_pd, cudaStream_t s) {
  if (g->num_levels <= 1) return GRAPHGP_OK;
  switch (type) {
    case GRAPHGP_MATERN12: return launch_generate_fused_kt<K, GRAPHGP_MATERN12>(g, kf, xi, v, not_pd, s);
    case GRAPHGP_MATERN32: return launch_generate_fused_kt<K, GRAPHGP_MATERN32>(g, kf, xi, v, not_pd, s);
    case GRAPHGP_MATERN52: return launch_generate_fused_kt<K, GRAPHGP_MATERN52>(g, kf, xi, v, not_pd, s);
    default: return launch_generate_fused_kt<K, GRAPHGP_SQEXP>(g, kf, xi, v, not_pd, s);
  }
}

#define GGP_FUSED_DISPATCH(call) \
  switch (g->kp) {               \
    case 4: call(4); break;      \
    case 8: call(8); break;      \
    case 12: call(12); break;    \
    default: call(16); break;    \
  }

int whiten_fused(graphgp_graph_t g, const graphgp_kernel* kern, const float* v, float* xi,
                 double* sq, double* logdet, unsigned long long* not_pd, cudaStream_t s) {
  Scratch sc(s);
  graphgp_factor_s f;
  int rc = dense_into(g, kern, sc, logdet, not_pd, f, s);
  if (rc == GRAPHGP_OK) rc = dense_matvec(f.L0inv, v, xi, g->n0, sq, s);
  if (rc == GRAPHGP_OK) {
    const KernF kf = make_kernf(*kern);
    if (g->kp > 16) return whiten_fused_group(g, kern->type, kf, v, xi, sq, logdet, not_pd, s);
#define GGP_CALL(K) rc = launch_whiten_fused<K>(g, kern->type, kf, v, xi, sq, logdet, not_pd, s)
    GGP_FUSED_DISPATCH(GGP_CALL)
#undef GGP_CALL
  }
  return rc;
}

}  // namespace
}  // namespace ggp

using namespace ggp;

static bool fused_ok(graphgp_graph_t g, const graphgp_kernel* kern) {
  return g && valid_kernel(kern) && g->k <= 32;
}

extern "C" int graphgp_generate_fused(graphgp_graph_t g, const graphgp_kernel* kern,
                                      const float* xi_d, float* v_d, uint64_t* not_pd_d,
                                      void* stream) {
  if (!fused_ok(g, kern) || !xi_d || !v_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* ld = nullptr;
  unsigned long long* bad = (unsigned long long*)not_pd_d;
  GGP_TRY(sc.alloc(&ld, 1));
  GGP_CUDA(cudaMemsetAsync(ld, 0, 8, s));
  if (!bad) {
    GGP_TRY(sc.alloc(&bad, 1));
    GGP_CUDA(cudaMemsetAsync(bad, 0, 8, s));
  }
  graphgp_factor_s f;
  int rc = dense_into(g, kern, sc, ld, bad, f, s);
  if (rc == GRAPHGP_OK) rc = dense_matvec(f.L0, xi_d, v_d, g->n0, nullptr, s);
  if (rc == GRAPHGP_OK) {
    const KernF kf = make_kernf(*kern);
    if (g->kp > 16) return generate_fused_group(g, kern->type, kf, xi_d, v_d, bad, s);
#define GGP_CALL(K) rc = launch_generate_fused<K>(g, kern->type, kf, xi_d, v_d, bad, s)
    GGP_FUSED_DISPATCH(GGP_CALL)
#undef GGP_CALL
  }
  return rc;
}

extern "C" int graphgp_whiten_fused(graphgp_graph_t g, const graphgp_kernel* kern,
                                    const float* v_d, float* xi_d, double* logdet_d,
                                    uint64_t* not_pd_d, void* stream) {
  if (!fused_ok(g, kern) || !v_d || !xi_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* ld = logdet_d;
  unsigned long long* bad = (unsigned long long*)not_pd_d;
  if (!ld) GGP_TRY(sc.alloc(&ld, 1));
  if (!bad) {
    GGP_TRY(sc.alloc(&bad, 1));
    GGP_CUDA(cudaMemsetAsync(bad, 0, 8, s));
  }
  GGP_CUDA(cudaMemsetAsync(ld, 0, 8, s));
  return whiten_fused(g, kern, v_d, xi_d, nullptr, ld, bad, s);
}

extern "C" int graphgp_nll_fused(graphgp_graph_t g, const graphgp_kernel* kern, const float* v_d,
                                 double* nll_d, uint64_t* not_pd_d, void* stream) {
  if (!fused_ok(g, kern) || !v_d || !nll_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* acc = nullptr;  // [0] xi.xi, [1] logdet
  unsigned long long* bad = (unsigned long long*)not_pd_d;
  GGP_TRY(sc.alloc(&acc, 2));
  GGP_CUDA(cudaMemsetAsync(acc, 0, 16, s));
  if (!bad) {
    GGP_TRY(sc.alloc(&bad, 1));
    GGP_CUDA(cudaMemsetAsync(bad, 0, 8, s));
  }
  GGP_TRY(whiten_fused(g, kern, v_d, g->tmp_vec, acc, acc + 1, bad, s));
  nll_fused_finish_kernel<<<1, 1, 0, s>>>(acc, acc + 1, nll_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}
