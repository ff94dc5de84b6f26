// Adjoints (Sec. 2.3: forward and backward derivatives of the conditioning
// steps, differentiated through the Cholesky factor).
//
// With every sparse row written as v_i = b_i . v_c(i) + sigma_i xi_i:
//  * whiten VJP (xi = L^-1 v, cotangent xibar, logdetbar), w_i = xibar_i/sigma_i:
//      vbar_i = w_i - sum over children (j, a) of i of w_j b_ja   (every row
//      j scatters -w_j b_ja to its neighbours), bbar_i = -w_i v_c, sigbar_i =
//      -w_i xi_i + 2 logdetbar / sigma_i;
//  * generate VJP (v = L xi, cotangent vbar): u = (I - B)^-T vbar by a reverse
//      level sweep, u_j = vbar_j + sum over children (i, a) of j of b_ia u_i
//      (every row i, once u_i is complete, scatters b_ia u_i to its
//      neighbours); xibar_i = sigma_i u_i, bbar_i = u_i v_c, sigbar_i = u_i xi_i;
//  * factor backward, per row, from b = K_cc^-1 K_ci and s = sigma^2:
//      sbar = sigbar/(2 sigma), g = K_cc^-1 bbar, Kbar_cc = -g b^T + sbar b b^T,
//      Kbar_ci = g - 2 sbar b, Kbar_ii = sbar, theta_bar += sum Kbar dK/dtheta.
//    The factors are recomputed (bit-identical to the forward), not stored.
//  * dense block (L0 = chol(K_00)): Lbar0 from the sweep, then
//      Kbar_00 = L0^-T Phi(L0^T Lbar0) L0^-1 (Phi: lower triangle, halved
//      diagonal), theta_bar += sum Kbar_00 dK_00/dtheta.
//  * NLL value and gradient in one pass (graphgp_nll_grad_fused): per row the
//      factor, xi_i, the value's terms, the whiten-VJP scatter and the
//      factor backward above, each conditional computed once.
// theta = (lengthscale, sigma2, nugget); theta_bar is accumulated in FP64.
#include <algorithm>

#include "pointwide.cuh"
#include "sweepsync.cuh"

namespace ggp {
namespace {

// ---- dense helpers ------------------------------------------------------------
// y_m = sum_{i >= m} M[i][m] x_i (transpose of a lower-triangular n0 x n0 M)
__global__ void dense_lower_tmatvec_kernel(const float* __restrict__ M, const float* __restrict__ x,
                                           float* __restrict__ y, int n0) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n0; m += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = m; i < n0; i++) s = fmaf(M[(int64_t)i * n0 + m], x[i], s);
    y[m] = s;
  }
}

// Lbar0[a][b] = sgn * u_a xi_b (b <= a) plus diag 2 logdetbar / L0_aa.
__global__ void dense_lbar_kernel(const float* __restrict__ u, const float* __restrict__ xi,
                                  const float* __restrict__ L0, int n0, float sgn, float ldbar,
                                  float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n0 * n0;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(e / n0), b = (int)(e % n0);
    float v = 0.0f;
    if (b <= a) v = sgn * u[a] * xi[b];
    if (a == b) v += 2.0f * ldbar / L0[e];
    out[e] = v;
  }
}

// C = op(A) B for n x n row-major matrices; op(A) = A^T when transA.  If phi,
// keeps the lower triangle of the result with the diagonal halved.
__global__ void dense_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                  float* __restrict__ C, int n, int transA, int phi) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(e / n), b = (int)(e % n);
    if (phi && b > a) {
      C[e] = 0.0f;
      continue;
    }
    float s = 0.0f;
    if (transA)
      for (int m = 0; m < n; m++) s = fmaf(A[(int64_t)m * n + a], B[(int64_t)m * n + b], s);
    else
      for (int m = 0; m < n; m++) s = fmaf(A[(int64_t)a * n + m], B[(int64_t)m * n + b], s);
    if (phi && a == b) s *= 0.5f;
    C[e] = s;
  }
}

__device__ void block_add3(double t0, double t1, double t2, double* out) {
  __shared__ double red[3][32];
  for (int o = 16; o; o >>= 1) {
    t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    t2 += __shfl_xor_sync(0xffffffffu, t2, o);
  }
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = t0;
    red[1][w] = t1;
    red[2][w] = t2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
      s0 += red[0][i];
      s1 += red[1][i];
      s2 += red[2][i];
    }
    atomicAdd(out + 0, s0);
    atomicAdd(out + 1, s1);
    atomicAdd(out + 2, s2);
  }
  __syncthreads();  // the partials may be reused by a following call
}

// theta_bar += sum_{a,b} Kbar[a][b] dK_ab/dtheta over the dense block.
template <int KT>
__global__ void dense_theta_kernel(const float* __restrict__ Kbar, const float4* __restrict__ xs,
                                   int n0, KernF kf, double* __restrict__ thetabar) {
  double tl = 0, ts = 0, tn = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n0 * n0;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(e / n0), b = (int)(e % n0);
    float kb = Kbar[e];
    if (a == b) {
      ts += kb;
      tn += kb;
    } else {
      float d2 = sqdist(xs[a], xs[b]);
      ts += (double)(kb * kappa_d2<KT>(kf, d2) / kf.s2);
      tl += (double)(kb * dkappa_dell_d2<KT>(kf, d2));
    }
  }
  block_add3(tl, ts, tn, thetabar);
}

// ---- adjoint sweeps by scatter ------------------------------------------------
// Both VJPs apply a transpose of the row operator: entry b_ia of row i moves
// a cotangent from position i to its neighbour c_a.  Rows are streamed in
// position order, LANES threads per row as in the forward sweeps (16-byte
// row loads), and each entry's contribution is added at its neighbour with a
// fire-and-forget atomic add in L2 (red.global.add.f32).  The additions into
// one position arrive in no fixed order, so results agree with the ordered
// sums to rounding, not bit for bit.
#define GGP_ADJ_KP_DISPATCH(kp, call) \
  switch (kp) {                       \
    case 4: call(4); break;           \
    case 8: call(8); break;           \
    case 12: call(12); break;         \
    case 16: call(16); break;         \
    case 20: call(20); break;         \
    case 24: call(24); break;         \
    case 28: call(28); break;         \
    case 32: call(32); break;         \
    case 48: call(48); break;         \
    default: call(64); break;         \
  }

template <int HP>
__device__ __forceinline__ void load_row_slice(int4 (&n)[HP / 4], float4 (&w)[HP / 4],
                                               const int32_t* __restrict__ nbr,
                                               const float* __restrict__ b, int64_t off,
                                               uint64_t pol) {
#pragma unroll
  for (int c = 0; c < HP / 4; c++) {
    n[c] = ld_stream_i4(reinterpret_cast<const int4*>(nbr + off) + c, pol);
    w[c] = ld_stream_f4(reinterpret_cast<const float4*>(b + off) + c, pol);
  }
}

template <int HP>
__device__ __forceinline__ void scatter_row(float* y, const int4 (&n)[HP / 4],
                                            const float4 (&w)[HP / 4], float a) {
  // padded entries (weight 0, neighbour 0) add nothing and are skipped
#pragma unroll
  for (int c = 0; c < HP / 4; c++) {
    if (w[c].x != 0.0f) atomicAdd(y + n[c].x, w[c].x * a);
    if (w[c].y != 0.0f) atomicAdd(y + n[c].y, w[c].y * a);
    if (w[c].z != 0.0f) atomicAdd(y + n[c].z, w[c].z * a);
    if (w[c].w != 0.0f) atomicAdd(y + n[c].w, w[c].w * a);
  }
}

// whiten VJP, sparse rows at positions [p_begin, p_end): vbar_p += w_p and
// vbar_c -= w_j b_j,c for every row j, w_j = xibar_j / sigma_j (for the whole
// graph vbar's sparse entries start at 0, its dense entries at
// L0^-T xibar_0).  No ordering between rows.
template <int KP>
__global__ void __launch_bounds__(256) whiten_adjoint_scatter_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, const float* __restrict__ sigma,
    const float* __restrict__ xibar, float* vbar, int64_t n0, int64_t p_begin, int64_t p_end) {
  constexpr int LANES = gen_lanes(KP), HP = KP / LANES, GPB = 256 / LANES;
  const int h = threadIdx.x % LANES;
  const uint64_t pol = l2_evict_first();
  const int64_t stride = (int64_t)gridDim.x * GPB;
  for (int64_t p = p_begin + (int64_t)blockIdx.x * GPB + threadIdx.x / LANES; p < p_end;
       p += stride) {
    int4 n[HP / 4];
    float4 w[HP / 4];
    load_row_slice<HP>(n, w, nbr, b, (p - n0) * KP + h * HP, pol);
    const float a = xibar[p] / sigma[p];
    if (h == 0) atomicAdd(vbar + p, a);
    scatter_row<HP>(vbar, n, w, -a);
  }
}

// generate VJP: u = (I - B)^-T vbar.  u starts as vbar; deepest level first,
// every row i of level l -- whose u_i is complete, all its children lying in
// deeper levels -- adds b_ia u_i at each neighbour c_a.  One cooperative
// launch, a grid-wide barrier between levels (the barrier's release orders a
// block's atomics before the next level's reads); the first row of a block's
// slice is loaded before the wait.
template <int KP>
__global__ void __launch_bounds__(256) generate_adjoint_scatter_kernel(
    const int32_t* __restrict__ nbr, const float* __restrict__ b, float* u,
    const int64_t* __restrict__ level_off, int num_levels, int64_t n0, LevelBarrier lb) {
  constexpr int LANES = gen_lanes(KP), HP = KP / LANES, GPB = 256 / LANES;
  __shared__ int s_flag;
  const int h = threadIdx.x % LANES;
  const uint64_t pol = l2_evict_first();
  const uint64_t pol_u = l2_evict_last();
  for (int l = num_levels - 1; l >= 1; l--) {
    const int64_t lo = level_off[l], cnt = level_off[l + 1] - lo;
    const int64_t per = (cnt + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = lo + min((int64_t)blockIdx.x * per, cnt);
    const int64_t hi = lo + min((int64_t)(blockIdx.x + 1) * per, cnt);
    int64_t p = b0 + threadIdx.x / LANES;
    int4 n[HP / 4];
    float4 w[HP / 4];
    if (p < hi) load_row_slice<HP>(n, w, nbr, b, (p - n0) * KP + h * HP, pol);
    if (l < num_levels - 1 && lb.wait(l + 1, gridDim.x, &s_flag)) return;
    while (p < hi) {
      const float a = ld_coherent_f(u + p, pol_u);
      int4 nn[HP / 4];
      float4 ww[HP / 4];
#pragma unroll
      for (int c = 0; c < HP / 4; c++) {
        nn[c] = n[c];
        ww[c] = w[c];
      }
      p += GPB;
      if (p < hi) load_row_slice<HP>(n, w, nbr, b, (p - n0) * KP + h * HP, pol);
      scatter_row<HP>(u, nn, ww, a);
    }
    __syncthreads();
    lb.arrive(l);
  }
}

int whiten_adjoint_scatter(graphgp_graph_t g, graphgp_factor_t f, const float* xibar, float* vbar,
                           int64_t p_begin, int64_t p_end, cudaStream_t s) {
  const int64_t grid = std::min<int64_t>((p_end - p_begin + 63) / 64, (int64_t)num_sms() * 8);
#define GGP_WSC(KP)                                                                              \
  whiten_adjoint_scatter_kernel<KP><<<(unsigned)grid, 256, 0, s>>>(g->nbr, f->b, f->sigma, xibar, \
                                                                   vbar, g->n0, p_begin, p_end)
  GGP_ADJ_KP_DISPATCH(g->kp, GGP_WSC);
#undef GGP_WSC
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

// ---- per-row factor backward ------------------------------------------------------
// Lane a's row of Kbar against dK/dtheta for the G-lane group form, after
// g = K_cc^-1 bbar (lane a holds g_a): Kbar_ac = -g_a b_c + sbar b_a b_c,
// Kbar_ai = g_a - 2 sbar b_a, Kbar_ii = sbar (lane 0); the three partial
// sums come back reduced over the group (every lane holds them).
template <int G, int KT>
__device__ __forceinline__ void group_row_theta(const PointState<G>& st, int a, int k, bool real,
                                                const KernF& kf, float g, float sbar, float& pl,
                                                float& ps, float& pn) {
  const unsigned full = 0xffffffffu;
  const float inv_s2 = 1.0f / kf.s2;
  pl = ps = pn = 0.0f;
  const float ba = st.b_own;
#pragma unroll
  for (int c = 0; c < G; c++) {
    if (c >= k) break;
    const float bc = __shfl_sync(full, st.b_own, c, G);
    const float kb = -g * bc + sbar * ba * bc;
    if (c == a) {
      ps += kb;
      pn += kb;
    } else {
      const KD kd = kappa_dkappa_d2<KT>(kf, st.D2[c]);
      ps += kb * kd.k * inv_s2;
      pl += kb * kd.dl;
    }
  }
  {
    const float kci = g - 2.0f * sbar * ba;
    const KD kd = kappa_dkappa_d2<KT>(kf, st.d2q);
    ps += kci * kd.k * inv_s2;
    pl += kci * kd.dl;
  }
  if (!real) pl = ps = pn = 0.0f;
  if (a == 0) {  // Kbar_ii = sbar
    ps += sbar;
    pn += sbar;
  }
#pragma unroll
  for (int o = G / 2; o; o >>= 1) {
    pl += __shfl_xor_sync(full, pl, o, G);
    ps += __shfl_xor_sync(full, ps, o, G);
    pn += __shfl_xor_sync(full, pn, o, G);
  }
}

// mode 0 (whiten): alpha_i = -xibar_i / sigma_i, beta = 2 logdetbar.
// mode 1 (generate): alpha_i = u_i, beta = 0; also writes xibar_i = sigma_i u_i.
// bbar_i = alpha_i v_c(i), sigbar_i = alpha_i xi_i + beta / sigma_i.
template <int G, int KT>
__global__ void __launch_bounds__(128) factor_backward_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int kp,
    int64_t n0, KernF kf, int mode, const float* __restrict__ coef, float beta,
    const float* __restrict__ v, const float* __restrict__ xi, float* __restrict__ xibar_out,
    double* __restrict__ thetabar, int64_t* __restrict__ rescue_rows,
    unsigned long long* __restrict__ rescue_count) {
  constexpr int PPW = 32 / G;
  constexpr int GS = PFLayout<G>::GS;
  __shared__ __align__(16) float Ls[4 * PPW * GS];
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int a = lane % G;
  const int warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  float* Lg = Ls + (warp * PPW + grp) * GS;
  double tl = 0.0, ts = 0.0, tn = 0.0;
  const int64_t total_groups = (int64_t)gridDim.x * 4 * PPW;
  const int64_t gid = ((int64_t)blockIdx.x * 4 + warp) * PPW + grp;
  const int64_t npts = N - n0;
  const int64_t iters = (npts + total_groups - 1) / total_groups;
  for (int64_t it = 0; it < iters; it++) {
    int64_t t = it * total_groups + gid;
    bool valid = t < npts;
    int64_t i = n0 + (valid ? t : 0);
    bool real = a < k;
    int32_t ca = real ? nbr[(i - n0) * kp + a] : 0;
    PointState<G> st;
    point_factor_group<G, KT>(st, a, k, kf, xs[ca], xs[i], Lg);
    __syncwarp();
    float sigma = st.sigma;
    float ci = coef[i];
    float alpha = mode == 0 ? -ci / sigma : ci;
    float xii = xi[i];
    float sigbar = alpha * xii + beta / sigma;
    float sbar = sigbar / (2.0f * sigma);
    float bbar = real ? alpha * v[ca] : 0.0f;
    float g = group_chol_solve<G>(st, a, k, bbar, Lg);
    __syncwarp();
    // row a of Kbar against dK/dtheta
    float pl, ps, pn;
    group_row_theta<G, KT>(st, a, k, real, kf, g, sbar, pl, ps, pn);
    // rows the forward factor recomputed in FP64 (rescue.cuh): the FP32 sums
    // above are discarded and the row goes to factor_backward_rescue_kernel
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const bool lane_bad = real && !isfinite(st.b_own);
    const bool rescue = st.clamped || row_error_too_large(st.max_ratio, st.varw, st.sigma, kf) ||
                        !isfinite(st.sigma) || (__ballot_sync(full, lane_bad) & gmask);
    if (valid && a == 0) {
      if (rescue) {
        rescue_rows[atomicAdd(rescue_count, 1ull)] = i;
      } else {
        tl += pl;
        ts += ps;
        tn += pn;
        if (mode == 1) xibar_out[i] = sigma * ci;
      }
    }
  }
  block_add3(tl, ts, tn, thetabar);
}

// The same per-row backward for 32 < k <= 64: one warp per point, the factor
// recomputed by point_factor_wide (bit-identical to the forward kernel), then
// g = K_cc^-1 bbar by two triangular solves in shared memory.  Lane a + 32 s
// takes row a + 32 s of Kbar against dK/dtheta (FP32 per row, FP64 across
// rows); rows needing the FP64 rescue go to factor_backward_rescue_kernel.
template <int KT>
__global__ void __launch_bounds__(128) factor_backward_wide_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int kp,
    int64_t n0, KernF kf, int mode, const float* __restrict__ coef, float beta,
    const float* __restrict__ v, const float* __restrict__ xi, float* __restrict__ xibar_out,
    double* __restrict__ thetabar, int64_t* __restrict__ rescue_rows,
    unsigned long long* __restrict__ rescue_count) {
  extern __shared__ __align__(16) unsigned char wide_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WideWarp& W = reinterpret_cast<WideWarp*>(wide_smem)[warp];
  double tl = 0.0, ts = 0.0, tn = 0.0;
  const float inv_s2 = 1.0f / kf.s2;
  const int64_t npts = N - n0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; t < npts; t += nw) {
    const int64_t i = n0 + t;
    const int32_t* row = nbr + t * kp;
    for (int a = lane; a < k; a += 32) W.x[a] = __ldg(xs + row[a]);
    __syncwarp();
    const float4 xq = __ldg(xs + i);
    const WideFactor r = point_factor_wide<KT>(W, k, kf, xq);
    if (wide_needs_rescue(W, r, k, kf)) {
      if (lane == 0) rescue_rows[atomicAdd(rescue_count, 1ull)] = i;
      __syncwarp();
      continue;
    }
    const float sigma = r.sigma;
    const float ci = coef[i];
    const float alpha = mode == 0 ? -ci / sigma : ci;
    const float sigbar = alpha * xi[i] + beta / sigma;
    const float sbar = sigbar / (2.0f * sigma);
    for (int a = lane; a < k; a += 32) W.g[a] = alpha * v[row[a]];
    __syncwarp();
    wide_chol_solve(W, k, r.inc);
    for (int a = lane; a < k; a += 32) {
      const float ga = W.g[a], ba = W.y[a];
      const float4 xa = W.x[a];
      float pl = 0.0f, ps = 0.0f, pn = 0.0f;
      for (int c = 0; c < k; c++) {
        const float bc = W.y[c];
        const float kb = -ga * bc + sbar * ba * bc;
        if (c == a) {
          ps += kb;
          pn += kb;
        } else {
          const KD kd = kappa_dkappa_d2<KT>(kf, sqdist(xa, W.x[c]));
          ps += kb * kd.k * inv_s2;
          pl += kb * kd.dl;
        }
      }
      const float kci = ga - 2.0f * sbar * ba;
      const KD kq = kappa_dkappa_d2<KT>(kf, sqdist(xa, xq));
      ps += kci * kq.k * inv_s2;
      pl += kci * kq.dl;
      tl += pl;
      ts += ps;
      tn += pn;
    }
    if (lane == 0) {  // Kbar_ii = sbar
      ts += sbar;
      tn += sbar;
      if (mode == 1) xibar_out[i] = sigma * ci;
    }
    __syncwarp();
  }
  block_add3(tl, ts, tn, thetabar);
}

// FP64 backward of the rows the per-row kernels handed over (rescue.cuh).
template <int G, int KT>
__global__ void __launch_bounds__(128) factor_backward_rescue_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int kp, int64_t n0,
    KernF kf, int mode, const float* __restrict__ coef, float beta, const float* __restrict__ v,
    const float* __restrict__ xi, float* __restrict__ xibar_out, double* __restrict__ thetabar,
    const int64_t* __restrict__ rows, const unsigned long long* __restrict__ count,
    unsigned long long cap) {
  double tl = 0.0, ts = 0.0, tn = 0.0;
  const int64_t n = (int64_t)(*count < cap ? *count : cap);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rows[r];
    const int32_t* row_ptr = nbr + (i - n0) * kp;
    Row64<G> R;
    row_factor64<G, KT>(R, xs, row_ptr, k, xs[i], kf);
    const float sg = (float)R.sigma;
    const float ci = coef[i];
    const double al = mode == 0 ? -(double)ci / sg : (double)ci;
    const double sb = al * (double)xi[i] + (double)beta / sg;
    row_backward64<G, KT>(R, xs, row_ptr, k, xs[i], kf, v, al, sb, sg, tl, ts, tn);
    if (mode == 1) xibar_out[i] = sg * ci;
  }
  block_add3(tl, ts, tn, thetabar);
}

// The per-row factor backward of one-thread-per-point rows, after
// point_factor_thread left the row's factor in p and its coordinates in the
// stage: g = K_cc^-1 (alpha v_c), then Kbar against dkappa/dtheta over the
// pairs.  Once g is solved, L is dead and the coordinates are reloaded for
// the kernel derivatives; the pair (a, c), c < a, takes Kbar_ac + Kbar_ca
// against the symmetric dkappa_ac.  Each row's sum (FP32, at most k + 1
// terms) goes straight into the thread's FP64 totals.
template <int K, int KT>
__device__ __forceinline__ void thread_row_backward(PointRegs<K>& p, const ThreadStage<K>& st,
                                                    const int32_t* row_ptr, int k,
                                                    const KernF& kf, float4 xq,
                                                    const float* __restrict__ v, float alpha,
                                                    float sbar, double& tl, double& ts,
                                                    double& tn) {
  const float inv_s2 = 1.0f / kf.s2;
  const int4* row = reinterpret_cast<const int4*>(row_ptr);
  float g[K];
  int32_t ca[K];
#pragma unroll
  for (int q = 0; q < K / 4; q++) {
    const int4 c = __ldg(row + q);
    ca[4 * q] = c.x;
    ca[4 * q + 1] = c.y;
    ca[4 * q + 2] = c.z;
    ca[4 * q + 3] = c.w;
  }
#pragma unroll
  for (int a = 0; a < K; a++) g[a] = a < k ? alpha * v[ca[a]] : 0.0f;
  thread_chol_solve<K>(p, k, g);
  // b and g into the stage (the kernel values there are consumed), then a
  // rolled loop over the pairs: row sums in FP32 (at most k + 1 terms),
  // added to the FP64 totals
  float* sb = st.E;
  float* sg = st.E + K * kThreadBlock;
#pragma unroll
  for (int a = 0; a < K; a++) {
    sb[a * kThreadBlock] = p.y[a];
    sg[a * kThreadBlock] = g[a];
  }
  ts += sbar;  // Kbar_ii = sbar
  tn += sbar;
#pragma unroll 1
  for (int a = 0; a < k; a++) {
    const float ga = sg[a * kThreadBlock], ba = sb[a * kThreadBlock];
    const float4 xa = st.X[a * kThreadBlock];
    {
      const float kaa = -ga * ba + sbar * ba * ba;
      float pl = 0.0f, ps = kaa;
      int c = 0;
      // four pairs per iteration, evaluated together and added in order
#pragma unroll 1
      for (; c + 4 <= a; c += 4) {
        float gc[4], bc[4];
        float4 xc[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          gc[u] = sg[(c + u) * kThreadBlock];
          bc[u] = sb[(c + u) * kThreadBlock];
          xc[u] = st.X[(c + u) * kThreadBlock];
        }
        float kb[4];
        KD kd[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          kb[u] = (-ga * bc[u] + sbar * ba * bc[u]) + (-gc[u] * ba + sbar * bc[u] * ba);
          kd[u] = kappa_dkappa_d2<KT>(kf, sqdist(xa, xc[u]));
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          ps += kb[u] * kd[u].k * inv_s2;
          pl += kb[u] * kd[u].dl;
        }
      }
#pragma unroll 1
      for (; c < a; c++) {
        const float gc = sg[c * kThreadBlock], bc = sb[c * kThreadBlock];
        const float kb = (-ga * bc + sbar * ba * bc) + (-gc * ba + sbar * bc * ba);
        const KD kd = kappa_dkappa_d2<KT>(kf, sqdist(xa, st.X[c * kThreadBlock]));
        ps += kb * kd.k * inv_s2;
        pl += kb * kd.dl;
      }
      const float kci = ga - 2.0f * sbar * ba;
      const KD kq = kappa_dkappa_d2<KT>(kf, sqdist(xa, xq));
      ps += kci * kq.k * inv_s2;
      pl += kci * kq.dl;
      tl += pl;
      ts += ps;
      tn += kaa;
    }
  }
}

// The same per-row backward with one thread per point and the factor in
// registers (k <= 16, K = padded row length), recomputed by
// point_factor_thread: bit-identical b and sigma to the forward kernel.
template <int K, int KT>
__global__ void __launch_bounds__(128) factor_backward_thread_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, int mode, const float* __restrict__ coef, float beta, const float* __restrict__ v,
    const float* __restrict__ xi, float* __restrict__ xibar_out, double* __restrict__ thetabar,
    int64_t* __restrict__ rescue_rows, unsigned long long* __restrict__ rescue_count,
    unsigned long long rescue_cap) {
  extern __shared__ __align__(16) unsigned char tstage[];
  const ThreadStage<K> st(tstage);
  double tl = 0.0, ts = 0.0, tn = 0.0;
  const int64_t npts = N - n0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n0 + t;
    const int32_t* row_ptr = nbr + t * K;
    const float4 xq = __ldg(xs + i);
    PointRegs<K> p;
    stage_coords<K>(st, xs, row_ptr, k);
    point_factor_thread<K, KT>(p, k, kf, st, xq);
    if (needs_rescue(p, k, kf)) {
      // listed for factor_backward_rescue_kernel; recomputed here when the list is full
      const unsigned long long slot = atomicAdd(rescue_count, 1ull);
      if (slot < rescue_cap) {
        rescue_rows[slot] = i;
        continue;
      }
      Row64<K> R;
      row_factor64<K, KT>(R, xs, row_ptr, k, xq, kf);
      const float sg = (float)R.sigma;
      const float ci = coef[i];
      const double alpha = mode == 0 ? -(double)ci / sg : (double)ci;
      const double sigbar = alpha * (double)xi[i] + (double)beta / sg;
      row_backward64<K, KT>(R, xs, row_ptr, k, xq, kf, v, alpha, sigbar, sg, tl, ts, tn);
      if (mode == 1) xibar_out[i] = sg * ci;
      continue;
    }
    const float sigma = p.sigma;
    const float ci = coef[i];
    const float alpha = mode == 0 ? -ci / sigma : ci;
    const float sigbar = alpha * xi[i] + beta / sigma;
    thread_row_backward<K, KT>(p, st, row_ptr, k, kf, xq, v, alpha, sigbar / (2.0f * sigma), tl,
                               ts, tn);
    if (mode == 1) xibar_out[i] = sigma * ci;
  }
  block_add3(tl, ts, tn, thetabar);
}

// NLL value and gradient in one pass, the factors recomputed and never stored
// (k <= 16, one thread per point).  Each row's b and sigma come from
// point_factor_thread with the factor kernel's FP64 rescue (warp_rescue), so
// they are bit-identical to a stored factor's; xi_i = (v_i - b . v_c) /
// sigma_i follows the stored sweeps' order.  The row then adds its share of
// what graphgp_nll + graphgp_nll_backward compute: xi_i^2 and log sigma_i
// to the value; w_i = nllbar xi_i / sigma_i at i and -w_i b_ia at each
// neighbour (vbar, atomic adds; vbar's sparse entries start at 0); and the
// row's factor backward with alpha = -w_i and sigbar = alpha xi_i +
// nllbar / sigma_i (the logdet cotangent nllbar / 2, doubled).  Rows sent to
// FP64 leave xi_i and nllbar xi_i in xi_out / xibar_out and are listed for
// factor_backward_rescue_kernel (recomputed here when the list is full).
// Iterations are uniform across the warp (warp_rescue is a collective).
template <int K, int KT>
__global__ void __launch_bounds__(128) nll_grad_fused_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, float nllbar, const float* __restrict__ v, float* vbar, float* __restrict__ xi_out,
    float* __restrict__ xibar_out, double* __restrict__ thetabar, double* __restrict__ acc,
    unsigned long long* __restrict__ not_pd, int64_t* __restrict__ rescue_rows,
    unsigned long long* __restrict__ rescue_count, unsigned long long rescue_cap) {
  extern __shared__ __align__(16) unsigned char tstage[];
  const ThreadStage<K> st(tstage);
  double* W = fused_rescue_ws<K>(tstage);
  const uint64_t pol_v = l2_evict_last();
  LogAcc lacc;
  double sq = 0.0, tl = 0.0, ts = 0.0, tn = 0.0;
  unsigned long long clamped = 0;
  const int64_t npts = N - n0;
  const int64_t total = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (npts + total - 1) / total;  // the same on every lane
  for (int64_t it = 0; it < iters; it++) {
    const int64_t t = it * total + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = t < npts;
    const int64_t i = n0 + (valid ? t : 0);
    const int32_t* row_ptr = nbr + (valid ? t : 0) * K;
    const float4 xq = __ldg(xs + i);
    PointRegs<K> p;
    if (valid) {
      stage_coords<K>(st, xs, row_ptr, k);
      point_factor_thread<K, KT>(p, k, kf, st, xq);
    }
    const bool rescue = valid && needs_rescue(p, k, kf);
    warp_rescue<K, KT>(p, rescue, xs, row_ptr, k, xq, kf, W);
    if (!valid) continue;
    const float sigma = p.sigma;
    const float xv = (ld_keep_f(v + i, pol_v) - dot_stored_order<K, false>(p.y, row_ptr, v, pol_v)) / sigma;
    sq += (double)xv * (double)xv;
    lacc.mul(sigma);
    clamped += p.clamped ? 1 : 0;
    const float xb = nllbar * xv;
    const float w = xb / sigma;
    atomicAdd(vbar + i, w);
#pragma unroll
    for (int q = 0; q < K / 4; q++) {
      const int4 c = __ldg(reinterpret_cast<const int4*>(row_ptr) + q);
      if (p.y[4 * q] != 0.0f) atomicAdd(vbar + c.x, p.y[4 * q] * -w);
      if (p.y[4 * q + 1] != 0.0f) atomicAdd(vbar + c.y, p.y[4 * q + 1] * -w);
      if (p.y[4 * q + 2] != 0.0f) atomicAdd(vbar + c.z, p.y[4 * q + 2] * -w);
      if (p.y[4 * q + 3] != 0.0f) atomicAdd(vbar + c.w, p.y[4 * q + 3] * -w);
    }
    if (rescue) {
      xi_out[i] = xv;
      xibar_out[i] = xb;
      const unsigned long long slot = atomicAdd(rescue_count, 1ull);
      if (slot < rescue_cap) {
        rescue_rows[slot] = i;
        continue;
      }
      Row64<K> R;
      row_factor64<K, KT>(R, xs, row_ptr, k, xq, kf);
      const float sg = (float)R.sigma;
      const double alpha = -(double)xb / sg;
      const double sigbar = alpha * (double)xv + (double)nllbar / sg;
      row_backward64<K, KT>(R, xs, row_ptr, k, xq, kf, v, alpha, sigbar, sg, tl, ts, tn);
      continue;
    }
    const float alpha = -xb / sigma;
    const float sigbar = alpha * xv + nllbar / sigma;
    thread_row_backward<K, KT>(p, st, row_ptr, k, kf, xq, v, alpha, sigbar / (2.0f * sigma), tl,
                               ts, tn);
  }
  block_add3(tl, ts, tn, thetabar);
  block_add_double(sq, acc);
  block_add_double(lacc.log_value(), acc + 1);
  unsigned long long c = clamped;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(not_pd, c);
}

// The FP64 conditional of a warp's row out of line: the rescue is rare, and
// inlined its state would raise the register count of the whole kernel.
template <int KT>
__device__ __noinline__ WarpRow64 warp_row_factor64_outlined(const float4* __restrict__ xs,
                                                            const int32_t* row, int k,
                                                            float4 xq, KernF kf, double* W) {
  return warp_row_factor64<32, KT>(xs, row, k, xq, kf, W);
}

// The one-pass NLL value and gradient for 16 < k <= 32: one warp per point,
// the 32-lane group factor (point_factor_group with the factor kernel's
// rescue decision), so b and sigma are the stored factor's; a row that needs
// FP64 takes its b and sigma from warp_row_factor64 for the value and the
// scatter and is listed for factor_backward_rescue_kernel (the list holds
// every row); the other rows run the group backward (group_chol_solve,
// group_row_theta) on the factor still in the warp's shared memory.
template <int KP, int KT>
__global__ void __launch_bounds__(128, 3) nll_grad_fused_group_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, float nllbar, const float* __restrict__ v, float* vbar, float* __restrict__ xi_out,
    float* __restrict__ xibar_out, double* __restrict__ thetabar, double* __restrict__ acc,
    unsigned long long* __restrict__ not_pd, int64_t* __restrict__ rescue_rows,
    unsigned long long* __restrict__ rescue_count) {
  constexpr int GS = PFLayout<32>::GS;
  __shared__ __align__(16) float Ls[4 * GS];
  extern __shared__ __align__(16) double gws[];  // 4 x 32 x 33 doubles (FP64 rescue)
  const int a = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  float* Lg = Ls + warp * GS;
  double* W = gws + warp * (32 * 33);
  const uint64_t pol_v = l2_evict_last();
  LogAcc lacc;
  double sq = 0.0, tl = 0.0, ts = 0.0, tn = 0.0;
  unsigned long long clamped = 0;
  const int64_t npts = N - n0;
  const int64_t nw = (int64_t)gridDim.x * 4;
  for (int64_t t = (int64_t)blockIdx.x * 4 + warp; t < npts; t += nw) {  // warp-uniform
    const int64_t i = n0 + t;
    const int32_t* row = nbr + t * KP;
    const bool real = a < k;
    const int32_t ca = real ? __ldg(row + a) : 0;
    const float4 xq = __ldg(xs + i);
    PointState<32> st;
    point_factor_group<32, KT>(st, a, k, kf, __ldg(xs + ca), xq, Lg);
    __syncwarp();
    const bool lane_bad = real && !isfinite(st.b_own);
    const bool rescue = st.clamped || row_error_too_large(st.max_ratio, st.varw, st.sigma, kf) ||
                        !isfinite(st.sigma) || __ballot_sync(full, lane_bad);
    float b = real ? st.b_own : 0.0f, sigma = st.sigma;
    bool clamp = st.clamped;
    if (rescue) {
      const WarpRow64 w = warp_row_factor64_outlined<KT>(xs, row, k, xq, kf, W);
      b = real ? (float)w.b : 0.0f;
      sigma = (float)w.sigma;
      clamp = w.clamped;
    }
    const float dot = warp_dot_stored_order<KP, false>(b, row, v, pol_v);
    float xv = 0.0f;
    if (a == 0) xv = (ld_keep_f(v + i, pol_v) - dot) / sigma;
    xv = __shfl_sync(full, xv, 0);
    const float xb = nllbar * xv;
    const float w = xb / sigma;
    if (a == 0) {
      sq += (double)xv * (double)xv;
      lacc.mul(sigma);
      clamped += clamp ? 1 : 0;
      atomicAdd(vbar + i, w);
    }
    if (real && b != 0.0f) atomicAdd(vbar + ca, b * -w);
    if (rescue) {
      if (a == 0) {
        xi_out[i] = xv;
        xibar_out[i] = xb;
        rescue_rows[atomicAdd(rescue_count, 1ull)] = i;
      }
      __syncwarp();
      continue;
    }
    const float alpha = -xb / sigma;
    const float sigbar = alpha * xv + nllbar / sigma;
    const float sbar = sigbar / (2.0f * sigma);
    const float bbar = real ? alpha * v[ca] : 0.0f;
    const float g = group_chol_solve<32>(st, a, k, bbar, Lg);
    __syncwarp();
    float pl, ps, pn;
    group_row_theta<32, KT>(st, a, k, real, kf, g, sbar, pl, ps, pn);
    if (a == 0) {
      tl += pl;
      ts += ps;
      tn += pn;
    }
    __syncwarp();
  }
  block_add3(tl, ts, tn, thetabar);
  block_add_double(sq, acc);
  block_add_double(a == 0 ? lacc.log_value() : 0.0, acc + 1);
  unsigned long long c = clamped;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(full, c, o);
  if (a == 0 && c) atomicAdd(not_pd, c);
}

__global__ void scale_kernel(const float* __restrict__ x, float s, float* __restrict__ y,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

__global__ void mul_kernel(const float* __restrict__ a, const float* __restrict__ x,
                           float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] * x[i];
}

template <int G>
int launch_factor_backward(graphgp_graph_t g, graphgp_factor_t f, int mode, const float* coef,
                           float beta, const float* v, const float* xi, float* xibar,
                           double* thetabar, const int32_t* nbr, int64_t N, int64_t n0v,
                           cudaStream_t s) {
  int64_t npts = N - n0v;
  if (npts <= 0) return GRAPHGP_OK;
  constexpr int PPW = 32 / G;
  unsigned grid = grid_for((npts + 4 * PPW - 1) / (4 * PPW) * 128, 128, 16);
  KernF kf = make_kernf(f->kern);
  Scratch sc(s);
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, npts));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  const unsigned rgrid = (unsigned)num_sms() * 2;
#define GGP_FB(KT)                                                                          \
  factor_backward_kernel<G, KT><<<grid, 128, 0, s>>>(g->xs, nbr, N, g->k, g->kp, n0v, \
                                                     kf, mode, coef, beta, v, xi, xibar,     \
                                                     thetabar, rows, cnt);                   \
  factor_backward_rescue_kernel<G, KT><<<rgrid, 128, 0, s>>>(                               \
      g->xs, nbr, g->k, g->kp, n0v, kf, mode, coef, beta, v, xi, xibar, thetabar, rows, cnt, \
      (unsigned long long)npts)
  switch (f->kern.type) {
    case GRAPHGP_MATERN12: GGP_FB(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_FB(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_FB(GRAPHGP_MATERN52); break;
    default: GGP_FB(GRAPHGP_SQEXP); break;
  }
#undef GGP_FB
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

constexpr int64_t kBackwardRescueMax = 1 << 20;  // rows listed for the FP64 backward

template <int K>
int launch_factor_backward_thread(graphgp_graph_t g, graphgp_factor_t f, int mode,
                                  const float* coef, float beta, const float* v, const float* xi,
                                  float* xibar, double* thetabar, const int32_t* nbr,
                                  int64_t N, int64_t n0v, cudaStream_t s) {
  const int64_t npts = N - n0v;
  if (npts <= 0) return GRAPHGP_OK;
  const unsigned grid = grid_for(npts, 128, 8);
  KernF kf = make_kernf(f->kern);
  Scratch sc(s);
  const unsigned long long cap = (unsigned long long)std::min<int64_t>(npts, kBackwardRescueMax);
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, cap));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  const unsigned rgrid = (unsigned)num_sms() * 2;
  constexpr size_t smem = ThreadStage<K>::kBytes;
#define GGP_FBT(KT)                                                                             \
  GGP_CUDA(allow_dyn_smem(factor_backward_thread_kernel<K, KT>, smem));                         \
  factor_backward_thread_kernel<K, KT><<<grid, kThreadBlock, smem, s>>>(                        \
      g->xs, nbr, N, g->k, n0v, kf, mode, coef, beta, v, xi, xibar, thetabar, rows, cnt, \
      cap);                                                                                     \
  factor_backward_rescue_kernel<K, KT><<<rgrid, 128, 0, s>>>(                                   \
      g->xs, nbr, g->k, g->kp, n0v, kf, mode, coef, beta, v, xi, xibar, thetabar, rows, cnt, cap)
  switch (f->kern.type) {
    case GRAPHGP_MATERN12: GGP_FBT(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_FBT(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_FBT(GRAPHGP_MATERN52); break;
    default: GGP_FBT(GRAPHGP_SQEXP); break;
  }
#undef GGP_FBT
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int K>
int launch_nll_grad_fused(graphgp_graph_t g, const graphgp_kernel* kern, float nllbar,
                          const float* v, float* vbar, float* xi_tmp, float* xibar_tmp,
                          double* thetabar, double* acc, unsigned long long* not_pd,
                          cudaStream_t s) {
  const int64_t npts = g->N - g->n0;
  if (npts <= 0) return GRAPHGP_OK;
  const unsigned grid = grid_for(npts, kThreadBlock, 8);
  const KernF kf = make_kernf(*kern);
  Scratch sc(s);
  const unsigned long long cap = (unsigned long long)std::min<int64_t>(npts, kBackwardRescueMax);
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, cap));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  const unsigned rgrid = (unsigned)num_sms() * 2;
  constexpr size_t smem = fused_smem<K>();
#define GGP_NGF(KT)                                                                              \
  GGP_CUDA(allow_dyn_smem(nll_grad_fused_kernel<K, KT>, smem));                                  \
  nll_grad_fused_kernel<K, KT><<<grid, kThreadBlock, smem, s>>>(                                 \
      g->xs, g->nbr, g->N, g->k, g->n0, kf, nllbar, v, vbar, xi_tmp, xibar_tmp, thetabar, acc,  \
      not_pd, rows, cnt, cap);                                                                   \
  factor_backward_rescue_kernel<K, KT><<<rgrid, 128, 0, s>>>(                                    \
      g->xs, g->nbr, g->k, g->kp, g->n0, kf, 0, xibar_tmp, nllbar, v, xi_tmp, nullptr, thetabar, \
      rows, cnt, cap)
  switch (kern->type) {
    case GRAPHGP_MATERN12: GGP_NGF(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_NGF(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_NGF(GRAPHGP_MATERN52); break;
    default: GGP_NGF(GRAPHGP_SQEXP); break;
  }
#undef GGP_NGF
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int KP>
int launch_nll_grad_fused_group(graphgp_graph_t g, const graphgp_kernel* kern, float nllbar,
                                const float* v, float* vbar, float* xi_tmp, float* xibar_tmp,
                                double* thetabar, double* acc, unsigned long long* not_pd,
                                cudaStream_t s) {
  const int64_t npts = g->N - g->n0;
  if (npts <= 0) return GRAPHGP_OK;
  const unsigned grid = grid_for((npts + 3) / 4 * 128, 128, 16);
  const KernF kf = make_kernf(*kern);
  Scratch sc(s);
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, npts));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  const unsigned rgrid = (unsigned)num_sms() * 2;
  constexpr size_t smem = (size_t)4 * 32 * 33 * sizeof(double);
#define GGP_NGG(KT)                                                                              \
  GGP_CUDA(cudaFuncSetAttribute(nll_grad_fused_group_kernel<KP, KT>,                            \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));        \
  nll_grad_fused_group_kernel<KP, KT><<<grid, 128, smem, s>>>(                                   \
      g->xs, g->nbr, g->N, g->k, g->n0, kf, nllbar, v, vbar, xi_tmp, xibar_tmp, thetabar, acc,  \
      not_pd, rows, cnt);                                                                        \
  factor_backward_rescue_kernel<32, KT><<<rgrid, 128, 0, s>>>(                                   \
      g->xs, g->nbr, g->k, g->kp, g->n0, kf, 0, xibar_tmp, nllbar, v, xi_tmp, nullptr, thetabar, \
      rows, cnt, (unsigned long long)npts)
  switch (kern->type) {
    case GRAPHGP_MATERN12: GGP_NGG(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_NGG(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_NGG(GRAPHGP_MATERN52); break;
    default: GGP_NGG(GRAPHGP_SQEXP); break;
  }
#undef GGP_NGG
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

__global__ void nll_value_kernel(const double* __restrict__ acc, double* __restrict__ out) {
  out[0] = 0.5 * acc[0] + 0.5 * acc[1];
}

int launch_factor_backward_wide(graphgp_graph_t g, graphgp_factor_t f, int mode,
                                const float* coef, float beta, const float* v, const float* xi,
                                float* xibar, double* thetabar, const int32_t* nbr,
                                  int64_t N, int64_t n0v, cudaStream_t s) {
  const int64_t npts = N - n0v;
  if (npts <= 0) return GRAPHGP_OK;
  constexpr int kWarps = 4;
  const size_t smem = kWarps * sizeof(WideWarp);
  const unsigned grid = grid_for((npts + kWarps - 1) / kWarps * 128, 128, 4);
  KernF kf = make_kernf(f->kern);
  Scratch sc(s);
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, npts));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  const unsigned rgrid = (unsigned)num_sms() * 2;
#define GGP_FBW(KT)                                                                            \
  GGP_CUDA(cudaFuncSetAttribute(factor_backward_wide_kernel<KT>,                               \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));      \
  factor_backward_wide_kernel<KT><<<grid, 32 * kWarps, smem, s>>>(                             \
      g->xs, nbr, N, g->k, g->kp, n0v, kf, mode, coef, beta, v, xi, xibar, thetabar,   \
      rows, cnt);                                                                              \
  factor_backward_rescue_kernel<kWideK, KT><<<rgrid, 128, 0, s>>>(                             \
      g->xs, nbr, g->k, g->kp, n0v, kf, mode, coef, beta, v, xi, xibar, thetabar, rows, cnt,  \
      (unsigned long long)npts)
  switch (f->kern.type) {
    case GRAPHGP_MATERN12: GGP_FBW(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_FBW(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_FBW(GRAPHGP_MATERN52); break;
    default: GGP_FBW(GRAPHGP_SQEXP); break;
  }
#undef GGP_FBW
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

int factor_backward_rows(graphgp_graph_t g, graphgp_factor_t f, int mode, const float* coef,
                         float beta, const float* v, const float* xi, float* xibar,
                         double* thetabar, int64_t t0, int64_t t1, cudaStream_t s) {
  if (t1 <= t0) return GRAPHGP_OK;
  const int32_t* nb = g->nbr + t0 * g->kp;
  const int64_t N = g->n0 + t1, n0v = g->n0 + t0;
  switch (g->kp) {
    case 4: return launch_factor_backward_thread<4>(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
    case 8: return launch_factor_backward_thread<8>(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
    case 12: return launch_factor_backward_thread<12>(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
    case 16: return launch_factor_backward_thread<16>(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
    case 20:
    case 24:
    case 28:
    case 32: return launch_factor_backward<32>(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
    default: return launch_factor_backward_wide(g, f, mode, coef, beta, v, xi, xibar, thetabar, nb, N, n0v, s);
  }
}

int factor_backward(graphgp_graph_t g, graphgp_factor_t f, int mode, const float* coef,
                    float beta, const float* v, const float* xi, float* xibar, double* thetabar,
                    cudaStream_t s) {
  return factor_backward_rows(g, f, mode, coef, beta, v, xi, xibar, thetabar, 0, g->N - g->n0, s);
}

}  // namespace

// Kbar_00 (n0 x n0, row-major, every entry a cotangent) of the dense block
// from u_0 and xi_0: Kbar = L0^-T Phi(L0^T Lbar0) L0^-1.
int dense_kbar(graphgp_graph_t g, graphgp_factor_t f, const float* u0, const float* xi0,
               float sgn, float ldbar, float* Kbar, cudaStream_t s) {
  int n0 = g->n0;
  int64_t nn = (int64_t)n0 * n0;
  Scratch sc(s);
  float *P = nullptr, *T = nullptr;
  GGP_TRY(sc.alloc(&P, nn));
  GGP_TRY(sc.alloc(&T, nn));
  unsigned grid = grid_for(nn, 256);
  dense_lbar_kernel<<<grid, 256, 0, s>>>(u0, xi0, f->L0, n0, sgn, ldbar, Kbar);
  dense_gemm_kernel<<<grid, 256, 0, s>>>(f->L0, Kbar, P, n0, 1, 1);     // Phi(L0^T Lbar0)
  dense_gemm_kernel<<<grid, 256, 0, s>>>(f->L0inv, P, T, n0, 1, 0);     // L0^-T P
  dense_gemm_kernel<<<grid, 256, 0, s>>>(T, f->L0inv, Kbar, n0, 0, 0);  // (L0^-T P) L0^-1
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

namespace {

int dense_backward(graphgp_graph_t g, graphgp_factor_t f, const float* u0, const float* xi0,
                   float sgn, float ldbar, double* thetabar, cudaStream_t s) {
  int n0 = g->n0;
  int64_t nn = (int64_t)n0 * n0;
  Scratch sc(s);
  float* Lb = nullptr;
  GGP_TRY(sc.alloc(&Lb, nn));
  GGP_TRY(dense_kbar(g, f, u0, xi0, sgn, ldbar, Lb, s));
  unsigned grid = grid_for(nn, 256);
  KernF kf = make_kernf(f->kern);
  switch (f->kern.type) {
    case GRAPHGP_MATERN12: dense_theta_kernel<GRAPHGP_MATERN12><<<grid, 256, 0, s>>>(Lb, g->xs, n0, kf, thetabar); break;
    case GRAPHGP_MATERN32: dense_theta_kernel<GRAPHGP_MATERN32><<<grid, 256, 0, s>>>(Lb, g->xs, n0, kf, thetabar); break;
    case GRAPHGP_MATERN52: dense_theta_kernel<GRAPHGP_MATERN52><<<grid, 256, 0, s>>>(Lb, g->xs, n0, kf, thetabar); break;
    default: dense_theta_kernel<GRAPHGP_SQEXP><<<grid, 256, 0, s>>>(Lb, g->xs, n0, kf, thetabar); break;
  }
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace

int run_whiten_backward(graphgp_graph_t g, graphgp_factor_t f, const float* v, const float* xi,
                        const float* xibar, double logdetbar, float* vbar, double* thetabar,
                        cudaStream_t s) {
  int n0 = g->n0;
  // dense: vbar_0 = L0^-T xibar_0 (then children are subtracted below)
  dense_lower_tmatvec_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f->L0inv, xibar, vbar, n0);
  GGP_CUDA(cudaGetLastError());
  if (thetabar) GGP_TRY(dense_backward(g, f, vbar, xi, -1.0f, (float)logdetbar, thetabar, s));
  if (g->N > n0) {
    GGP_CUDA(cudaMemsetAsync(vbar + n0, 0, (g->N - n0) * sizeof(float), s));
    GGP_TRY(whiten_adjoint_scatter(g, f, xibar, vbar, n0, g->N, s));
  }
  if (thetabar)
    GGP_TRY(factor_backward(g, f, 0, xibar, (float)(2.0 * logdetbar), v, xi, nullptr, thetabar, s));
  return GRAPHGP_OK;
}

int run_generate_backward(graphgp_graph_t g, graphgp_factor_t f, const float* xi, const float* v,
                          const float* vbar, float* xibar, double* thetabar, cudaStream_t s) {
  float* u = g->tmp_vec;
  int n0 = g->n0;
  GGP_CUDA(cudaMemcpyAsync(u, vbar, g->N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (g->num_levels > 1) {
    GGP_CUDA(cudaMemsetAsync(g->level_bar, 0, g->num_levels * sizeof(uint32_t), s));
    LevelBarrier lb{g->level_bar, g->err, g->max_spin};
    const int32_t* nb = g->nbr;
    const float* bw = f->b;
    const int64_t* lo = g->level_off_d;
    int nl = g->num_levels;
    int64_t n0l = n0;
    void* args[] = {(void*)&nb, (void*)&bw, (void*)&u, (void*)&lo, (void*)&nl, (void*)&n0l,
                    (void*)&lb};
#define GGP_GSC(KP)                                                                              \
  {                                                                                              \
    static int max_grid_dev[kMaxDevices] = {};                                                   \
    const int max_grid = coop_grid_cached(max_grid_dev, generate_adjoint_scatter_kernel<KP>, 256); \
    const int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>((g->max_level_size + 63) / 64, 1)); \
    GGP_CUDA(cudaLaunchCooperativeKernel((const void*)generate_adjoint_scatter_kernel<KP>,       \
                                         dim3(grid), dim3(256), args, 0, s));                    \
  }
    GGP_ADJ_KP_DISPATCH(g->kp, GGP_GSC);
#undef GGP_GSC
  }
  // dense: xibar_0 = L0^T u_0, Lbar0 = tril(u_0 xi_0^T)
  dense_lower_tmatvec_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f->L0, u, xibar, n0);
  GGP_CUDA(cudaGetLastError());
  if (!thetabar) {  // vector cotangent only: xibar_i = sigma_i u_i
    if (g->N > n0)
      mul_kernel<<<grid_for(g->N - n0, 256), 256, 0, s>>>(f->sigma + n0, u + n0, xibar + n0,
                                                           g->N - n0);
    GGP_CUDA(cudaGetLastError());
    return GRAPHGP_OK;
  }
  GGP_TRY(dense_backward(g, f, u, xi, 1.0f, 0.0f, thetabar, s));
  GGP_TRY(factor_backward(g, f, 1, u, 0.0f, v, xi, xibar, thetabar, s));
  return GRAPHGP_OK;
}

int run_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
               cudaStream_t s);

// ---- row ranges (sharding by position range) ---------------------------------
// The NLL and its gradient restricted to the positions [p0, p1) whose factor a
// row-range handle holds: the sums over disjoint ranges add up to the whole.

// sum_e b_e v[c_e] of one row in the stored sweeps' order (gen_lanes slices,
// two alternating accumulators per slice, slices combined as their xor
// shuffles do), so xi is bit-identical to the whiten sweep's.
__device__ __forceinline__ float row_dot_stored_order(const float* __restrict__ b,
                                                      const int32_t* __restrict__ c, int kp,
                                                      const float* __restrict__ v) {
  const int lanes = gen_lanes(kp), hp = kp / lanes;
  float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int h = 0; h < lanes; h++) {
    float acc0 = 0.0f, acc1 = 0.0f;
    for (int e = h * hp; e < (h + 1) * hp; e += 4) {
      acc0 = fmaf(b[e], v[c[e]], acc0);
      acc1 = fmaf(b[e + 1], v[c[e + 1]], acc1);
      acc0 = fmaf(b[e + 2], v[c[e + 2]], acc0);
      acc1 = fmaf(b[e + 3], v[c[e + 3]], acc1);
    }
    part[h] = acc0 + acc1;
  }
  if (lanes == 4) return (part[0] + part[2]) + (part[1] + part[3]);
  if (lanes == 2) return part[0] + part[1];
  return part[0];
}

// xi_i = (v_i - b_i . v_c(i)) / sigma_i for rows t in [t0, t1); optional FP64
// sum of xi_i^2 (added to *sq).
__global__ void whiten_rows_kernel(const int32_t* __restrict__ nbr, const float* __restrict__ b,
                                   const float* __restrict__ sigma, const float* __restrict__ v,
                                   float* __restrict__ xi, int kp, int64_t n0, int64_t t0,
                                   int64_t t1, double* __restrict__ sq) {
  double local = 0.0;
  for (int64_t t = t0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < t1;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n0 + t;
    const float acc = row_dot_stored_order(b + t * kp, nbr + t * kp, kp, v);
    const float out = (v[i] - acc) / sigma[i];
    xi[i] = out;
    local += (double)out * (double)out;
  }
  if (sq) block_add_double(local, sq);
}

// y[m] += sum_{i >= m} M[i][m] x[i] for the n0 x n0 lower-triangular M.
__global__ void dense_tmatvec_acc_kernel(const float* __restrict__ M, const float* __restrict__ x,
                                         float* __restrict__ y, int n0) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n0; m += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = m; i < n0; i++) s = fmaf(M[(int64_t)i * n0 + m], x[i], s);
    y[m] += s;
  }
}

__global__ void nll_rows_finish_kernel(const double* __restrict__ sq,
                                       const double* __restrict__ logdet,
                                       double* __restrict__ out) {
  out[0] = 0.5 * sq[0] + 0.5 * logdet[0];
}

// xi over the factor's positions into xi (full length; other entries untouched).
int whiten_rows(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
                cudaStream_t s) {
  const int64_t p0 = f->row_begin, p1 = f->row_end;
  if (p0 == 0) GGP_TRY(dense_matvec(f->L0inv, v, xi, g->n0, sq, s));
  const int64_t t0 = std::max<int64_t>(p0, g->n0) - g->n0, t1 = p1 - g->n0;
  if (t1 > t0) {
    whiten_rows_kernel<<<grid_for(t1 - t0, 256), 256, 0, s>>>(g->nbr, f->b, f->sigma, v, xi, g->kp,
                                                              g->n0, t0, t1, sq);
    GGP_CUDA(cudaGetLastError());
  }
  return GRAPHGP_OK;
}

}  // namespace ggp

using namespace ggp;

static bool rows_ok(graphgp_graph_t g, graphgp_factor_t f) {
  return g && f && f->g == g && f->row_end >= 0;
}

extern "C" int graphgp_nll_rows(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                                double* out_d, void* stream) {
  if (!rows_ok(g, f) || !v_d || !out_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* sq = nullptr;
  GGP_TRY(sc.alloc(&sq, 1));
  GGP_CUDA(cudaMemsetAsync(sq, 0, sizeof(double), s));
  GGP_TRY(whiten_rows(g, f, v_d, g->tmp_vec2, sq, s));
  nll_rows_finish_kernel<<<1, 1, 0, s>>>(sq, f->logdet, out_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

extern "C" int graphgp_nll_backward_rows(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                                         double nllbar, float* vbar_d, double* thetabar_d,
                                         void* stream) {
  if (!rows_ok(g, f) || !v_d || !vbar_d || !thetabar_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  float* xi = g->tmp_vec2;
  float* xibar = g->tmp_vec;
  GGP_TRY(whiten_rows(g, f, v_d, xi, nullptr, s));
  scale_kernel<<<grid_for(g->N, 256), 256, 0, s>>>(xi, (float)nllbar, xibar, g->N);
  GGP_CUDA(cudaGetLastError());
  const int n0 = g->n0;
  const int64_t p0 = f->row_begin, p1 = f->row_end;
  if (p0 == 0) {
    // dense rows: u_0 = L0^-T xibar_0 into vbar_0, and the dense block's theta part
    Scratch sc(s);
    float* u0 = nullptr;
    GGP_TRY(sc.alloc(&u0, n0));
    dense_lower_tmatvec_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f->L0inv, xibar, u0, n0);
    dense_tmatvec_acc_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f->L0inv, xibar, vbar_d, n0);
    GGP_CUDA(cudaGetLastError());
    GGP_TRY(dense_backward(g, f, u0, xi, -1.0f, (float)(0.5 * nllbar), thetabar_d, s));
  }
  const int64_t t0 = std::max<int64_t>(p0, n0) - n0, t1 = p1 - n0;
  if (t1 > t0) {
    // the neighbours of a range belong to other rows and ranges: atomic adds
    GGP_TRY(whiten_adjoint_scatter(g, f, xibar, vbar_d, n0 + t0, n0 + t1, s));
    GGP_TRY(factor_backward_rows(g, f, 0, xibar, (float)nllbar, v_d, xi, nullptr, thetabar_d, t0,
                                 t1, s));
  }
  return GRAPHGP_OK;
}


static bool pair_ok(graphgp_graph_t g, graphgp_factor_t f) {
  return g && f && f->g == g && f->row_end < 0;
}

extern "C" int graphgp_generate_backward(graphgp_graph_t g, graphgp_factor_t f, const float* xi_d,
                                         const float* v_d, const float* vbar_d, float* xibar_d,
                                         double* thetabar_d, void* stream) {
  if (!pair_ok(g, f) || !xi_d || !v_d || !vbar_d || !xibar_d) return GRAPHGP_ERR_INVALID;
  return run_generate_backward(g, f, xi_d, v_d, vbar_d, xibar_d, thetabar_d, (cudaStream_t)stream);
}

extern "C" int graphgp_whiten_backward(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                                       const float* xi_d, const float* xibar_d, double logdetbar,
                                       float* vbar_d, double* thetabar_d, void* stream) {
  if (!pair_ok(g, f) || !xi_d || !v_d || !xibar_d || !vbar_d) return GRAPHGP_ERR_INVALID;
  return run_whiten_backward(g, f, v_d, xi_d, xibar_d, logdetbar, vbar_d, thetabar_d,
                             (cudaStream_t)stream);
}

extern "C" int graphgp_nll_backward(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                                    double nllbar, float* vbar_d, double* thetabar_d,
                                    void* stream) {
  if (!pair_ok(g, f) || !v_d || !vbar_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  float* xi = g->tmp_vec2;
  float* xibar = g->tmp_vec;
  GGP_TRY(run_whiten(g, f, v_d, xi, nullptr, s));
  scale_kernel<<<grid_for(g->N, 256), 256, 0, s>>>(xi, (float)nllbar, xibar, g->N);
  GGP_CUDA(cudaGetLastError());
  return run_whiten_backward(g, f, v_d, xi, xibar, 0.5 * nllbar, vbar_d, thetabar_d, s);
}

// NLL value and gradient with the factors recomputed in the pass (the
// on-the-fly form of graphgp_nll + graphgp_nll_backward).
extern "C" int graphgp_nll_grad_fused(graphgp_graph_t g, const graphgp_kernel* kern,
                                      const float* v_d, double nllbar, double* nll_d,
                                      float* vbar_d, double* thetabar_d, uint64_t* not_pd_d,
                                      void* stream) {
  if (!g || !valid_kernel(kern) || g->k > 32 || !v_d || !nll_d || !vbar_d || !thetabar_d)
    return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* bad = (unsigned long long*)not_pd_d;
  Scratch sc(s);
  double* acc = nullptr;  // [0] xi.xi, [1] logdet
  GGP_TRY(sc.alloc(&acc, 2));
  GGP_CUDA(cudaMemsetAsync(acc, 0, 16, s));
  if (!bad) {
    GGP_TRY(sc.alloc(&bad, 1));
    GGP_CUDA(cudaMemsetAsync(bad, 0, 8, s));
  }
  const int n0 = g->n0;
  float* xi = g->tmp_vec2;  // xi_0 and the FP64 rows' xi
  float* xb = g->tmp_vec;   // nllbar xi for the same positions
  graphgp_factor_s f;
  GGP_TRY(dense_into(g, kern, sc, acc + 1, bad, f, s));
  GGP_TRY(dense_matvec(f.L0inv, v_d, xi, n0, acc, s));
  scale_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(xi, (float)nllbar, xb, n0);
  dense_lower_tmatvec_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f.L0inv, xb, vbar_d, n0);
  GGP_CUDA(cudaGetLastError());
  GGP_TRY(dense_backward(g, &f, vbar_d, xi, -1.0f, (float)(0.5 * nllbar), thetabar_d, s));
  if (g->N > n0) {
    GGP_CUDA(cudaMemsetAsync(vbar_d + n0, 0, (g->N - n0) * sizeof(float), s));
    int rc = GRAPHGP_OK;
    switch (g->kp) {
      case 4: rc = launch_nll_grad_fused<4>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 8: rc = launch_nll_grad_fused<8>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 12: rc = launch_nll_grad_fused<12>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 16: rc = launch_nll_grad_fused<16>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 20: rc = launch_nll_grad_fused_group<20>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 24: rc = launch_nll_grad_fused_group<24>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      case 28: rc = launch_nll_grad_fused_group<28>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
      default: rc = launch_nll_grad_fused_group<32>(g, kern, (float)nllbar, v_d, vbar_d, xi, xb, thetabar_d, acc, bad, s); break;
    }
    GGP_TRY(rc);
  }
  nll_value_kernel<<<1, 1, 0, s>>>(acc, nll_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}
