// Per-point conditional factor of Sec. 2.1 Eq. 2 for 32 < k <= 64 (the
// paper's stated range of the on-GPU method reaches k of about 64): one warp
// per point, the k x k matrix in shared memory.  Shared by the factor kernel
// and the factor-backward kernel, which recomputes the factor, so both see
// bit-identical b and sigma.
//
// The same increment or covariance form as pointfactor.cuh (chosen per row
// from the nearest neighbour's variogram value): M and m are built from
// variogram or kernel values, and b is recovered from beta = M^-1 m.  Right-looking
// Cholesky of M by columns: at step j the pivot L_jj is the updated diagonal
// entry (floored at 1e-7 of kappa(0) + nugget as in the other paths), column
// j is scaled by 1 / L_jj, and the trailing rows are updated, lane a + 32 s
// owning row a + j + 1 + 32 s.  The forward solve y = L^-1 m rides along,
// sigma^2 = Var(w) - y.y accumulates in compensated FP32, and beta = L^-T y
// is a backward sweep over the columns.  The row stride is 65 floats, so a
// warp reading one column of 32 rows touches 32 different banks.
#pragma once

#include "pointfactor.cuh"

namespace ggp {

constexpr int kWideK = 64;   // largest k of this path
constexpr int kWideLd = 65;  // row stride of L in shared memory (floats)

struct WideWarp {
  float L[kWideK * kWideLd];  // M, then L = chol(M): lower triangle, row-major
  float4 x[kWideK];           // neighbour coordinates
  float y[kWideK];            // m, then y = L^-1 m, then beta = L^-T y, then b
  float g[kWideK];            // the diagonal of M during the factor; backward:
                              // right-hand side, then K_cc^-1 rhs
};

struct WideFactor {
  float sigma;
  bool clamped;     // a pivot or sigma^2 was floored
  float max_ratio;  // max_j M_jj / pivot_j
  float varw;       // Var(w)
  bool inc;         // increment form
};

// Factor of the point at xq whose k neighbour coordinates are in W.x.  All 32
// lanes call it; every lane returns the same WideFactor.
template <int KT>
__device__ __forceinline__ WideFactor point_factor_wide(WideWarp& W, int k, const KernF& kf,
                                                        float4 xq) {
  const int lane = threadIdx.x & 31;
  const float k0 = kf.s2 + kf.nug;
  const float nug = kf.nug;
  const bool inc = kappa_gamma_d2<KT>(kf, sqdist(W.x[0], xq)).g < 0.5f * kf.s2;
  // entries e = gamma (increment form) or kappa: W.L[a][c] = e_ac (c < a),
  // W.y[a] = e_ai
  for (int a = 1; a < k; a++) {
    const float4 xa = W.x[a];
    for (int c = lane; c < a; c += 32) {
      const KG kg = kappa_gamma_d2<KT>(kf, sqdist(xa, W.x[c]));
      W.L[a * kWideLd + c] = inc ? kg.g : kg.k;
    }
  }
  for (int a = lane; a < k; a += 32) {
    const KG kg = kappa_gamma_d2<KT>(kf, sqdist(W.x[a], xq));
    W.y[a] = inc ? kg.g : kg.k;
  }
  __syncwarp();
  const float e0i = W.y[0];
  if (inc) {  // M and m (column 0 last: its entries are g_a0)
    for (int a = 1; a < k; a++) {
      const float ga0 = W.L[a * kWideLd];
      for (int c = 1 + lane; c < a; c += 32)
        W.L[a * kWideLd + c] = ((ga0 + W.L[c * kWideLd]) - W.L[a * kWideLd + c]) + nug;
    }
    for (int a = 1 + lane; a < k; a += 32) {
      const float ga0 = W.L[a * kWideLd];
      W.L[a * kWideLd + a] = 2.0f * (ga0 + nug);
      W.g[a] = 2.0f * (ga0 + nug);
      W.y[a] = ((ga0 + e0i) - W.y[a]) + nug;
    }
    __syncwarp();
    for (int a = 1 + lane; a < k; a += 32) W.L[a * kWideLd] = -(W.L[a * kWideLd] + nug);
  } else {
    for (int a = 1 + lane; a < k; a += 32) {
      W.L[a * kWideLd + a] = k0;
      W.g[a] = k0;
    }
  }
  if (lane == 0) {
    W.L[0] = k0;
    W.g[0] = k0;
    W.y[0] = inc ? -(e0i + nug) : e0i;
  }
  __syncwarp();
  WideFactor r{0.0f, false, 1.0f, inc ? 2.0f * (e0i + nug) : k0, inc};
  DF s2{r.varw, 0.0f};
  const float pfloor = kPdFloor * k0;
  for (int j = 0; j < k; j++) {
    float piv = W.L[j * kWideLd + j];
    if (!(piv > pfloor)) {
      piv = pfloor;
      r.clamped = true;
    }
    const float ljj = sqrtf(piv);
    const float inv = 1.0f / ljj;
    r.max_ratio = fmaxf(r.max_ratio, W.g[j] * inv * inv);
    const float yj = W.y[j] * inv;
    s2 = df_sub_square(s2, yj);
    __syncwarp();  // every lane has read L_jj and y_j
    float l0 = 0.0f, l1 = 0.0f;
    const int a0 = j + 1 + lane, a1 = a0 + 32;
    if (a0 < k) {
      l0 = W.L[a0 * kWideLd + j] * inv;
      W.L[a0 * kWideLd + j] = l0;
      W.y[a0] = fmaf(-l0, yj, W.y[a0]);
    }
    if (a1 < k) {
      l1 = W.L[a1 * kWideLd + j] * inv;
      W.L[a1 * kWideLd + j] = l1;
      W.y[a1] = fmaf(-l1, yj, W.y[a1]);
    }
    if (lane == 0) {
      W.L[j * kWideLd + j] = ljj;
      W.y[j] = yj;
    }
    __syncwarp();
    // trailing update: L_ac -= L_aj L_cj for j < c <= a
    for (int c = j + 1; c < k; c++) {
      const float lcj = W.L[c * kWideLd + j];
      if (a0 < k && c <= a0) W.L[a0 * kWideLd + c] = fmaf(-l0, lcj, W.L[a0 * kWideLd + c]);
      if (a1 < k && c <= a1) W.L[a1 * kWideLd + c] = fmaf(-l1, lcj, W.L[a1 * kWideLd + c]);
    }
    __syncwarp();
  }
  float sig2 = s2.hi + s2.lo;
  if (!(sig2 > pfloor)) {
    sig2 = pfloor;
    r.clamped = true;
  }
  r.sigma = sqrtf(sig2);
  // beta = L^-T y, last entry first
  for (int j = k - 1; j >= 0; j--) {
    const float bj = W.y[j] * (1.0f / W.L[j * kWideLd + j]);
    __syncwarp();
    for (int a = lane; a < j; a += 32) W.y[a] = fmaf(-W.L[j * kWideLd + a], bj, W.y[a]);
    if (lane == 0) W.y[j] = bj;
    __syncwarp();
  }
  // increment form: b_0 = 1 + beta_0 - sum_{a>=1} beta_a
  if (lane == 0 && inc) {
    float sb = 0.0f;
    for (int a = 1; a < k; a++) sb += W.y[a];
    W.y[0] = (1.0f + W.y[0]) - sb;
  }
  __syncwarp();
  return r;
}

// W.g <- K_cc^-1 W.g = T^T M^-1 T W.g with the factor left in W.L by
// point_factor_wide.
__device__ __forceinline__ void wide_chol_solve(WideWarp& W, int k, bool inc) {
  const int lane = threadIdx.x & 31;
  if (inc) {
    const float r0 = W.g[0];
    __syncwarp();
    for (int a = 1 + lane; a < k; a += 32) W.g[a] -= r0;
    __syncwarp();
  }
  for (int j = 0; j < k; j++) {
    const float zj = W.g[j] * (1.0f / W.L[j * kWideLd + j]);
    __syncwarp();
    for (int a = j + 1 + lane; a < k; a += 32) W.g[a] = fmaf(-W.L[a * kWideLd + j], zj, W.g[a]);
    if (lane == 0) W.g[j] = zj;
    __syncwarp();
  }
  for (int j = k - 1; j >= 0; j--) {
    const float gj = W.g[j] * (1.0f / W.L[j * kWideLd + j]);
    __syncwarp();
    for (int a = lane; a < j; a += 32) W.g[a] = fmaf(-W.L[j * kWideLd + a], gj, W.g[a]);
    if (lane == 0) W.g[j] = gj;
    __syncwarp();
  }
  if (lane == 0 && inc) {
    float sg = 0.0f;
    for (int a = 1; a < k; a++) sg += W.g[a];
    W.g[0] -= sg;
  }
  __syncwarp();
}

// The rescue decision of the other paths (rescue.cuh), uniform over the warp.
__device__ __forceinline__ bool wide_needs_rescue(const WideWarp& W, const WideFactor& r, int k,
                                                  const KernF& kf) {
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (int a = lane; a < k; a += 32) bad |= !isfinite(W.y[a]);
  bad = __any_sync(0xffffffffu, bad);
  return bad || r.clamped || row_error_too_large(r.max_ratio, r.varw, r.sigma, kf) ||
         !isfinite(r.sigma);
}

}  // namespace ggp
