// Per-point conditional factor of Sec. 2.1 Eq. 2, computed by a group of G
// lanes of one warp (G = 8, 16 or 32 >= k).  Shared by the factor kernel and
// the adjoint kernels, which recompute the factors instead of storing them,
// so that both see bit-identical b and sigma.
//
// Lane a holds row a of K_cc in registers.  Left-looking Cholesky: at step j
// every lane forms its Schur value t_a = K_aj - sum_{m<j} L_am L_jm from its
// own row and row j of L (published in shared memory by lane j at earlier
// steps); lane j's t is the pivot.  The forward solve y = L^-1 K_ci rides
// along, sigma^2 = K_ii - y.y accumulates in compensated FP32 (exact
// two-product, two-sum), and b = L^-T y is a backward sweep over L's columns.
// Rows and columns k..G-1 are identity padding.  A pivot at or below 1e-7 of
// its diagonal entry is raised to that floor and flagged.
#pragma once

#include "common.cuh"

namespace ggp {

constexpr float kPdFloor = 1e-7f;

struct DF {  // double-float: value = hi + lo
  float hi, lo;
};

__device__ __forceinline__ DF df_sub_square(DF s, float y) {
  float p = __fmul_rn(y, y);
  float e = __fmaf_rn(y, y, -p);  // p + e == y*y exactly
  float t = __fsub_rn(s.hi, p);
  float bb = __fsub_rn(t, s.hi);
  float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(-p, bb));
  float lo = __fsub_rn(__fadd_rn(s.lo, err), e);
  float h = __fadd_rn(t, lo);
  float l = __fsub_rn(lo, __fsub_rn(h, t));
  return DF{h, l};
}

template <int G>
struct PointState {
  float A[G];      // row a of L (lower part valid)
  float D2[G];     // squared distances |x_a - x_b|^2 of row a
  float d2q;       // |x_a - x_i|^2
  float inv_own;   // 1 / L_aa
  float y_own;     // y_a
  float b_own;     // b_a
  float sigma;     // conditional standard deviation (same on all lanes)
  bool clamped;    // a pivot was floored (same on all lanes)
};

// Shared-memory row stride and per-group footprint (floats) for G lanes.
template <int G>
struct PFLayout {
  static constexpr int SG = G + 4;
  static constexpr int GS = G * SG + 4;
};

template <int G, int KT>
__device__ __forceinline__ void point_factor_group(PointState<G>& st, int a, int k,
                                                   const KernF& kf, float4 xa, float4 xq,
                                                   float* Lg) {
  constexpr int SG = PFLayout<G>::SG;
  const unsigned full = 0xffffffffu;
  const bool real = a < k;
  const float k0 = kf.s2 + kf.nug;
#pragma unroll
  for (int bcol = 0; bcol < G; bcol++) {
    float bx = __shfl_sync(full, xa.x, bcol, G);
    float by = __shfl_sync(full, xa.y, bcol, G);
    float bz = __shfl_sync(full, xa.z, bcol, G);
    float dx = xa.x - bx, dy = xa.y - by, dz = xa.z - bz;
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    st.D2[bcol] = d2;
    float kv = kappa_d2<KT>(kf, d2);
    bool both = real && bcol < k;
    st.A[bcol] = (bcol == a) ? (real ? k0 : 1.0f) : (both ? kv : 0.0f);
  }
  st.d2q = sqdist(xa, xq);
  float c = real ? kappa_d2<KT>(kf, st.d2q) : 0.0f;
  const float diag = real ? k0 : 1.0f;
  DF s2{k0, 0.0f};
  st.clamped = false;
  st.inv_own = 1.0f;
  st.y_own = 0.0f;
#pragma unroll
  for (int j = 0; j < G; j++) {
    if (j >= k) break;
    float tv = st.A[j];
    float t2 = 0.0f;
#pragma unroll
    for (int m = 0; m + 4 <= j; m += 4) {
      float4 r = *reinterpret_cast<const float4*>(Lg + j * SG + m);
      tv = fmaf(-st.A[m], r.x, tv);
      t2 = fmaf(-st.A[m + 1], r.y, t2);
      tv = fmaf(-st.A[m + 2], r.z, tv);
      t2 = fmaf(-st.A[m + 3], r.w, t2);
    }
#pragma unroll
    for (int m = (j / 4) * 4; m < j; m++) tv = fmaf(-st.A[m], Lg[j * SG + m], tv);
    tv += t2;
    float piv = __shfl_sync(full, tv, j, G);
    float pfloor = kPdFloor * __shfl_sync(full, diag, j, G);
    if (!(piv > pfloor)) {
      piv = pfloor;
      st.clamped = true;
    }
    float ljj = sqrtf(piv);
    float inv = 1.0f / ljj;
    float laj = (a == j) ? ljj : tv * inv;
    st.A[j] = laj;
    if (a == j) st.inv_own = inv;
    Lg[a * SG + j] = laj;
    float yj = __shfl_sync(full, c, j, G) * inv;
    if (a == j) st.y_own = yj;
    if (a > j) c = fmaf(-laj, yj, c);
    s2 = df_sub_square(s2, yj);
    __syncwarp(full);
  }
  float sig2 = s2.hi + s2.lo;
  if (!(sig2 > kPdFloor * k0)) {
    sig2 = kPdFloor * k0;
    st.clamped = true;
  }
  st.sigma = sqrtf(sig2);
  // b = L^-T y, last entry first; lane a keeps d_a = y_a - sum_{m>a} L_ma b_m
  float d = st.y_own;
  st.b_own = 0.0f;
#pragma unroll
  for (int j = G - 1; j >= 0; j--) {
    if (j >= k) continue;
    float bj = __shfl_sync(full, d * st.inv_own, j, G);
    if (a == j) st.b_own = bj;
    if (a < j) d = fmaf(-Lg[j * SG + a], bj, d);
  }
}

// Solves K_cc g = r for the factor held by the group (L rows in st.A and in
// Lg); lane a supplies r_a and receives g_a.
template <int G>
__device__ __forceinline__ float group_chol_solve(const PointState<G>& st, int a, int k,
                                                  float r, const float* Lg) {
  constexpr int SG = PFLayout<G>::SG;
  const unsigned full = 0xffffffffu;
  float z_own = 0.0f;
#pragma unroll
  for (int j = 0; j < G; j++) {
    if (j >= k) break;
    float zj = __shfl_sync(full, r * st.inv_own, j, G);
    if (a == j) z_own = zj;
    if (a > j) r = fmaf(-st.A[j], zj, r);
  }
  float d = z_own, g_own = 0.0f;
#pragma unroll
  for (int j = G - 1; j >= 0; j--) {
    if (j >= k) continue;
    float gj = __shfl_sync(full, d * st.inv_own, j, G);
    if (a == j) g_own = gj;
    if (a < j) d = fmaf(-Lg[j * SG + a], gj, d);
  }
  return g_own;
}

}  // namespace ggp
