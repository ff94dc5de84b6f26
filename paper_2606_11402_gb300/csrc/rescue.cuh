// FP64 rescue of single conditionals (Sec. 2.1 Eq. 2).
//
// The per-point factors run in FP32 (pointfactor.cuh).  Their error grows
// like the scaled condition number of the matrix the row factors times
// 2^-24 (max_j M_jj / pivot_j, read off the FP32 Cholesky, bounds it from
// below), and sigma^2 = Var(w) - y.y loses a further factor
// Var(w) / sigma^2 to cancellation where the conditional variance is tiny
// (clouds without nugget).  The row's error estimate is
//   est = 2^-20 max_j (M_jj / pivot_j) (1 + 2^-8 Var(w) / sigma^2).
// On FP32 emulations of the increment form (headline, differentiation,
// clustered and tiny clouds, 4000 rows each) the element-wise sigma error
// stays below 1.2 est and the weights' relative error below 2 est on 99 % of
// the rows.  A row whose estimate exceeds the
// kernel's rescue_tol (graphgp.h), whose FP32 factor floored a pivot or
// sigma^2, or whose b or sigma is not finite is recomputed here in FP64 from
// the FP32 coordinates, in the covariance form of Eq. 2: kernel values from
// FP64 distances, Cholesky by rows, forward and backward solves,
// sigma^2 = K_ii - y.y, with the same pivot floor (1e-7 of the diagonal).
// Every kernel that evaluates a conditional (factor, on-the-fly sweeps,
// factor backward) takes the same decision on the same FP32 values and calls
// the same code, so stored and recomputed factors agree.
#pragma once

#include "common.cuh"

namespace ggp {

constexpr double kPdFloor64 = 1e-7;

// The row-error estimate above against the kernel's threshold (kf.resc_T =
// rescue_tol 2^24, negative = every row): true when the FP32 row must be
// recomputed.  A non-positive pivot makes the ratio negative or infinite;
// such rows were floored and are rescued by the caller's clamp test anyway.
__device__ __forceinline__ bool row_error_too_large(float max_ratio, float varw, float sigma,
                                                    const KernF& kf) {
  const float canc = varw / (sigma * sigma);
  return !(max_ratio * (16.0f + 0.0625f * canc) <= kf.resc_T);
}

__host__ __device__ constexpr int tri64(int a, int c) { return a * (a + 1) / 2 + c; }

template <int KT>
__device__ __forceinline__ double kappa64(const KernF& p, double r) {
  const double s2 = p.s2d, l = p.elld;
  if (KT == GRAPHGP_SQEXP) return s2 * exp(-0.5 * (r / l) * (r / l));
  if (KT == GRAPHGP_MATERN12) return s2 * exp(-r / l);
  if (KT == GRAPHGP_MATERN32) {
    const double a = 1.7320508075688772 * r / l;
    return s2 * (1.0 + a) * exp(-a);
  }
  const double a = 2.2360679774997896 * r / l;
  return s2 * (1.0 + a + a * a / 3.0) * exp(-a);
}

template <int KT>
__device__ __forceinline__ double dkappa64_dell(const KernF& p, double r) {
  const double s2 = p.s2d, l = p.elld;
  if (KT == GRAPHGP_SQEXP) return s2 * exp(-0.5 * (r / l) * (r / l)) * r * r / (l * l * l);
  if (KT == GRAPHGP_MATERN12) return s2 * exp(-r / l) * r / (l * l);
  if (KT == GRAPHGP_MATERN32) {
    const double a = 1.7320508075688772 * r / l;
    return s2 * a * a * exp(-a) / l;
  }
  const double a = 2.2360679774997896 * r / l;
  return s2 * a * a * (1.0 + a) * exp(-a) / (3.0 * l);
}

__device__ __forceinline__ double dist64(float4 a, float4 b) {
  const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y,
               dz = (double)a.z - (double)b.z;
  return sqrt(dx * dx + dy * dy + dz * dz);
}

// Row state of the FP64 conditional: L (packed lower), b, sigma.
template <int KMAX>
struct Row64 {
  double L[KMAX * (KMAX + 1) / 2];
  double b[KMAX];
  double sigma;
  bool clamped;
};

// Factor of the row with neighbours row[0..k) (indices into xs) and point xq.
template <int KMAX, int KT>
__device__ __noinline__ void row_factor64(Row64<KMAX>& R, const float4* __restrict__ xs,
                                          const int32_t* row, int k, float4 xq, const KernF& p) {
  const double k0 = kappa64<KT>(p, 0.0) + p.nugd;
  R.clamped = false;
  for (int i = 0; i < k; i++) {
    const float4 xi = __ldg(xs + row[i]);
    for (int j = 0; j <= i; j++) {
      double s = (i == j) ? k0 : kappa64<KT>(p, dist64(xi, __ldg(xs + row[j])));
      for (int m = 0; m < j; m++) s -= R.L[tri64(i, m)] * R.L[tri64(j, m)];
      if (i == j) {
        const double fl = kPdFloor64 * k0;
        if (!(s > fl)) {
          s = fl;
          R.clamped = true;
        }
        R.L[tri64(i, i)] = sqrt(s);
      } else {
        R.L[tri64(i, j)] = s / R.L[tri64(j, j)];
      }
    }
    R.b[i] = kappa64<KT>(p, dist64(xi, xq));
  }
  // y = L^-1 K_ci, sigma^2 = K_ii - y.y, b = L^-T y
  for (int i = 0; i < k; i++) {
    double s = R.b[i];
    for (int m = 0; m < i; m++) s -= R.L[tri64(i, m)] * R.b[m];
    R.b[i] = s / R.L[tri64(i, i)];
  }
  double s2 = k0;
  for (int i = 0; i < k; i++) s2 -= R.b[i] * R.b[i];
  if (!(s2 > kPdFloor64 * k0)) {
    s2 = kPdFloor64 * k0;
    R.clamped = true;
  }
  R.sigma = sqrt(s2);
  for (int i = k - 1; i >= 0; i--) {
    double s = R.b[i];
    for (int m = i + 1; m < k; m++) s -= R.L[tri64(m, i)] * R.b[m];
    R.b[i] = s / R.L[tri64(i, i)];
  }
}

// The FP64 conditional of one row computed by a whole warp (k <= KMAX <= 32):
// lane a owns neighbour a and row a of K_cc in shared memory (W: KMAX x
// (KMAX + 1) doubles per warp).  Lane a evaluates its row of kernel values (FP64 distances from the
// FP32 coordinates), then a right-looking Cholesky by columns with the pivot
// floor of row_factor64 (1e-7 of the diagonal), the forward solve riding
// along and sigma^2 = K_ii - y.y summed in column order, and the backward
// solve b = L^-T y.  A single thread needs k(k+1)/2 FP64 exponentials and
// k^3/6 dependent FP64 multiply-adds for a row, at the low FP64 rate of this
// GPU; the warp spreads both over its lanes.  Every path that rescues a row
// with k <= 32 (factor, on-the-fly sweeps) uses this routine, so stored and
// recomputed factors agree bit for bit.  All 32 lanes must call it with the
// same arguments; lane a receives b_a (0 for a >= k).
struct WarpRow64 {
  double b;       // this lane's weight
  double sigma;   // same on every lane
  bool clamped;   // same on every lane
};

template <int KMAX, int KT>
__device__ __noinline__ WarpRow64 warp_row_factor64(const float4* __restrict__ xs,
                                                    const int32_t* row, int k, float4 xq,
                                                    const KernF& p, double* W) {
  static_assert(KMAX <= 32, "one lane per neighbour");
  constexpr int LD = KMAX + 1;
  const unsigned full = 0xffffffffu;
  const int a = threadIdx.x & 31;
  const bool real = a < k;
  const double k0 = kappa64<KT>(p, 0.0) + p.nugd;
  const float4 xa = real ? __ldg(xs + row[a]) : make_float4(0.f, 0.f, 0.f, 0.f);
  double* La = W + a * LD;
  for (int c = 0; c < k; c++) {
    float4 xc;
    xc.x = __shfl_sync(full, xa.x, c);
    xc.y = __shfl_sync(full, xa.y, c);
    xc.z = __shfl_sync(full, xa.z, c);
    if (real && c < a) La[c] = kappa64<KT>(p, dist64(xa, xc));
  }
  double y = real ? kappa64<KT>(p, dist64(xa, xq)) : 0.0;
  if (real) La[a] = k0;
  __syncwarp();
  const double fl = kPdFloor64 * k0;
  bool clamped = false;
  double s2 = k0;
  for (int j = 0; j < k; j++) {
    double piv = __shfl_sync(full, a == j ? La[j] : 0.0, j);
    if (!(piv > fl)) {
      piv = fl;
      clamped = true;
    }
    const double ljj = sqrt(piv);
    const double yj = __shfl_sync(full, y, j) / ljj;
    s2 -= yj * yj;
    double laj = 0.0;
    if (real && a > j) {
      laj = La[j] / ljj;
      La[j] = laj;
      y -= laj * yj;
    }
    if (a == j) {
      La[j] = ljj;
      y = yj;
    }
    __syncwarp();
    // trailing update of row a: L_ac -= L_aj L_cj for j < c <= a
    if (real && a > j)
      for (int c = j + 1; c <= a; c++) La[c] -= laj * W[c * LD + j];
    __syncwarp();
  }
  if (!(s2 > fl)) {
    s2 = fl;
    clamped = true;
  }
  // b = L^-T y, last entry first
  double d = y;
  double b = 0.0;
  for (int j = k - 1; j >= 0; j--) {
    const double bj = __shfl_sync(full, a == j ? d / La[j] : 0.0, j);
    if (a == j) b = bj;
    if (real && a < j) d -= W[j * LD + a] * bj;
  }
  __syncwarp();
  return WarpRow64{real ? b : 0.0, sqrt(s2), clamped};
}

// The row's contribution to thetabar = (d/dl, d/dsigma2, d/dnugget) from the
// cotangents of its weights, bbar_a = alpha v_c(a), and of its conditional
// standard deviation, sigbar (Sec. 2.3; with s = sigma^2, g = K_cc^-1 bbar:
// Kbar_cc = -g b^T + sbar b b^T, Kbar_ci = g - 2 sbar b, Kbar_ii = sbar).
// R holds the row's factor; sigma is the FP32 value the sweeps used.
template <int KMAX, int KT>
__device__ __noinline__ void row_backward64(const Row64<KMAX>& R, const float4* __restrict__ xs,
                                            const int32_t* row, int k, float4 xq, const KernF& p,
                                            const float* __restrict__ v, double alpha,
                                            double sigbar, double sigma, double& tl, double& ts,
                                            double& tn) {
  double g[KMAX];
  const double sbar = sigbar / (2.0 * sigma);
  for (int i = 0; i < k; i++) g[i] = alpha * (double)v[row[i]];
  for (int i = 0; i < k; i++) {
    double s = g[i];
    for (int m = 0; m < i; m++) s -= R.L[tri64(i, m)] * g[m];
    g[i] = s / R.L[tri64(i, i)];
  }
  for (int i = k - 1; i >= 0; i--) {
    double s = g[i];
    for (int m = i + 1; m < k; m++) s -= R.L[tri64(m, i)] * g[m];
    g[i] = s / R.L[tri64(i, i)];
  }
  double pl = 0.0, ps = sbar, pn = sbar;  // Kbar_ii = sbar
  for (int a = 0; a < k; a++) {
    const float4 xa = __ldg(xs + row[a]);
    const double kaa = -g[a] * R.b[a] + sbar * R.b[a] * R.b[a];
    ps += kaa;
    pn += kaa;
    for (int c = 0; c < a; c++) {
      const double kb = (-g[a] * R.b[c] + sbar * R.b[a] * R.b[c]) + (-g[c] * R.b[a] + sbar * R.b[c] * R.b[a]);
      const double r = dist64(xa, __ldg(xs + row[c]));
      ps += kb * kappa64<KT>(p, r) / p.s2d;
      pl += kb * dkappa64_dell<KT>(p, r);
    }
    const double kci = g[a] - 2.0 * sbar * R.b[a];
    const double r = dist64(xa, xq);
    ps += kci * kappa64<KT>(p, r) / p.s2d;
    pl += kci * dkappa64_dell<KT>(p, r);
  }
  tl += pl;
  ts += ps;
  tn += pn;
}

}  // namespace ggp
