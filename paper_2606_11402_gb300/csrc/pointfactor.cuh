// Per-point conditional factor of Sec. 2.1 Eq. 2 in FP32: the weights
// b_i = K_ic K_cc^-1 and sigma_i^2 = K_ii - K_ic K_cc^-1 K_ci.
//
// Increment form.  Where neighbours are close on the scale of the
// lengthscale, every entry of K_cc is close to kappa(0): FP32 keeps only the
// leading digits of kappa(r), and the Cholesky of K_cc then cancels them
// (condition numbers of 1e5-1e11 on the measured clouds).  Such rows are
// factored in increments of the field instead, an exact change of variables:
// with c_0 the nearest neighbour, z_0 = x(c_0), z_a = x(c_a) - x(c_0)
// (a >= 1) and the target w = x(i) - x(c_0),
//   M_00 = kappa(0) + nugget,       M_a0 = -(g_a0 + nugget),
//   M_ab = (g_a0 + g_b0) - g_ab + nugget (1 + [a = b]),
//   m_0  = -(g_0i + nugget),        m_a  = (g_a0 + g_0i) - g_ai + nugget,
//   Var(w) = 2 (g_0i + nugget),
// where g = kappa(0) - kappa(r) is the variogram, evaluated with a small
// relative error even as r -> 0 (gamma_d2).  With L = chol(M),
// y = L^-1 m and beta = L^-T y, E[w | z] = beta . z gives the weights
// b_a = beta_a (a >= 1), b_0 = 1 + beta_0 - sum_{a>=1} beta_a, and
// sigma^2 = Var(w) - y.y.  The change of variables is unit lower triangular,
// so the pivots of M equal those of K_cc (conditional variances) and the
// floor policy below is the covariance form's; only the rounding differs.
// K_cc^-1 r (the backward) is T^T M^-1 T r with (T r)_a = r_a - r_0.
// A row whose nearest neighbour is far (g_0i >= kappa(0) / 2) has small
// weights, which the recovery of b_0 would swamp with its rounding error; it
// keeps the covariance form (M = K_cc, m = K_ci, Var(w) = K_ii, b = beta,
// T = identity).  The choice is made per row from g_0i.
//
// A pivot at or below 1e-7 of kappa(0) + nugget is raised to that floor and
// flagged; so is sigma^2.  max_ratio = max_j M_jj / pivot_j (pivot after the
// floor) bounds the scaled condition number of M from below and gives the
// row's error estimate (rescue.cuh).
//
// Group form: a group of G lanes of one warp (G = 8, 16 or 32 >= k), lane a
// holding row a of M in registers.  Left-looking Cholesky: at step j every
// lane forms its Schur value t_a = M_aj - sum_{m<j} L_am L_jm from its own
// row and row j of L (published in shared memory by lane j at earlier
// steps); lane j's t is the pivot.  The forward solve y = L^-1 m rides along,
// sigma^2 = Var(w) - y.y accumulates in compensated FP32 (exact two-product,
// two-sum), and beta = L^-T y is a backward sweep over L's columns.  Rows and
// columns k..G-1 are identity padding.  Shared by the factor kernel and the
// adjoint kernels, which recompute the factors instead of storing them, so
// that both see bit-identical b and sigma.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "rescue.cuh"

namespace ggp {

constexpr float kPdFloor = 1e-7f;

// Running product of sigma^2 values in FP64 with a separate binary exponent
// (one log per thread at the end).
struct LogAcc {
  double m = 1.0;
  int e = 0;
  __device__ void mul(float sigma) {
    m *= (double)sigma * (double)sigma;
    int ex;
    m = frexp(m, &ex);
    e += ex;
  }
  __device__ double log_value() const { return log(m) + (double)e * 0.69314718055994530942; }
};

// Block-wide FP64 sum (blockDim.x a multiple of 32, at most 1024), added to
// *out.  The trailing barrier lets a kernel call it again at once: the
// shared partials are not overwritten while thread 0 still reads them.
__device__ inline void block_add_double(double v, double* out) {
  __shared__ double red[32];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    atomicAdd(out, s);
  }
  __syncthreads();
}

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
  float A[G];      // row a of M, then of L (lower part valid)
  float D2[G];     // squared distances |x_a - x_b|^2 of row a
  float d2q;       // |x_a - x_i|^2
  float inv_own;   // 1 / L_aa
  float y_own;     // y_a
  float b_own;     // b_a (covariance-form weight of neighbour a)
  float sigma;     // conditional standard deviation (same on all lanes)
  bool clamped;    // a pivot was floored (same on all lanes)
  float max_ratio; // max_j M_jj / pivot_j (same on all lanes)
  float varw;      // Var(w) (same on all lanes)
  bool inc;        // increment form (same on all lanes)
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
  const float nug = kf.nug;
  st.d2q = sqdist(xa, xq);
  const KG qa = kappa_gamma_d2<KT>(kf, st.d2q);
  st.inc = __shfl_sync(full, qa.g, 0, G) < 0.5f * kf.s2;
  const bool inc = st.inc;
  const float eai = inc ? qa.g : qa.k;  // entry (a, i) before the change of variables
  const float e0i = __shfl_sync(full, eai, 0, G);
  float ea0 = 0.0f;  // entry (a, 0)
#pragma unroll
  for (int bcol = 0; bcol < G; bcol++) {
    float bx = __shfl_sync(full, xa.x, bcol, G);
    float by = __shfl_sync(full, xa.y, bcol, G);
    float bz = __shfl_sync(full, xa.z, bcol, G);
    float dx = xa.x - bx, dy = xa.y - by, dz = xa.z - bz;
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    st.D2[bcol] = d2;
    const KG kg = kappa_gamma_d2<KT>(kf, d2);
    const float ev = inc ? kg.g : kg.k;
    if (bcol == 0) ea0 = ev;
    const float e0b = __shfl_sync(full, ev, 0, G);  // entry (0, bcol) from row 0
    const bool both = real && bcol < k;
    float m;
    if (bcol == a) {
      m = real ? ((a == 0 || !inc) ? k0 : 2.0f * (ea0 + nug)) : 1.0f;
    } else if (!inc) {
      m = ev;
    } else if (a == 0) {
      m = -(e0b + nug);
    } else if (bcol == 0) {
      m = -(ea0 + nug);
    } else {
      m = ((ea0 + e0b) - ev) + nug;
    }
    st.A[bcol] = both || bcol == a ? m : 0.0f;
  }
  float c = !real ? 0.0f
                  : !inc ? eai : (a == 0 ? -(e0i + nug) : ((ea0 + e0i) - eai) + nug);
  st.varw = inc ? 2.0f * (e0i + nug) : k0;
  DF s2{st.varw, 0.0f};
  const float pfloor = kPdFloor * k0;
  st.clamped = false;
  st.max_ratio = 1.0f;
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
    const float mjj = __shfl_sync(full, st.A[j], j, G);
    tv += t2;
    float piv = __shfl_sync(full, tv, j, G);
    if (!(piv > pfloor)) {
      piv = pfloor;
      st.clamped = true;
    }
    float ljj = sqrtf(piv);
    float inv = 1.0f / ljj;
    st.max_ratio = fmaxf(st.max_ratio, mjj * inv * inv);
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
  if (!(sig2 > pfloor)) {
    sig2 = pfloor;
    st.clamped = true;
  }
  st.sigma = sqrtf(sig2);
  // beta = L^-T y, last entry first; lane a keeps d_a = y_a - sum_{m>a} L_ma beta_m
  float d = st.y_own;
  st.b_own = 0.0f;
#pragma unroll
  for (int j = G - 1; j >= 0; j--) {
    if (j >= k) continue;
    float bj = __shfl_sync(full, d * st.inv_own, j, G);
    if (a == j) st.b_own = bj;
    if (a < j) d = fmaf(-Lg[j * SG + a], bj, d);
  }
  // increment form: b_0 = 1 + beta_0 - sum_{a>=1} beta_a (summed in lane order)
  float sb = 0.0f;
#pragma unroll
  for (int j = 1; j < G; j++) sb += __shfl_sync(full, st.b_own, j, G);
  if (a == 0 && inc) st.b_own = (1.0f + st.b_own) - sb;
}

// Solves K_cc g = r for the factor held by the group (L rows in st.A and in
// Lg): g = T^T M^-1 T r.  Lane a supplies r_a (zero for a >= k) and receives
// g_a.
template <int G>
__device__ __forceinline__ float group_chol_solve(const PointState<G>& st, int a, int k,
                                                  float r, const float* Lg) {
  constexpr int SG = PFLayout<G>::SG;
  const unsigned full = 0xffffffffu;
  const float r0 = __shfl_sync(full, r, 0, G);
  if (st.inc && a >= 1 && a < k) r -= r0;
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
  float sg = 0.0f;
#pragma unroll
  for (int j = 1; j < G; j++) sg += __shfl_sync(full, g_own, j, G);
  if (a == 0 && st.inc) g_own -= sg;
  return g_own;
}



// ---- one thread per point (k <= 16) ----------------------------------------
// The same arithmetic as point_factor_group, element by element and in the
// same order, but with the whole lower triangle of L in one thread's
// registers: no shuffles, no shared memory, each variogram value evaluated
// once (the group form evaluates every row in full on its lanes).  K is the padded
// row length (4, 8, 12 or 16); entries a >= k are identity padding, which
// passes through every step without changing the real entries (unit pivot,
// zero off-diagonal, zero right-hand side), so all loops run K steps.  The
// column loops are unrolled at compile time (static_for) so that every
// register-array index is a constant.

__host__ __device__ constexpr int tri(int a, int c) { return a * (a + 1) / 2 + c; }

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

template <int K>
struct PointRegs {
  float L[K * (K + 1) / 2];  // M, then L = chol(M): L[tri(a, c)], c <= a
  float y[K];                // m, y = L^-1 m, beta = L^-T y, then b (zero for a >= k)
  float sigma;
  bool clamped;
  float max_ratio;           // max_j M_jj / pivot_j
  float varw;                // Var(w)
  bool inc;                  // increment form
  // 1 / L_jj, recomputed where needed (the same correctly rounded quotient)
  __device__ __forceinline__ float inv(int j) const { return 1.0f / L[tri(j, j)]; }
};

// Schur value t = K_aj - sum_{m<j} L_am L_jm with the group form's two
// accumulators (m = 0, 2 mod 4 and m = 1, 3 mod 4 over whole blocks of four).
template <int K, int J, int A>
__device__ __forceinline__ float schur_value(const PointRegs<K>& p) {
  float tv = p.L[tri(A, J)];
  float t2 = 0.0f;
#pragma unroll
  for (int m = 0; m + 4 <= J; m += 4) {
    tv = fmaf(-p.L[tri(A, m)], p.L[tri(J, m)], tv);
    t2 = fmaf(-p.L[tri(A, m + 1)], p.L[tri(J, m + 1)], t2);
    tv = fmaf(-p.L[tri(A, m + 2)], p.L[tri(J, m + 2)], tv);
    t2 = fmaf(-p.L[tri(A, m + 3)], p.L[tri(J, m + 3)], t2);
  }
#pragma unroll
  for (int m = (J / 4) * 4; m < J; m++) tv = fmaf(-p.L[tri(A, m)], p.L[tri(J, m)], tv);
  return tv + t2;
}

// Shared-memory staging of the one-thread-per-point kernels (blocks of
// kThreadBlock threads).  Evaluating the kernel values of a conditional
// fully unrolled, with the whole factor live in registers, made the code
// larger than the instruction cache (ncu: "no instruction" was the largest
// stall).  The thread instead stages its k neighbour coordinates and then
// its k(k-1)/2 + k kernel values in shared memory in a rolled loop, and the
// unrolled factor reads them back.  Entry e of thread t sits at
// [e * kThreadBlock + t] (consecutive threads, consecutive words).
constexpr int kThreadBlock = 128;

template <int K>
struct ThreadStage {
  static constexpr int kPairs = K * (K - 1) / 2;            // (a, c), c < a
  static constexpr int kEntries = kPairs + K;                // and (a, i)
  static constexpr size_t kBytes = (size_t)kThreadBlock * (16 * K + 4 * kEntries);
  float4* X;  // neighbour coordinates, X[a * kThreadBlock]
  float* E;   // kernel values, E[e * kThreadBlock]
  __device__ __forceinline__ ThreadStage(unsigned char* smem) {
    X = reinterpret_cast<float4*>(smem) + threadIdx.x;
    E = reinterpret_cast<float*>(smem + (size_t)16 * K * kThreadBlock) + threadIdx.x;
  }
};

__host__ __device__ constexpr int pair_ix(int a, int c) { return a * (a - 1) / 2 + c; }

// Loads the k neighbour coordinates of a row (int4 index loads, float4
// gathers) into the stage; entries k..K-1 are not written.
template <int K>
__device__ __forceinline__ void stage_coords(const ThreadStage<K>& st,
                                             const float4* __restrict__ xs,
                                             const int32_t* __restrict__ row, int k) {
#pragma unroll
  for (int q = 0; q < K / 4; q++) {
    if (4 * q >= k) break;
    const int4 c = __ldg(reinterpret_cast<const int4*>(row) + q);
    st.X[(4 * q) * kThreadBlock] = __ldg(xs + c.x);
    if (4 * q + 1 < k) st.X[(4 * q + 1) * kThreadBlock] = __ldg(xs + c.y);
    if (4 * q + 2 < k) st.X[(4 * q + 2) * kThreadBlock] = __ldg(xs + c.z);
    if (4 * q + 3 < k) st.X[(4 * q + 3) * kThreadBlock] = __ldg(xs + c.w);
  }
}

// The factor of the row whose coordinates stage_coords put in `st`.
template <int K, int KT>
__device__ __forceinline__ void point_factor_thread(PointRegs<K>& p, int k, const KernF& kf,
                                                    const ThreadStage<K>& st, float4 xq) {
  const float k0 = kf.s2 + kf.nug;
  const float nug = kf.nug;
  const KG q0 = kappa_gamma_d2<KT>(kf, sqdist(st.X[0], xq));
  const bool inc = q0.g < 0.5f * kf.s2;
  p.inc = inc;
  // gamma (increment form) or kappa (covariance form) of every pair and of
  // every neighbour with the point, in a rolled loop taking four pairs per
  // iteration: their coordinates are read before any value is stored, so
  // the four evaluations overlap
#pragma unroll 1
  for (int a = 1; a < k; a++) {
    const float4 xa = st.X[a * kThreadBlock];
    float* ea = st.E + pair_ix(a, 0) * kThreadBlock;
    int c = 0;
#pragma unroll 1
    for (; c + 4 <= a; c += 4) {
      float4 xc[4];
#pragma unroll
      for (int u = 0; u < 4; u++) xc[u] = st.X[(c + u) * kThreadBlock];
      float e[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const KG kg = kappa_gamma_d2<KT>(kf, sqdist(xa, xc[u]));
        e[u] = inc ? kg.g : kg.k;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) ea[(c + u) * kThreadBlock] = e[u];
    }
#pragma unroll 1
    for (; c < a; c++) {
      const KG kg = kappa_gamma_d2<KT>(kf, sqdist(xa, st.X[c * kThreadBlock]));
      ea[c * kThreadBlock] = inc ? kg.g : kg.k;
    }
    const KG kq = kappa_gamma_d2<KT>(kf, sqdist(xa, xq));
    st.E[(ThreadStage<K>::kPairs + a) * kThreadBlock] = inc ? kq.g : kq.k;
  }
  // into registers; padding rows and columns (a >= k) are zero
  static_for<1, K>([&](auto Ar) {
    constexpr int a = decltype(Ar)::value;
    const bool real = a < k;
#pragma unroll
    for (int c = 0; c < a; c++) p.L[tri(a, c)] = real ? st.E[pair_ix(a, c) * kThreadBlock] : 0.0f;
    p.y[a] = real ? st.E[(ThreadStage<K>::kPairs + a) * kThreadBlock] : 0.0f;
  });
  p.y[0] = inc ? q0.g : q0.k;
  // M and m (column 0 last: in the increment form its entries are g_a0)
  const float e0i = p.y[0];
  static_for<1, K>([&](auto Ac) {
    constexpr int a = decltype(Ac)::value;
    const bool real = a < k;
    const float ea0 = p.L[tri(a, 0)];
#pragma unroll
    for (int c = 1; c < a; c++)
      p.L[tri(a, c)] = real ? (inc ? ((ea0 + p.L[tri(c, 0)]) - p.L[tri(a, c)]) + nug : p.L[tri(a, c)])
                            : 0.0f;
    p.L[tri(a, a)] = real ? (inc ? 2.0f * (ea0 + nug) : k0) : 1.0f;
    p.y[a] = real ? (inc ? ((ea0 + e0i) - p.y[a]) + nug : p.y[a]) : 0.0f;
  });
#pragma unroll
  for (int a = 1; a < K; a++)
    p.L[tri(a, 0)] = a < k ? (inc ? -(p.L[tri(a, 0)] + nug) : p.L[tri(a, 0)]) : 0.0f;
  p.L[tri(0, 0)] = k0;
  p.y[0] = inc ? -(e0i + nug) : e0i;
  p.varw = inc ? 2.0f * (e0i + nug) : k0;
  DF s2{p.varw, 0.0f};
  bool clamped = false;
  float max_ratio = 1.0f;
  const float pfloor = kPdFloor * k0;
  static_for<0, K>([&](auto Jc) {
    constexpr int j = decltype(Jc)::value;
    const float mjj = p.L[tri(j, j)];
    float piv = schur_value<K, j, j>(p);
    if (!(piv > pfloor)) {
      piv = pfloor;
      clamped = true;
    }
    const float ljj = sqrtf(piv);
    const float inv = 1.0f / ljj;
    max_ratio = fmaxf(max_ratio, mjj * inv * inv);  // padding: 1
    static_for<j + 1, K>([&](auto Ac) {
      constexpr int a = decltype(Ac)::value;
      p.L[tri(a, j)] = schur_value<K, j, a>(p) * inv;
    });
    p.L[tri(j, j)] = ljj;
    const float yj = p.y[j] * inv;
    p.y[j] = yj;
#pragma unroll
    for (int a = j + 1; a < K; a++) p.y[a] = fmaf(-p.L[tri(a, j)], yj, p.y[a]);
    s2 = df_sub_square(s2, yj);
  });
  float sig2 = s2.hi + s2.lo;
  if (!(sig2 > pfloor)) {
    sig2 = pfloor;
    clamped = true;
  }
  p.clamped = clamped;
  p.max_ratio = max_ratio;
  p.sigma = sqrtf(sig2);
  // beta = L^-T y, last entry first
  static_for<0, K>([&](auto Jr) {
    constexpr int j = K - 1 - decltype(Jr)::value;
    const float bj = p.y[j] * p.inv(j);
    p.y[j] = bj;
#pragma unroll
    for (int a = 0; a < j; a++) p.y[a] = fmaf(-p.L[tri(j, a)], bj, p.y[a]);
  });
  // increment form: b_0 = 1 + beta_0 - sum_{a>=1} beta_a (padding entries are zero)
  float sb = 0.0f;
#pragma unroll
  for (int a = 1; a < K; a++) sb += p.y[a];
  if (inc) p.y[0] = (1.0f + p.y[0]) - sb;
}

// Solves K_cc g = r in place with the factor of point_factor_thread
// (g = T^T M^-1 T r, same operation order as group_chol_solve); r must be
// zero at padding entries.
template <int K>
__device__ __forceinline__ void thread_chol_solve(const PointRegs<K>& p, int k, float (&r)[K]) {
#pragma unroll
  for (int a = 1; a < K; a++)
    if (p.inc && a < k) r[a] -= r[0];
  static_for<0, K>([&](auto Jc) {
    constexpr int j = decltype(Jc)::value;
    const float zj = r[j] * p.inv(j);
    r[j] = zj;
#pragma unroll
    for (int a = j + 1; a < K; a++) r[a] = fmaf(-p.L[tri(a, j)], zj, r[a]);
  });
  static_for<0, K>([&](auto Jr) {
    constexpr int j = K - 1 - decltype(Jr)::value;
    const float gj = r[j] * p.inv(j);
    r[j] = gj;
#pragma unroll
    for (int a = 0; a < j; a++) r[a] = fmaf(-p.L[tri(j, a)], gj, r[a]);
  });
  float sg = 0.0f;
#pragma unroll
  for (int a = 1; a < K; a++) sg += r[a];
  if (p.inc) r[0] -= sg;
}

// Whether a conditional computed in FP32 must be recomputed in FP64 (see
// rescue.cuh): a floored pivot or sigma^2, a row-error estimate above the
// kernel's threshold, or a non-finite weight or sigma.
template <int K>
__device__ __forceinline__ bool needs_rescue(const PointRegs<K>& p, int k, const KernF& kf) {
  bool bad = p.clamped || row_error_too_large(p.max_ratio, p.varw, p.sigma, kf) ||
             !isfinite(p.sigma);
#pragma unroll
  for (int a = 0; a < K; a++) bad |= !isfinite(p.y[a]);
  return bad;
}

// Shared memory of the warp-cooperative FP64 rescue (rescue.cuh) for one warp
// of a one-thread-per-point kernel: K (K + 1) doubles.
template <int K>
__host__ __device__ constexpr size_t warp_rescue_bytes() { return (size_t)K * (K + 1) * sizeof(double); }

// The rows of the warp's lanes with `need` set are recomputed in FP64, one
// row at a time by the whole warp (warp_row_factor64); each such lane
// receives its b (zero past k), sigma and floor flag, rounded to FP32.  Every
// lane of the warp must call this (a collective); W is the warp's shared
// memory of warp_rescue_bytes<K>().
template <int K, int KT>
__device__ __forceinline__ void warp_rescue(PointRegs<K>& p, bool need,
                                            const float4* __restrict__ xs, const int32_t* row,
                                            int k, float4 xq, const KernF& kf, double* W) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(full, need);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const int32_t* r = reinterpret_cast<const int32_t*>(
        __shfl_sync(full, reinterpret_cast<unsigned long long>(row), src));
    float4 q;
    q.x = __shfl_sync(full, xq.x, src);
    q.y = __shfl_sync(full, xq.y, src);
    q.z = __shfl_sync(full, xq.z, src);
    q.w = 0.0f;
    const WarpRow64 w = warp_row_factor64<K, KT>(xs, r, k, q, kf, W);
    float* bf = reinterpret_cast<float*>(W);
    bf[lane] = (float)w.b;
    __syncwarp();
    if (lane == src) {
#pragma unroll
      for (int a = 0; a < K; a++) p.y[a] = a < k ? bf[a] : 0.0f;
      p.sigma = (float)w.sigma;
      p.clamped = w.clamped;
    }
    __syncwarp();
  }
}

// Dynamic shared memory of the one-thread-per-point fused kernels: the
// staging area, then each warp's FP64 rescue workspace.
template <int K>
constexpr size_t fused_smem() { return ThreadStage<K>::kBytes + 4 * warp_rescue_bytes<K>(); }

template <int K>
__device__ __forceinline__ double* fused_rescue_ws(unsigned char* smem) {
  return reinterpret_cast<double*>(smem + ThreadStage<K>::kBytes) +
         (threadIdx.x >> 5) * (warp_rescue_bytes<K>() / sizeof(double));
}

}  // namespace ggp
