// Per-point conditioning factors (Sec. 2.1 Eq. 2; Alg. 1) and the dense
// initial block (the dense initial batch of Alg. 1; Sec. 2.2 "Batch
// construction").
//
// Per point i with c = c(i): b_i = K_ic K_cc^-1 and sigma_i^2 =
// K_ii - K_ic K_cc^-1 K_ci.  A group of G lanes (G = 8, 16 or 32 >= k) of one
// warp owns one point; lane a holds row a of K_cc in registers.  The
// Cholesky factor is built column by column (left-looking): at step j every
// lane forms its Schur value from its own row and row j of L, which lane j
// published to shared memory in earlier steps; lane j's value is the pivot.
// The forward solve y = L^-1 K_ci rides along (right-looking on the lanes'
// K_ci entries), sigma^2 = K_ii - y.y is accumulated in compensated FP32
// (two-sum / two-product), and b = L^-T y is a backward sweep reading L's
// columns from shared memory.  Pivots below 1e-7 of their diagonal entry are
// raised to that floor and counted.  logdet = sum log sigma_i^2 is reduced in
// FP64 from the stored FP32 sigma (a running FP64 product with separate
// exponent, one log per thread).
#include "pointwide.cuh"

namespace ggp {
namespace {

// Rows whose FP32 factor needs the FP64 rescue (rescue.cuh) are listed here
// and recomputed afterwards by factor_rescue_kernel, one thread per row, so
// that a warp does not stall on the FP64 row of one of its points.  A row
// that finds the list full is recomputed in place.
struct RescueList {
  int64_t* rows;
  unsigned long long* count;
  unsigned long long cap;
  __device__ __forceinline__ bool defer(int64_t i) const {
    const unsigned long long slot = atomicAdd(count, 1ull);
    if (slot < cap) {
      rows[slot] = i;
      return true;
    }
    return false;
  }
};

// The rows [t0, t1) of the sparse positions, seen by the factor kernels as a
// graph of their own: positions n0 + t0 .. n0 + t1 - 1, neighbour and weight
// rows shifted by t0 (position indices stay global).
struct RowView {
  const int32_t* nbr;
  float* b;
  int64_t N, n0;
};

template <int G, int KT>
__global__ void __launch_bounds__(128) point_factor_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int kp,
    int64_t n0, KernF kf, float* __restrict__ b_out, float* __restrict__ sigma_out,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd, RescueList rl) {
  constexpr int PPW = 32 / G;  // points per warp
  constexpr int GS = PFLayout<G>::GS;
  __shared__ __align__(16) float Ls[4 * PPW * GS];
  // FP64 rescue workspace of each warp (dynamic: 4 G (G + 1) doubles)
  extern __shared__ __align__(16) double gwsm[];
  double* Wwarp = gwsm + (threadIdx.x >> 5) * (G * (G + 1));
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int a = lane % G;
  const int warp = threadIdx.x >> 5;
  float* Lg = Ls + (warp * PPW + grp) * GS;
  LogAcc acc;
  unsigned long long clamped_rows = 0;
  const int64_t total_groups = (int64_t)gridDim.x * 4 * PPW;
  const int64_t gid = ((int64_t)blockIdx.x * 4 + warp) * PPW + grp;
  const int64_t npts = N - n0;
  const int64_t iters = (npts + total_groups - 1) / total_groups;
  for (int64_t it = 0; it < iters; it++) {
    int64_t t = it * total_groups + gid;
    bool valid = t < npts;
    int64_t i = n0 + (valid ? t : 0);
    int32_t ca = a < k ? nbr[(i - n0) * kp + a] : 0;
    PointState<G> st;
    point_factor_group<G, KT>(st, a, k, kf, xs[ca], xs[i], Lg);
    __syncwarp();
    // rescue decision, uniform over the group's lanes
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const bool lane_bad = a < k && !isfinite(st.b_own);
    const bool rescue = st.clamped || row_error_too_large(st.max_ratio, st.varw, st.sigma, kf) ||
                        !isfinite(st.sigma) || (__ballot_sync(0xffffffffu, lane_bad) & gmask);
    static_assert(G == 32, "the group factor kernel runs one point per warp");
    bool deferred = false;
    if (valid && rescue && a == 0) deferred = rl.defer(i);
    deferred = __shfl_sync(0xffffffffu, deferred, 0);
    if (valid && rescue && !deferred) {  // list full: the warp recomputes the row in place
      const WarpRow64 w = warp_row_factor64<G, KT>(xs, nbr + (i - n0) * kp, k, xs[i], kf, Wwarp);
      if (a < kp) b_out[(i - n0) * kp + a] = a < k ? (float)w.b : 0.0f;
      if (a == 0) {
        const float sg = (float)w.sigma;
        sigma_out[i] = sg;
        acc.mul(sg);
        if (w.clamped) clamped_rows++;
      }
    }
    if (valid && !deferred) {
      if (rescue) {
      } else {
        if (a < kp) b_out[(i - n0) * kp + a] = a < k ? st.b_own : 0.0f;
        if (a == 0) {
          sigma_out[i] = st.sigma;
          acc.mul(st.sigma);
          if (st.clamped) clamped_rows++;
        }
      }
    }
  }
  double lv = (a == 0) ? acc.log_value() : 0.0;
  block_add_double(lv, logdet);
  for (int o = 16; o; o >>= 1) clamped_rows += __shfl_xor_sync(0xffffffffu, clamped_rows, o);
  if (lane == 0 && clamped_rows) atomicAdd(not_pd, clamped_rows);
}

// One thread per point for k <= 16 (K = padded row length): the neighbour row
// arrives as int4 loads, the k + 1 coordinates as float4 gathers, and the
// whole factor stays in registers (point_factor_thread).  Same values as the
// group kernel, bit for bit.
template <int K, int KT>
__global__ void __launch_bounds__(128) point_factor_thread_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int64_t n0,
    KernF kf, float* __restrict__ b_out, float* __restrict__ sigma_out,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd, RescueList rl) {
  extern __shared__ __align__(16) unsigned char tstage[];
  const ThreadStage<K> st(tstage);
  double* W = reinterpret_cast<double*>(tstage + ThreadStage<K>::kBytes) +
              (threadIdx.x >> 5) * (warp_rescue_bytes<K>() / sizeof(double));
  LogAcc acc;
  unsigned long long clamped_rows = 0;
  const int64_t npts = N - n0;
  const int64_t total = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (npts + total - 1) / total;  // the same on every lane
  for (int64_t it = 0; it < iters; it++) {
    const int64_t t = it * total + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = t < npts;
    const int64_t i = n0 + (valid ? t : 0);
    const int32_t* row = nbr + (valid ? t : 0) * K;
    PointRegs<K> p;
    const float4 xq = __ldg(xs + i);
    bool deferred = false, rescue = false;
    if (valid) {
      stage_coords<K>(st, xs, row, k);
      point_factor_thread<K, KT>(p, k, kf, st, xq);
      if (needs_rescue(p, k, kf)) {
        deferred = rl.defer(i);
        rescue = !deferred;
      }
    }
    warp_rescue<K, KT>(p, rescue, xs, row, k, xq, kf, W);  // list full: in place
    if (!valid || deferred) continue;
    float4* bo = reinterpret_cast<float4*>(b_out + t * K);
#pragma unroll
    for (int q = 0; q < K / 4; q++)
      bo[q] = make_float4(p.y[4 * q], p.y[4 * q + 1], p.y[4 * q + 2], p.y[4 * q + 3]);
    sigma_out[i] = p.sigma;
    acc.mul(p.sigma);
    if (p.clamped) clamped_rows++;
  }
  block_add_double(acc.log_value(), logdet);
  for (int o = 16; o; o >>= 1) clamped_rows += __shfl_xor_sync(0xffffffffu, clamped_rows, o);
  if ((threadIdx.x & 31) == 0 && clamped_rows) atomicAdd(not_pd, clamped_rows);
}

// 32 < k <= 64: one warp per point with the factor in shared memory
// (pointwide.cuh).  Rows that need the FP64 rescue are recomputed by lane 0.
template <int KT>
__global__ void __launch_bounds__(128) point_factor_wide_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int kp,
    int64_t n0, KernF kf, float* __restrict__ b_out, float* __restrict__ sigma_out,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd, RescueList rl) {
  extern __shared__ __align__(16) unsigned char wide_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WideWarp& W = reinterpret_cast<WideWarp*>(wide_smem)[warp];
  LogAcc acc;
  unsigned long long clamped_rows = 0;
  const int64_t npts = N - n0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; t < npts; t += nw) {
    const int64_t i = n0 + t;
    const int32_t* row = nbr + t * kp;
    for (int a = lane; a < k; a += 32) W.x[a] = __ldg(xs + row[a]);
    __syncwarp();
    const float4 xq = __ldg(xs + i);
    WideFactor r = point_factor_wide<KT>(W, k, kf, xq);
    if (wide_needs_rescue(W, r, k, kf)) {
      bool deferred = false;
      if (lane == 0) deferred = rl.defer(i);
      if (__shfl_sync(0xffffffffu, deferred, 0)) continue;
      if (lane == 0) {
        Row64<kWideK> R;
        row_factor64<kWideK, KT>(R, xs, row, k, xq, kf);
        for (int e = 0; e < kp; e++) b_out[t * kp + e] = e < k ? (float)R.b[e] : 0.0f;
        const float sg = (float)R.sigma;
        sigma_out[i] = sg;
        acc.mul(sg);
        if (R.clamped) clamped_rows++;
      }
    } else {
      for (int a = lane; a < kp; a += 32) b_out[t * kp + a] = a < k ? W.y[a] : 0.0f;
      if (lane == 0) {
        sigma_out[i] = r.sigma;
        acc.mul(r.sigma);
        if (r.clamped) clamped_rows++;
      }
    }
    __syncwarp();
  }
  double lv = (lane == 0) ? acc.log_value() : 0.0;
  block_add_double(lv, logdet);
  for (int o = 16; o; o >>= 1) clamped_rows += __shfl_xor_sync(0xffffffffu, clamped_rows, o);
  if (lane == 0 && clamped_rows) atomicAdd(not_pd, clamped_rows);
}

// The FP64 rows listed by the factor kernels: b (row stride kp), sigma, and
// their log-determinant and floor counts.
// k <= 32: one warp per listed row (warp_row_factor64, the routine of every
// other rescue of these k).
template <int KMAX, int KT>
__global__ void __launch_bounds__(128) factor_rescue_warp_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int kp, int64_t n0,
    KernF kf, RescueList rl, float* __restrict__ b_out, float* __restrict__ sigma_out,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd) {
  __shared__ double Wsm[4][KMAX * (KMAX + 1)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  LogAcc acc;
  unsigned long long clamped_rows = 0;
  const unsigned long long cnt = *rl.count;
  const int64_t n = (int64_t)(cnt < rl.cap ? cnt : rl.cap);
  for (int64_t r = blockIdx.x * 4 + warp; r < n; r += (int64_t)gridDim.x * 4) {
    const int64_t i = rl.rows[r];
    const int64_t t = i - n0;
    const WarpRow64 w = warp_row_factor64<KMAX, KT>(xs, nbr + t * kp, k, __ldg(xs + i), kf,
                                                    Wsm[warp]);
    if (lane < kp) b_out[t * kp + lane] = lane < k ? (float)w.b : 0.0f;
    if (lane == 0) {
      const float sg = (float)w.sigma;
      sigma_out[i] = sg;
      acc.mul(sg);
      if (w.clamped) clamped_rows++;
    }
  }
  block_add_double(lane == 0 ? acc.log_value() : 0.0, logdet);
  for (int o = 16; o; o >>= 1) clamped_rows += __shfl_xor_sync(0xffffffffu, clamped_rows, o);
  if (lane == 0 && clamped_rows) atomicAdd(not_pd, clamped_rows);
}

// k > 32: one thread per listed row.
template <int KMAX, int KT>
__global__ void __launch_bounds__(128) factor_rescue_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int kp, int64_t n0,
    KernF kf, RescueList rl, float* __restrict__ b_out, float* __restrict__ sigma_out,
    double* __restrict__ logdet, unsigned long long* __restrict__ not_pd) {
  LogAcc acc;
  unsigned long long clamped_rows = 0;
  const unsigned long long cnt = *rl.count;
  const int64_t n = (int64_t)(cnt < rl.cap ? cnt : rl.cap);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rl.rows[r];
    const int64_t t = i - n0;
    Row64<KMAX> R;
    row_factor64<KMAX, KT>(R, xs, nbr + t * kp, k, __ldg(xs + i), kf);
    for (int e = 0; e < kp; e++) b_out[t * kp + e] = e < k ? (float)R.b[e] : 0.0f;
    const float sg = (float)R.sigma;
    sigma_out[i] = sg;
    acc.mul(sg);
    if (R.clamped) clamped_rows++;
  }
  block_add_double(acc.log_value(), logdet);
  for (int o = 16; o; o >>= 1) clamped_rows += __shfl_xor_sync(0xffffffffu, clamped_rows, o);
  if ((threadIdx.x & 31) == 0 && clamped_rows) atomicAdd(not_pd, clamped_rows);
}

template <int KMAX>
int launch_rescue(int type, graphgp_graph_t g, graphgp_factor_t f, const KernF& kf,
                  const RescueList& rl, const RowView& rv, cudaStream_t s) {
  const unsigned grid = 4 * (unsigned)num_sms();
#define GGP_RS(KT)                                                                          \
  if constexpr (KMAX <= 32) {                                                               \
    factor_rescue_warp_kernel<KMAX, KT><<<grid, 128, 0, s>>>(                               \
        g->xs, rv.nbr, g->k, g->kp, rv.n0, kf, rl, rv.b, f->sigma, f->logdet, f->not_pd);   \
  } else {                                                                                  \
    factor_rescue_kernel<KMAX, KT><<<grid, 128, 0, s>>>(                                    \
        g->xs, rv.nbr, g->k, g->kp, rv.n0, kf, rl, rv.b, f->sigma, f->logdet, f->not_pd);   \
  }
  switch (type) {
    case GRAPHGP_MATERN12: GGP_RS(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_RS(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_RS(GRAPHGP_MATERN52); break;
    default: GGP_RS(GRAPHGP_SQEXP); break;
  }
#undef GGP_RS
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

// What the FP32 dense factor leaves for dense_finish_kernel.
struct DenseCheck {
  double logdet;           // sum log L0_ii^2 of the FP32 block
  unsigned long long bad;  // floored pivots
  float min_piv;           // smallest pivot before flooring
};

// Dense block: K_00 (lower triangle) in global memory.
template <int KT>
__global__ void dense_fill_kernel(const float4* __restrict__ xs, int n0, KernF kf,
                                  float* __restrict__ A) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n0 * n0;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n0), j = (int)(e % n0);
    float v = 0.0f;
    if (j < i) v = kappa_d2<KT>(kf, sqdist(xs[i], xs[j]));
    else if (j == i) v = kf.s2 + kf.nug;
    A[e] = v;
  }
}

// One block, left-looking Cholesky by columns on the n0 x n0 matrix in
// global memory (L2-resident), with the pivot floor; then L0^-1 column by
// column; sigma_i = L0_ii; adds sum log L0_ii^2 to logdet.
__global__ void __launch_bounds__(1024) dense_chol_kernel(float* __restrict__ A,
                                                          float* __restrict__ W, int n0,
                                                          float* __restrict__ sigma,
                                                          DenseCheck* __restrict__ chk) {
  extern __shared__ float rowj[];  // [n0]
  __shared__ float s_inv;
  __shared__ unsigned long long s_bad;
  __shared__ float s_minpiv;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_minpiv = A[0];
  }
  const float k0 = A[0];
  for (int j = 0; j < n0; j++) {
    for (int m = threadIdx.x; m < j; m += blockDim.x) rowj[m] = A[(int64_t)j * n0 + m];
    __syncthreads();
    for (int r = j + threadIdx.x; r < n0; r += blockDim.x) {
      const float* ar = A + (int64_t)r * n0;
      float t0 = ar[j], t1 = 0.0f;
      int m = 0;
      for (; m + 1 < j; m += 2) {
        t0 = fmaf(-ar[m], rowj[m], t0);
        t1 = fmaf(-ar[m + 1], rowj[m + 1], t1);
      }
      if (m < j) t0 = fmaf(-ar[m], rowj[m], t0);
      float tv = t0 + t1;
      if (r == j) {
        float fl = kPdFloor * k0;
        s_minpiv = fminf(s_minpiv, tv);
        if (!(tv > fl)) {
          tv = fl;
          s_bad++;
        }
        float l = sqrtf(tv);
        A[(int64_t)j * n0 + j] = l;
        s_inv = 1.0f / l;
      } else {
        rowj[n0 - 1 - (r - j - 1)] = tv;  // park in the unused tail of rowj
      }
    }
    __syncthreads();
    float inv = s_inv;
    for (int r = j + 1 + threadIdx.x; r < n0; r += blockDim.x)
      A[(int64_t)r * n0 + j] = rowj[n0 - 1 - (r - j - 1)] * inv;
    __syncthreads();
  }
  // inverse: column c solves L w = e_c
  for (int c = threadIdx.x; c < n0; c += blockDim.x) {
    for (int i = 0; i < c; i++) W[(int64_t)i * n0 + c] = 0.0f;
    W[(int64_t)c * n0 + c] = 1.0f / A[(int64_t)c * n0 + c];
    for (int i = c + 1; i < n0; i++) {
      const float* ar = A + (int64_t)i * n0;
      float t = 0.0f;
      for (int m = c; m < i; m++) t = fmaf(ar[m], W[(int64_t)m * n0 + c], t);
      W[(int64_t)i * n0 + c] = -t / ar[i];
    }
  }
  __syncthreads();
  double lsum = 0.0;
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    float l = A[(int64_t)i * n0 + i];
    sigma[i] = l;
    lsum += log((double)l * (double)l);
  }
  block_add_double(lsum, &chk->logdet);
  if (threadIdx.x == 0) {
    chk->bad = s_bad;
    chk->min_piv = s_minpiv;
  }
}

// Dense block with the lower triangle held in shared memory (n0 <= 320): one
// block of 1024 threads, four threads per row for every dot product.
//   Cholesky, left-looking by columns: t_r = A_rj - sum_{m<j} L_rm L_jm for
//   r >= j, pivot t_j (floored at 1e-7 K_00 and counted), L_rj = t_r / L_jj.
//   Inverse in place, last column first: with the trailing block already
//   inverted (W2), column j of W = L^-1 is W_jj = 1 / L_jj and
//   W_rj = -W_jj sum_{j<m<=r} W2_rm L_mj for r > j.
// Outputs as dense_chol_kernel: L0 and L0^-1 row-major with zero upper part,
// sigma_i = L0_ii, logdet += sum log L0_ii^2 (FP64), not-PD count.
constexpr int kDenseSmemMax = 320;
__device__ __forceinline__ int tri_ix(int r, int c) { return r * (r + 1) / 2 + c; }

__global__ void __launch_bounds__(1024) dense_chol_smem_kernel(float* __restrict__ A,
                                                               float* __restrict__ W, int n0,
                                                               float* __restrict__ sigma,
                                                               DenseCheck* __restrict__ chk) {
  extern __shared__ float S[];         // [tri(n0)] packed lower triangle
  float* tr = S + n0 * (n0 + 1) / 2;   // [n0] column values of one step
  __shared__ unsigned long long s_bad;
  __shared__ float s_minpiv;
  const int w = threadIdx.x >> 2, part = threadIdx.x & 3;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_minpiv = A[0];
  }
  for (int e = threadIdx.x; e < n0 * n0; e += blockDim.x) {
    const int r = e / n0, c = e - r * n0;
    if (c <= r) S[tri_ix(r, c)] = A[e];
  }
  __syncthreads();
  const float fl = kPdFloor * S[0];
  for (int j = 0; j < n0; j++) {
    const float* Lj = S + tri_ix(j, 0);
    for (int r0 = 0; r0 < n0; r0 += 256) {
      const int r = r0 + w;
      float acc = 0.0f;
      if (r >= j && r < n0) {
        const float* Lr = S + tri_ix(r, 0);
        for (int m = part; m < j; m += 4) acc = fmaf(Lr[m], Lj[m], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (part == 0 && r >= j && r < n0) tr[r] = S[tri_ix(r, j)] - acc;
    }
    __syncthreads();
    float piv = tr[j];
    const bool bad = !(piv > fl);
    if (bad) piv = fl;
    const float ljj = sqrtf(piv);
    const float inv = 1.0f / ljj;
    for (int r = j + 1 + threadIdx.x; r < n0; r += blockDim.x) S[tri_ix(r, j)] = tr[r] * inv;
    if (threadIdx.x == 0) {
      S[tri_ix(j, j)] = ljj;
      s_minpiv = fminf(s_minpiv, tr[j]);
      if (bad) s_bad++;
    }
    __syncthreads();
  }
  double lsum = 0.0;
  for (int e = threadIdx.x; e < n0 * n0; e += blockDim.x) {
    const int r = e / n0, c = e - r * n0;
    A[e] = c <= r ? S[tri_ix(r, c)] : 0.0f;
  }
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    const float l = S[tri_ix(i, i)];
    sigma[i] = l;
    lsum += log((double)l * (double)l);
  }
  __syncthreads();
  for (int j = n0 - 1; j >= 0; j--) {
    const float d = 1.0f / S[tri_ix(j, j)];
    for (int r0 = 0; r0 < n0; r0 += 256) {
      const int r = r0 + w;
      float acc = 0.0f;
      if (r > j && r < n0) {
        const float* Wr = S + tri_ix(r, 0);
        for (int m = j + 1 + part; m <= r; m += 4) acc = fmaf(Wr[m], S[tri_ix(m, j)], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (part == 0 && r > j && r < n0) tr[r] = -d * acc;
    }
    __syncthreads();
    for (int r = j + 1 + threadIdx.x; r < n0; r += blockDim.x) S[tri_ix(r, j)] = tr[r];
    if (threadIdx.x == 0) S[tri_ix(j, j)] = d;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n0 * n0; e += blockDim.x) {
    const int r = e / n0, c = e - r * n0;
    W[e] = c <= r ? S[tri_ix(r, c)] : 0.0f;
  }
  block_add_double(lsum, &chk->logdet);
  if (threadIdx.x == 0) {
    chk->bad = s_bad;
    chk->min_piv = s_minpiv;
  }
}

// Accepts the FP32 dense block or recomputes it in FP64.  The FP32 block's
// error is estimated like a conditional's (rescue.cuh): every dense row is a
// conditional on all earlier dense points, with K_jj = K_00 for every j, so
// est = 2^-24 (K_00 / p_min)^2 from the smallest FP32 pivot p_min.  When the
// estimate exceeds the kernel's rescue_tol or a pivot was floored, the block
// is refactored from the coordinates in FP64 (K_00 from FP64 distances,
// left-looking Cholesky with the same floor, inverse by forward substitution)
// and rounded to FP32; else the FP32 block's log-determinant and floor count
// are taken.  One block of 1024 threads; Lw, Ww are n0 x n0 FP64 work arrays.
template <int KT>
__global__ void __launch_bounds__(1024) dense_finish_kernel(
    const float4* __restrict__ xs, int n0, KernF kf, const DenseCheck* __restrict__ chk,
    double* __restrict__ Lw, double* __restrict__ Ww, float* __restrict__ L0,
    float* __restrict__ L0inv, float* __restrict__ sigma, double* __restrict__ logdet,
    unsigned long long* __restrict__ not_pd) {
  extern __shared__ double tcol[];  // [n0]
  __shared__ unsigned long long s_bad;
  const float k0f = kf.s2 + kf.nug;
  const float r32 = k0f / chk->min_piv;
  const bool redo = chk->bad > 0 || !(r32 * r32 <= kf.resc_T);
  if (!redo) {
    if (threadIdx.x == 0) {
      atomicAdd(logdet, chk->logdet);
      if (chk->bad) atomicAdd(not_pd, chk->bad);
    }
    return;
  }
  if (threadIdx.x == 0) s_bad = 0;
  const double k0 = kf.s2d + kf.nugd;
  for (int64_t e = threadIdx.x; e < (int64_t)n0 * n0; e += blockDim.x) {
    const int i = (int)(e / n0), j = (int)(e % n0);
    Lw[e] = j < i ? kappa64<KT>(kf, dist64(xs[i], xs[j])) : (j == i ? k0 : 0.0);
  }
  __syncthreads();
  const double fl = kPdFloor64 * k0;
  for (int j = 0; j < n0; j++) {
    const double* Lj = Lw + (int64_t)j * n0;
    for (int r = j + threadIdx.x; r < n0; r += blockDim.x) {
      const double* Lr = Lw + (int64_t)r * n0;
      double t = Lr[j];
      for (int m = 0; m < j; m++) t -= Lr[m] * Lj[m];
      tcol[r] = t;
    }
    __syncthreads();
    double piv = tcol[j];
    if (!(piv > fl)) piv = fl;
    const double ljj = sqrt(piv);
    for (int r = j + 1 + threadIdx.x; r < n0; r += blockDim.x) Lw[(int64_t)r * n0 + j] = tcol[r] / ljj;
    if (threadIdx.x == 0) {
      Lw[(int64_t)j * n0 + j] = ljj;
      if (!(tcol[j] > fl)) s_bad++;
    }
    __syncthreads();
  }
  // L^-1 column by column (forward substitution), one column per thread
  for (int c = threadIdx.x; c < n0; c += blockDim.x) {
    Ww[(int64_t)c * n0 + c] = 1.0 / Lw[(int64_t)c * n0 + c];
    for (int i = c + 1; i < n0; i++) {
      const double* Li = Lw + (int64_t)i * n0;
      double t = 0.0;
      for (int m = c; m < i; m++) t += Li[m] * Ww[(int64_t)m * n0 + c];
      Ww[(int64_t)i * n0 + c] = -t / Li[i];
    }
  }
  __syncthreads();
  double lsum = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)n0 * n0; e += blockDim.x) {
    const int i = (int)(e / n0), j = (int)(e % n0);
    L0[e] = j <= i ? (float)Lw[e] : 0.0f;
    L0inv[e] = j <= i ? (float)Ww[e] : 0.0f;
    if (i == j) {
      const float l = (float)Lw[e];
      sigma[i] = l;
      lsum += log((double)l * (double)l);
    }
  }
  block_add_double(lsum, logdet);
  if (threadIdx.x == 0 && s_bad) atomicAdd(not_pd, s_bad);
}

template <int G>
int launch_point(int type, graphgp_graph_t g, graphgp_factor_t f, const KernF& kf,
                 const RescueList& rl, const RowView& rv, cudaStream_t s) {
  int64_t npts = rv.N - rv.n0;
  constexpr int PPW = 32 / G;
  int64_t groups_per_block = 4 * PPW;
  unsigned grid = grid_for((npts + groups_per_block - 1) / groups_per_block * 128, 128, 16);
  constexpr size_t smem = 4 * (size_t)G * (G + 1) * sizeof(double);
#define GGP_PF(KT)                                                                       \
  GGP_CUDA(cudaFuncSetAttribute(point_factor_kernel<G, KT>,                              \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
  point_factor_kernel<G, KT><<<grid, 128, smem, s>>>(g->xs, rv.nbr, rv.N, g->k, g->kp,     \
                                                     rv.n0, kf, rv.b, f->sigma, f->logdet, \
                                                     f->not_pd, rl)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_PF(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_PF(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_PF(GRAPHGP_MATERN52); break;
    default: GGP_PF(GRAPHGP_SQEXP); break;
  }
#undef GGP_PF
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

template <int K>
int launch_point_thread(int type, graphgp_graph_t g, graphgp_factor_t f, const KernF& kf,
                        const RescueList& rl, const RowView& rv, cudaStream_t s) {
  const int64_t npts = rv.N - rv.n0;
  const unsigned grid = grid_for(npts, kThreadBlock, 8);
  constexpr size_t smem = ThreadStage<K>::kBytes + 4 * warp_rescue_bytes<K>();
#define GGP_PT(KT)                                                                            \
  GGP_CUDA(allow_dyn_smem(point_factor_thread_kernel<K, KT>, smem));                          \
  point_factor_thread_kernel<K, KT><<<grid, kThreadBlock, smem, s>>>(                         \
      g->xs, rv.nbr, rv.N, g->k, rv.n0, kf, rv.b, f->sigma, f->logdet, f->not_pd, rl)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_PT(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_PT(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_PT(GRAPHGP_MATERN52); break;
    default: GGP_PT(GRAPHGP_SQEXP); break;
  }
#undef GGP_PT
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

constexpr int kWideWarps = 4;  // warps per block of the wide kernels
constexpr int64_t kRescueListMax = 1 << 20;  // rows listed for the FP64 rescue kernel

int launch_point_wide(int type, graphgp_graph_t g, graphgp_factor_t f, const KernF& kf,
                      const RescueList& rl, const RowView& rv, cudaStream_t s) {
  const int64_t npts = rv.N - rv.n0;
  const size_t smem = kWideWarps * sizeof(WideWarp);
  const unsigned grid = grid_for((npts + kWideWarps - 1) / kWideWarps * 128, 128, 4);
#define GGP_PW(KT)                                                                           \
  GGP_CUDA(cudaFuncSetAttribute(point_factor_wide_kernel<KT>,                                \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));    \
  point_factor_wide_kernel<KT><<<grid, 32 * kWideWarps, smem, s>>>(                          \
      g->xs, rv.nbr, rv.N, g->k, g->kp, rv.n0, kf, rv.b, f->sigma, f->logdet, f->not_pd, rl)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_PW(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_PW(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_PW(GRAPHGP_MATERN52); break;
    default: GGP_PW(GRAPHGP_SQEXP); break;
  }
#undef GGP_PW
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace

int point_factor_rows(graphgp_graph_t g, graphgp_factor_t f, const KernF& kf, int type,
                      int64_t t0, int64_t t1, cudaStream_t s) {
  if (t1 <= t0) return GRAPHGP_OK;
  const int64_t npts = t1 - t0;
  const RowView rv{g->nbr + t0 * g->kp, f->b + t0 * g->kp, g->n0 + t1, g->n0 + t0};
  Scratch sc(s);
  RescueList rl;
  rl.cap = (unsigned long long)std::min<int64_t>(npts, kRescueListMax);
  GGP_TRY(sc.alloc(&rl.rows, rl.cap));
  GGP_TRY(sc.alloc(&rl.count, 1));
  GGP_CUDA(cudaMemsetAsync(rl.count, 0, sizeof(unsigned long long), s));
  switch (g->kp) {
    case 4: GGP_TRY(launch_point_thread<4>(type, g, f, kf, rl, rv, s)); return launch_rescue<4>(type, g, f, kf, rl, rv, s);
    case 8: GGP_TRY(launch_point_thread<8>(type, g, f, kf, rl, rv, s)); return launch_rescue<8>(type, g, f, kf, rl, rv, s);
    case 12: GGP_TRY(launch_point_thread<12>(type, g, f, kf, rl, rv, s)); return launch_rescue<12>(type, g, f, kf, rl, rv, s);
    case 16: GGP_TRY(launch_point_thread<16>(type, g, f, kf, rl, rv, s)); return launch_rescue<16>(type, g, f, kf, rl, rv, s);
    case 20:
    case 24:
    case 28:
    case 32: GGP_TRY(launch_point<32>(type, g, f, kf, rl, rv, s)); return launch_rescue<32>(type, g, f, kf, rl, rv, s);
    default: GGP_TRY(launch_point_wide(type, g, f, kf, rl, rv, s)); return launch_rescue<kWideK>(type, g, f, kf, rl, rv, s);
  }
}

int point_factor(graphgp_graph_t g, graphgp_factor_t f, const KernF& kf, int type,
                 cudaStream_t s) {
  return point_factor_rows(g, f, kf, type, 0, g->N - g->n0, s);
}

int dense_factor(graphgp_graph_t g, graphgp_factor_t f, const KernF& kf, int type,
                 cudaStream_t s) {
  int n0 = g->n0;
  unsigned grid = grid_for((int64_t)n0 * n0, 256);
  switch (type) {
    case GRAPHGP_MATERN12: dense_fill_kernel<GRAPHGP_MATERN12><<<grid, 256, 0, s>>>(g->xs, n0, kf, f->L0); break;
    case GRAPHGP_MATERN32: dense_fill_kernel<GRAPHGP_MATERN32><<<grid, 256, 0, s>>>(g->xs, n0, kf, f->L0); break;
    case GRAPHGP_MATERN52: dense_fill_kernel<GRAPHGP_MATERN52><<<grid, 256, 0, s>>>(g->xs, n0, kf, f->L0); break;
    default: dense_fill_kernel<GRAPHGP_SQEXP><<<grid, 256, 0, s>>>(g->xs, n0, kf, f->L0); break;
  }
  GGP_CUDA(cudaGetLastError());
  Scratch sc(s);
  DenseCheck* chk = nullptr;
  double* work = nullptr;
  GGP_TRY(sc.alloc(&chk, 1));
  GGP_TRY(sc.alloc(&work, 2 * (size_t)n0 * n0));
  GGP_CUDA(cudaMemsetAsync(chk, 0, sizeof(DenseCheck), s));
  if (n0 <= kDenseSmemMax) {
    const size_t smem = ((size_t)n0 * (n0 + 1) / 2 + n0) * sizeof(float);
    GGP_CUDA(cudaFuncSetAttribute(dense_chol_smem_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dense_chol_smem_kernel<<<1, 1024, smem, s>>>(f->L0, f->L0inv, n0, f->sigma, chk);
  } else {
    dense_chol_kernel<<<1, 1024, n0 * sizeof(float), s>>>(f->L0, f->L0inv, n0, f->sigma, chk);
  }
  GGP_CUDA(cudaGetLastError());
  double* Lw = work;
  double* Ww = work + (size_t)n0 * n0;
  const size_t smem64 = (size_t)n0 * sizeof(double);
#define GGP_DF(KT)                                                                             \
  dense_finish_kernel<KT><<<1, 1024, smem64, s>>>(g->xs, n0, kf, chk, Lw, Ww, f->L0, f->L0inv, \
                                                  f->sigma, f->logdet, f->not_pd)
  switch (type) {
    case GRAPHGP_MATERN12: GGP_DF(GRAPHGP_MATERN12); break;
    case GRAPHGP_MATERN32: GGP_DF(GRAPHGP_MATERN32); break;
    case GRAPHGP_MATERN52: GGP_DF(GRAPHGP_MATERN52); break;
    default: GGP_DF(GRAPHGP_SQEXP); break;
  }
#undef GGP_DF
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace ggp

using namespace ggp;

static int factor_impl(graphgp_graph_t g, const graphgp_kernel* kern, int64_t p0, int64_t p1,
                       bool rows, void* stream, graphgp_factor_t* out) {
  if (!out) return GRAPHGP_ERR_INVALID;
  *out = nullptr;
  if (!g || !kern || kern->type < 0 || kern->type > 3 || !(kern->sigma2 > 0) ||
      !(kern->lengthscale > 0) || !(kern->nugget >= 0) || !std::isfinite(kern->rescue_tol))
    return GRAPHGP_ERR_INVALID;
  if (p0 < 0 || p1 > g->N || p0 > p1 || (p0 > 0 && p0 < g->n0) || (p0 == 0 && p1 < g->n0))
    return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  graphgp_factor_t f = new (std::nothrow) graphgp_factor_s();
  if (!f) return GRAPHGP_ERR_OOM;
  f->g = g;
  f->kern = *kern;
  if (rows) {
    f->row_begin = p0;
    f->row_end = p1;
  }
  auto fail = [&](int rc) {
    f->mem.free_all();
    delete f;
    return rc;
  };
  int rc = [&]() -> int {
    GGP_TRY(f->mem.alloc(&f->b, (g->N - g->n0) * g->kp));
    GGP_TRY(f->mem.alloc(&f->sigma, g->N));
    GGP_TRY(f->mem.alloc(&f->L0, (int64_t)g->n0 * g->n0));
    GGP_TRY(f->mem.alloc(&f->L0inv, (int64_t)g->n0 * g->n0));
    GGP_TRY(f->mem.alloc(&f->logdet, 1));
    GGP_TRY(f->mem.alloc(&f->not_pd, 1));
    GGP_CUDA(cudaMemsetAsync(f->logdet, 0, 8, s));
    GGP_CUDA(cudaMemsetAsync(f->not_pd, 0, 8, s));
    KernF kf = make_kernf(*kern);
    if (rows) {  // rows outside the range stay zero
      GGP_CUDA(cudaMemsetAsync(f->b, 0, (g->N - g->n0) * g->kp * sizeof(float), s));
      GGP_CUDA(cudaMemsetAsync(f->sigma, 0, g->N * sizeof(float), s));
      GGP_CUDA(cudaMemsetAsync(f->L0, 0, (int64_t)g->n0 * g->n0 * sizeof(float), s));
      GGP_CUDA(cudaMemsetAsync(f->L0inv, 0, (int64_t)g->n0 * g->n0 * sizeof(float), s));
    }
    if (p0 == 0) GGP_TRY(dense_factor(g, f, kf, kern->type, s));
    const int64_t t0 = std::max<int64_t>(p0, g->n0) - g->n0, t1 = std::max<int64_t>(p1 - g->n0, 0);
    GGP_TRY(point_factor_rows(g, f, kf, kern->type, t0, t1, s));
    return GRAPHGP_OK;
  }();
  if (rc < 0) return fail(rc);
  *out = f;
  return GRAPHGP_OK;
}

extern "C" int graphgp_factor(graphgp_graph_t g, const graphgp_kernel* kern, void* stream,
                              graphgp_factor_t* out) {
  if (!g) {
    if (out) *out = nullptr;
    return GRAPHGP_ERR_INVALID;
  }
  return factor_impl(g, kern, 0, g->N, false, stream, out);
}

extern "C" int graphgp_factor_rows(graphgp_graph_t g, const graphgp_kernel* kern,
                                   int64_t pos_begin, int64_t pos_end, void* stream,
                                   graphgp_factor_t* out) {
  if (!g) {
    if (out) *out = nullptr;
    return GRAPHGP_ERR_INVALID;
  }
  return factor_impl(g, kern, pos_begin, pos_end, true, stream, out);
}

extern "C" int graphgp_factor_export(graphgp_factor_t f, float* b_d, float* sigma_d, float* L0_d,
                                     void* stream) {
  if (!f) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  graphgp_graph_t g = f->g;
  if (b_d && g->N > g->n0)
    GGP_CUDA(cudaMemcpy2DAsync(b_d, g->k * 4, f->b, g->kp * 4, g->k * 4, g->N - g->n0,
                               cudaMemcpyDeviceToDevice, s));
  if (sigma_d)
    GGP_CUDA(cudaMemcpyAsync(sigma_d, f->sigma, g->N * 4, cudaMemcpyDeviceToDevice, s));
  if (L0_d)
    GGP_CUDA(cudaMemcpyAsync(L0_d, f->L0, (int64_t)g->n0 * g->n0 * 4, cudaMemcpyDeviceToDevice, s));
  return GRAPHGP_OK;
}

extern "C" void graphgp_factor_destroy(graphgp_factor_t f) {
  if (!f) return;
  cudaDeviceSynchronize();
  f->mem.free_all();
  delete f;
}
