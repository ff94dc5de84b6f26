// Gradient of the negative log-likelihood with respect to the point
// coordinates, the graph (order, neighbour lists, depth levels) held fixed.
//
// The derivatives of Sec. 2.3 give, for every conditional i, the cotangents
// of its covariance entries (with s = sigma_i^2, g = K_cc^-1 bbar):
//   Kbar_cc[a][c] = -g_a b_c + sbar b_a b_c,  Kbar_ci[a] = g_a - 2 sbar b_a,
// and for the dense block Kbar_00 = L0^-T Phi(L0^T Lbar0) L0^-1.  A
// stationary entry K_ab = kappa(|x_a - x_b|) moves with both of its points:
// d K_ab / d x_a = h(r) (x_a - x_b) with h(r) = kappa'(r) / r, and the
// opposite for x_b.  So point p collects
//   sum over entries (p, q) of (Kbar_pq + Kbar_qp) h(r_pq) (x_p - x_q).
// Each sparse conditional is one warp (the factor recomputed in shared
// memory, pointwide.cuh, for every k <= 64); lane a adds the terms of
// neighbour a, and the warp adds those of the point itself.  Sums are FP64
// atomics in graph order, written out in input order at the end.
#include "pointwide.cuh"

namespace ggp {

int run_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
               cudaStream_t s);
int dense_kbar(graphgp_graph_t g, graphgp_factor_t f, const float* u0, const float* xi0,
               float sgn, float ldbar, float* Kbar, cudaStream_t s);

namespace {

// kappa'(r) / r from the squared distance; Matern-1/2 has no derivative at
// r = 0, where the direction vanishes and the value is taken as 0.
template <int KT>
__device__ __forceinline__ float kappa_h_d2(const KernF& p, float d2) {
  const float il = p.inv_ell;
  if (KT == GRAPHGP_SQEXP) return -p.s2 * il * il * expf(-0.5f * d2 * il * il);
  const float r = sqrtf(d2);
  if (KT == GRAPHGP_MATERN12) return r > 0.0f ? -p.s2 * il * expf(-r * il) / r : 0.0f;
  if (KT == GRAPHGP_MATERN32) return -3.0f * p.s2 * il * il * expf(-1.7320508075688772f * r * il);
  const float a = 2.2360679774997896f * r * il;
  return -(5.0f / 3.0f) * p.s2 * il * il * (1.0f + a) * expf(-a);
}

template <int KT>
__device__ __forceinline__ double kappa_h64(const KernF& p, double r) {
  const double s2 = p.s2d, l = p.elld;
  if (KT == GRAPHGP_SQEXP) return -s2 * exp(-0.5 * (r / l) * (r / l)) / (l * l);
  if (KT == GRAPHGP_MATERN12) return r > 0.0 ? -s2 * exp(-r / l) / (l * r) : 0.0;
  if (KT == GRAPHGP_MATERN32) return -3.0 * s2 * exp(-1.7320508075688772 * r / l) / (l * l);
  const double a = 2.2360679774997896 * r / l;
  return -5.0 * s2 * (1.0 + a) * exp(-a) / (3.0 * l * l);
}

__device__ __forceinline__ void add3(double* acc, int64_t p, double x, double y, double z) {
  atomicAdd(acc + 3 * p, x);
  atomicAdd(acc + 3 * p + 1, y);
  atomicAdd(acc + 3 * p + 2, z);
}

// Sparse conditionals: whiten cotangents of the NLL (xibar = nllbar xi,
// logdetbar = nllbar / 2), so bbar_a = alpha v_c(a) with alpha = -xibar_i /
// sigma_i and sigbar_i = alpha xi_i + nllbar / sigma_i.
template <int KT>
__global__ void __launch_bounds__(128) position_backward_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int64_t N, int k, int kp,
    int64_t n0, KernF kf, const float* __restrict__ v, const float* __restrict__ xi,
    float nllbar, double* __restrict__ acc, int64_t* __restrict__ rescue_rows,
    unsigned long long* __restrict__ rescue_count) {
  extern __shared__ __align__(16) unsigned char wide_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WideWarp& W = reinterpret_cast<WideWarp*>(wide_smem)[warp];
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
    const float xii = xi[i];
    const float alpha = -(nllbar * xii) / sigma;
    const float sbar = (alpha * xii + nllbar / sigma) / (2.0f * sigma);
    for (int a = lane; a < k; a += 32) W.g[a] = alpha * v[row[a]];
    __syncwarp();
    wide_chol_solve(W, k, r.inc);
    double qx = 0.0, qy = 0.0, qz = 0.0;  // terms of the point itself
    for (int a = lane; a < k; a += 32) {
      const float ga = W.g[a], ba = W.y[a];
      const float4 xa = W.x[a];
      float ax = 0.0f, ay = 0.0f, az = 0.0f;
      for (int c = 0; c < k; c++) {
        if (c == a) continue;
        const float bc = W.y[c], gc = W.g[c];
        const float4 xc = W.x[c];
        const float w = (-ga * bc + sbar * ba * bc) + (-gc * ba + sbar * bc * ba);
        const float hw = w * kappa_h_d2<KT>(kf, sqdist(xa, xc));
        ax = fmaf(hw, xa.x - xc.x, ax);
        ay = fmaf(hw, xa.y - xc.y, ay);
        az = fmaf(hw, xa.z - xc.z, az);
      }
      const float hq = (ga - 2.0f * sbar * ba) * kappa_h_d2<KT>(kf, sqdist(xa, xq));
      const float dx = xa.x - xq.x, dy = xa.y - xq.y, dz = xa.z - xq.z;
      ax = fmaf(hq, dx, ax);
      ay = fmaf(hq, dy, ay);
      az = fmaf(hq, dz, az);
      qx -= (double)(hq * dx);
      qy -= (double)(hq * dy);
      qz -= (double)(hq * dz);
      add3(acc, row[a], ax, ay, az);
    }
    for (int o = 16; o; o >>= 1) {
      qx += __shfl_xor_sync(0xffffffffu, qx, o);
      qy += __shfl_xor_sync(0xffffffffu, qy, o);
      qz += __shfl_xor_sync(0xffffffffu, qz, o);
    }
    if (lane == 0) add3(acc, i, qx, qy, qz);
    __syncwarp();
  }
}

// Conditionals the warp kernel handed over, in FP64 (rescue.cuh), one
// thread per row.
template <int KT>
__global__ void __launch_bounds__(128) position_backward_rescue_kernel(
    const float4* __restrict__ xs, const int32_t* __restrict__ nbr, int k, int kp, int64_t n0,
    KernF kf, const float* __restrict__ v, const float* __restrict__ xi, float nllbar,
    double* __restrict__ acc, const int64_t* __restrict__ rows,
    const unsigned long long* __restrict__ count) {
  const int64_t n = (int64_t)*count;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rows[r];
    const int32_t* row = nbr + (i - n0) * kp;
    const float4 xq = xs[i];
    Row64<kWideK> R;
    row_factor64<kWideK, KT>(R, xs, row, k, xq, kf);
    const double sigma = (double)(float)R.sigma;
    const double xii = xi[i];
    const double alpha = -((double)nllbar * xii) / sigma;
    const double sbar = (alpha * xii + (double)nllbar / sigma) / (2.0 * sigma);
    double g[kWideK];
    for (int a = 0; a < k; a++) g[a] = alpha * (double)v[row[a]];
    for (int a = 0; a < k; a++) {
      double s = g[a];
      for (int m = 0; m < a; m++) s -= R.L[tri64(a, m)] * g[m];
      g[a] = s / R.L[tri64(a, a)];
    }
    for (int a = k - 1; a >= 0; a--) {
      double s = g[a];
      for (int m = a + 1; m < k; m++) s -= R.L[tri64(m, a)] * g[m];
      g[a] = s / R.L[tri64(a, a)];
    }
    double qx = 0.0, qy = 0.0, qz = 0.0;
    for (int a = 0; a < k; a++) {
      const float4 xa = xs[row[a]];
      double ax = 0.0, ay = 0.0, az = 0.0;
      for (int c = 0; c < k; c++) {
        if (c == a) continue;
        const float4 xc = xs[row[c]];
        const double w = (-g[a] * R.b[c] + sbar * R.b[a] * R.b[c]) +
                         (-g[c] * R.b[a] + sbar * R.b[c] * R.b[a]);
        const double hw = w * kappa_h64<KT>(kf, dist64(xa, xc));
        ax += hw * ((double)xa.x - xc.x);
        ay += hw * ((double)xa.y - xc.y);
        az += hw * ((double)xa.z - xc.z);
      }
      const double hq = (g[a] - 2.0 * sbar * R.b[a]) * kappa_h64<KT>(kf, dist64(xa, xq));
      const double dx = (double)xa.x - xq.x, dy = (double)xa.y - xq.y, dz = (double)xa.z - xq.z;
      ax += hq * dx;
      ay += hq * dy;
      az += hq * dz;
      qx -= hq * dx;
      qy -= hq * dy;
      qz -= hq * dz;
      add3(acc, row[a], ax, ay, az);
    }
    add3(acc, i, qx, qy, qz);
  }
}

// Dense block: point p < n0 collects (Kbar_pq + Kbar_qp) h(r_pq) (x_p - x_q).
template <int KT>
__global__ void dense_position_kernel(const float* __restrict__ Kbar,
                                      const float4* __restrict__ xs, int n0, KernF kf,
                                      double* __restrict__ acc) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n0; p += gridDim.x * blockDim.x) {
    const float4 xp = xs[p];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int q = 0; q < n0; q++) {
      if (q == p) continue;
      const float4 xq = xs[q];
      const float w = Kbar[(int64_t)p * n0 + q] + Kbar[(int64_t)q * n0 + p];
      const float hw = w * kappa_h_d2<KT>(kf, sqdist(xp, xq));
      ax += (double)(hw * (xp.x - xq.x));
      ay += (double)(hw * (xp.y - xq.y));
      az += (double)(hw * (xp.z - xq.z));
    }
    add3(acc, p, ax, ay, az);
  }
}

// out[order[p]] = acc[p] (graph order -> input order), FP64 -> FP32.
__global__ void scatter_points_kernel(const double* __restrict__ acc,
                                      const int32_t* __restrict__ order, int64_t N,
                                      float* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = order[p];
    out[3 * q] = (float)acc[3 * p];
    out[3 * q + 1] = (float)acc[3 * p + 1];
    out[3 * q + 2] = (float)acc[3 * p + 2];
  }
}

// u_0 = L0^-T xibar_0 (the dense block's share of the whiten adjoint).
__global__ void dense_u0_kernel(const float* __restrict__ L0inv, const float* __restrict__ xi,
                                float nllbar, int n0, float* __restrict__ u0) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n0; m += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = m; i < n0; i++) s = fmaf(L0inv[(int64_t)i * n0 + m], nllbar * xi[i], s);
    u0[m] = s;
  }
}

template <int KT>
int launch_positions(graphgp_graph_t g, graphgp_factor_t f, const float* v, const float* xi,
                     float nllbar, double* acc, cudaStream_t s) {
  const int n0 = g->n0;
  const int64_t npts = g->N - n0;
  const KernF kf = make_kernf(f->kern);
  Scratch sc(s);
  // dense block
  float *u0 = nullptr, *Kbar = nullptr;
  GGP_TRY(sc.alloc(&u0, n0));
  GGP_TRY(sc.alloc(&Kbar, (int64_t)n0 * n0));
  dense_u0_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(f->L0inv, xi, nllbar, n0, u0);
  GGP_CUDA(cudaGetLastError());
  GGP_TRY(dense_kbar(g, f, u0, xi, -1.0f, 0.5f * nllbar, Kbar, s));
  dense_position_kernel<KT><<<(n0 + 127) / 128, 128, 0, s>>>(Kbar, g->xs, n0, kf, acc);
  GGP_CUDA(cudaGetLastError());
  if (npts <= 0) return GRAPHGP_OK;
  // sparse conditionals, then the rows that need FP64
  int64_t* rows = nullptr;
  unsigned long long* cnt = nullptr;
  GGP_TRY(sc.alloc(&rows, npts));
  GGP_TRY(sc.alloc(&cnt, 1));
  GGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  constexpr int kWarps = 4;
  const size_t smem = kWarps * sizeof(WideWarp);
  GGP_CUDA(cudaFuncSetAttribute(position_backward_kernel<KT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = grid_for((npts + kWarps - 1) / kWarps * 128, 128, 4);
  position_backward_kernel<KT><<<grid, 32 * kWarps, smem, s>>>(
      g->xs, g->nbr, g->N, g->k, g->kp, n0, kf, v, xi, nllbar, acc, rows, cnt);
  GGP_CUDA(cudaGetLastError());
  position_backward_rescue_kernel<KT><<<(unsigned)num_sms() * 2, 128, 0, s>>>(
      g->xs, g->nbr, g->k, g->kp, n0, kf, v, xi, nllbar, acc, rows, cnt);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace
}  // namespace ggp

using namespace ggp;

extern "C" int graphgp_nll_backward_points(graphgp_graph_t g, graphgp_factor_t f,
                                           const float* v_d, double nllbar, float* pbar_d,
                                           void* stream) {
  if (!g || !f || f->g != g || f->row_end >= 0 || !v_d || !pbar_d) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* acc = nullptr;
  GGP_TRY(sc.alloc(&acc, 3 * g->N));
  GGP_CUDA(cudaMemsetAsync(acc, 0, 3 * g->N * sizeof(double), s));
  float* xi = g->tmp_vec2;  // the whitened field of v
  GGP_TRY(run_whiten(g, f, v_d, xi, nullptr, s));
  int rc = GRAPHGP_OK;
  switch (f->kern.type) {
    case GRAPHGP_MATERN12: rc = launch_positions<GRAPHGP_MATERN12>(g, f, v_d, xi, (float)nllbar, acc, s); break;
    case GRAPHGP_MATERN32: rc = launch_positions<GRAPHGP_MATERN32>(g, f, v_d, xi, (float)nllbar, acc, s); break;
    case GRAPHGP_MATERN52: rc = launch_positions<GRAPHGP_MATERN52>(g, f, v_d, xi, (float)nllbar, acc, s); break;
    default: rc = launch_positions<GRAPHGP_SQEXP>(g, f, v_d, xi, (float)nllbar, acc, s); break;
  }
  if (rc < 0) return rc;
  scatter_points_kernel<<<grid_for(g->N, 256), 256, 0, s>>>(acc, g->order, g->N, pbar_d);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}
