// Internal definitions shared by the CUDA translation units of libgraphgp.
// GraphGP: "GraphGP: Scalable Gaussian Processes with Vecchia's Approximation".
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "graphgp.h"
#include "variogram_poly.cuh"

namespace ggp {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
struct Status {
  int code = GRAPHGP_OK;
};

#define GGP_CUDA(call)                                                    \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      std::fprintf(stderr, "graphgp: %s failed: %s (%s:%d)\n", #call,     \
                   cudaGetErrorString(e_), __FILE__, __LINE__);           \
      return (e_ == cudaErrorMemoryAllocation) ? GRAPHGP_ERR_OOM          \
                                               : GRAPHGP_ERR_CUDA;        \
    }                                                                     \
  } while (0)

#define GGP_TRY(expr)           \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ < 0) return rc_;    \
  } while (0)

// bits of the device error word held by every graph
enum : uint32_t { ERRBIT_TIMEOUT = 1u, ERRBIT_INDEX = 2u };

// Device allocation that remembers its size (for graphgp_graph_info).
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <class T>
  int alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    size_t b = count * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e == cudaErrorMemoryAllocation ? GRAPHGP_ERR_OOM : GRAPHGP_ERR_CUDA;
    }
    ptrs.push_back((void*)*p);
    bytes += b;
    return GRAPHGP_OK;
  }
  void release(void* p, size_t b) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
        bytes -= b;
      }
  }
  void free_all() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

// Stream-ordered scratch that lives for one host call: allocated and freed
// on the call's stream, so it is released only after the work that uses it.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  int alloc(T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e == cudaErrorMemoryAllocation ? GRAPHGP_ERR_OOM : GRAPHGP_ERR_CUDA;
    }
    ptrs.push_back((void*)*p);
    return GRAPHGP_OK;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// Rows of the neighbour and weight matrices are padded to a multiple of four
// entries (sixteen for k > 32, which keeps the number of compiled sweep
// variants small) so that every row starts on a 16-byte boundary; padding
// entries point at position 0 with weight 0.
inline int row_stride(int k) { return k <= 32 ? (k + 3) & ~3 : (k + 15) & ~15; }

// Largest number of neighbours per point.
constexpr int kMaxK = 64;

// Spatial tile of the whiten sweep: this many consecutive k-d in-order ranks.
constexpr int64_t kTileR = 4096;

}  // namespace ggp

// The handle types named in graphgp.h.
struct graphgp_graph_s {
  int64_t N = 0;
  int k = 0, kp = 0, n0 = 0, num_levels = 0;
  int64_t max_spin = 0;
  ggp::DevArena mem;
  float* pts_in = nullptr;     // [N*3] input order, canonicalised
  float4* xs = nullptr;        // [N] coordinates in graph order (w unused)
  int32_t* order = nullptr;    // [N] position -> input index
  int32_t* nbr = nullptr;      // [(N-n0)*kp] positions, nearest first
  std::vector<int64_t> level_off_h;  // [num_levels+1]
  int64_t* level_off_d = nullptr;
  int64_t max_level_size = 0;     // largest depth level >= 1
  uint32_t* level_bar = nullptr;  // [num_levels] arrivals of the sweep barrier
  // spatial tiles of the whiten sweep: tile t holds the positions whose
  // spatial key (k-d in-order rank) lies in [t R, (t+1) R); inside every level
  // those positions are contiguous, starting at tile_start[t * num_levels + l]
  int64_t tile_R = 0, n_tiles = 0;
  int32_t* tile_start = nullptr;  // [(n_tiles + 1) * num_levels]
  uint32_t* err = nullptr;        // device error word
  // tree (graphs built here only)
  bool has_tree = false;
  int32_t* tree_point = nullptr;
  uint8_t* split_dim = nullptr;
  int32_t* inorder = nullptr;
  int32_t* depth_tree = nullptr;
  int32_t* nbr_tree = nullptr;   // [(N-n0)*k]
  float* tmp_vec = nullptr;      // [N] work vector for nll / adjoints
  float* tmp_vec2 = nullptr;     // [N]
};

struct graphgp_factor_s {
  graphgp_graph_t g = nullptr;
  graphgp_kernel kern{};
  ggp::DevArena mem;
  float* b = nullptr;        // [(N-n0)*kp]
  float* sigma = nullptr;    // [N]
  float* L0 = nullptr;       // [n0*n0] row-major lower
  float* L0inv = nullptr;    // [n0*n0] row-major lower
  double* logdet = nullptr;  // [1]
  unsigned long long* not_pd = nullptr;  // [1]
  // positions whose conditionals this handle holds: [row_begin, row_end);
  // row_end < 0 for a whole-graph factor (graphgp_factor)
  int64_t row_begin = 0, row_end = -1;
};

namespace ggp {

// ---------------------------------------------------------------------------
// FP32 covariance (Sec. 2.1): kappa from the squared distance.
// ---------------------------------------------------------------------------
struct KernF {
  float s2, inv_ell, nug;
  float resc_T;            // FP64 rescue threshold of the row-error estimate x 2^24, rescue.cuh
  double s2d, elld, nugd;  // the same parameters in FP64 (rescue path)
};

// Default per-row error estimate above which a conditional is recomputed in
// FP64 (rescue.cuh): 2^-7.  The estimate is conservative: on the measured
// workloads the element-wise sigma error stays below 1e-3 at this setting,
// and it sends 0.05 % of the headline cloud's rows, 0.3 % of a clustered
// cloud's and 8 % of the nugget-free large-dynamic-range cloud's to FP64.
constexpr double kDefaultRescueTol = 0.0078125;

template <int KT>
__device__ __forceinline__ float kappa_d2(const KernF& p, float d2) {
  if (KT == GRAPHGP_SQEXP) {
    return p.s2 * expf(-0.5f * d2 * p.inv_ell * p.inv_ell);
  } else {
    float r = sqrtf(d2);
    if (KT == GRAPHGP_MATERN12) {
      return p.s2 * expf(-r * p.inv_ell);
    } else if (KT == GRAPHGP_MATERN32) {
      float a = 1.7320508075688772f * r * p.inv_ell;
      return p.s2 * (1.0f + a) * expf(-a);
    } else {
      float a = 2.2360679774997896f * r * p.inv_ell;
      return p.s2 * (1.0f + a + a * a * (1.0f / 3.0f)) * expf(-a);
    }
  }
}

// Variogram gamma(r) = kappa(0) - kappa(r) (nugget excluded) from the squared
// distance, in FP32 with a small relative error all the way down to r -> 0,
// where kappa(r) is close to kappa(0) and 1 - kappa(r)/kappa(0) computed from
// kappa would keep none of its digits.  The increment form of the per-point
// factors (pointfactor.cuh) is built from these values.  Below a switch point
// gamma is a product of positive factors, one of them a short polynomial
// (variogram_poly.cuh) for a function without cancellation; above it the
// closed form, which there loses at most a small factor to cancellation:
//   SE (u = r^2 / 2l^2), Matern-1/2 (u = r/l), u < 1/2:
//       1 - e^-u = u psi(u),  psi(u) = (1 - e^-u) / u     (closed form: <= 2.6x)
//   Matern-3/2, a = sqrt3 r/l < 1:
//       1 - (1 + a) e^-a = a^2 phi(a) e^-a,  phi(a) = (e^a - 1 - a) / a^2
//                                                        (closed form: <= 2.8x)
//   Matern-5/2, a = sqrt5 r/l < 2:
//       1 - (1 + a + a^2/3) e^-a = a^2 phi(a) e^-a,
//       phi(a) = (e^a - 1 - a - a^2/3) / a^2              (closed form: <= 2.4x)
struct KG {
  float k, g;  // kappa(r), gamma(r)
};

// kappa and gamma from one exponential (the per-point factors pick one of
// the two per row).
template <int KT>
__device__ __forceinline__ KG kappa_gamma_d2(const KernF& p, float d2) {
  if (KT == GRAPHGP_SQEXP || KT == GRAPHGP_MATERN12) {
    const float u = KT == GRAPHGP_SQEXP ? 0.5f * d2 * p.inv_ell * p.inv_ell : sqrtf(d2) * p.inv_ell;
    const float e = expf(-u);
    return KG{p.s2 * e, p.s2 * (u < 0.5f ? u * poly_exp1(u) : 1.0f - e)};
  } else if (KT == GRAPHGP_MATERN32) {
    const float a = 1.7320508075688772f * sqrtf(d2) * p.inv_ell;
    const float e = expf(-a);
    const float pe = (1.0f + a) * e;
    return KG{p.s2 * pe, p.s2 * (a < 1.0f ? a * a * poly_m32(a) * e : 1.0f - pe)};
  } else {
    const float a = 2.2360679774997896f * sqrtf(d2) * p.inv_ell;
    const float e = expf(-a);
    const float pe = (1.0f + a + a * a * (1.0f / 3.0f)) * e;
    return KG{p.s2 * pe, p.s2 * (a < 2.0f ? a * a * poly_m52(a) * e : 1.0f - pe)};
  }
}

// gamma alone (the same values as kappa_gamma_d2's .g).
template <int KT>
__device__ __forceinline__ float gamma_d2(const KernF& p, float d2) {
  return kappa_gamma_d2<KT>(p, d2).g;
}

// d kappa / d lengthscale from the squared distance (FP32).
template <int KT>
__device__ __forceinline__ float dkappa_dell_d2(const KernF& p, float d2) {
  float il = p.inv_ell;
  if (KT == GRAPHGP_SQEXP) {
    return p.s2 * expf(-0.5f * d2 * il * il) * d2 * il * il * il;
  } else {
    float r = sqrtf(d2);
    if (KT == GRAPHGP_MATERN12) {
      return p.s2 * expf(-r * il) * r * il * il;
    } else if (KT == GRAPHGP_MATERN32) {
      float a = 1.7320508075688772f * r * il;
      return p.s2 * a * a * expf(-a) * il;
    } else {
      float a = 2.2360679774997896f * r * il;
      return p.s2 * a * a * (1.0f + a) * expf(-a) * il * (1.0f / 3.0f);
    }
  }
}


// kappa and d kappa / d lengthscale of one distance from one exponential
// (the kernel-parameter gradient needs both for every covariance entry);
// the same values as kappa_d2 and dkappa_dell_d2.
struct KD {
  float k, dl;
};

template <int KT>
__device__ __forceinline__ KD kappa_dkappa_d2(const KernF& p, float d2) {
  const float il = p.inv_ell;
  if (KT == GRAPHGP_SQEXP) {
    const float e = expf(-0.5f * d2 * il * il);
    return KD{p.s2 * e, p.s2 * e * d2 * il * il * il};
  } else {
    const float r = sqrtf(d2);
    if (KT == GRAPHGP_MATERN12) {
      const float e = expf(-r * il);
      return KD{p.s2 * e, p.s2 * e * r * il * il};
    } else if (KT == GRAPHGP_MATERN32) {
      const float a = 1.7320508075688772f * r * il;
      const float e = expf(-a);
      return KD{p.s2 * (1.0f + a) * e, p.s2 * a * a * e * il};
    } else {
      const float a = 2.2360679774997896f * r * il;
      const float e = expf(-a);
      return KD{p.s2 * (1.0f + a + a * a * (1.0f / 3.0f)) * e,
                p.s2 * a * a * (1.0f + a) * e * il * (1.0f / 3.0f)};
    }
  }
}

__device__ __forceinline__ float sqdist(float4 a, float4 b) {
  float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

inline KernF make_kernf(const graphgp_kernel& k) {
  KernF p;
  p.s2 = (float)k.sigma2;
  p.inv_ell = (float)(1.0 / k.lengthscale);
  p.nug = (float)k.nugget;
  const double tol = k.rescue_tol == 0.0 ? kDefaultRescueTol : k.rescue_tol;
  p.resc_T = tol < 0.0 ? -1.0f : (float)(tol * 16777216.0);
  p.s2d = k.sigma2;
  p.elld = k.lengthscale;
  p.nugd = k.nugget;
  return p;
}

// Device-dependent launch sizes are cached per device index.
constexpr int kMaxDevices = 64;

inline int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev >= 0 && dev < kMaxDevices) ? dev : 0;
}

inline int num_sms() {
  static int cache[kMaxDevices] = {};
  const int dev = current_device();
  if (!cache[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}

// Kernels whose dynamic shared memory grows with the number of depth levels
// (two int32 per level in the tile walks): above the 48 KB a launch gets by
// default the kernel must opt in, up to the 227 KB of one block.
template <class F>
inline cudaError_t allow_dyn_smem(F fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

inline unsigned grid_for(int64_t n, int block, int64_t cap_per_sm = 32) {
  int64_t g = (n + block - 1) / block;
  int64_t cap = (int64_t)num_sms() * cap_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// entry points implemented across translation units
// ---------------------------------------------------------------------------
// radix sort of (key, value) pairs, stable, keys compared on `bits` low bits
int radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in,
                     uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                     int bits, cudaStream_t s);
// on-the-fly sweeps of the 32-lane group form (16 < k <= 32), fused_group.cu
int whiten_fused_group(graphgp_graph_t g, int type, const KernF& kf, const float* v, float* xi,
                       double* sq, double* logdet, unsigned long long* not_pd, cudaStream_t s);
int generate_fused_group(graphgp_graph_t g, int type, const KernF& kf, const float* xi, float* v,
                         unsigned long long* not_pd, cudaStream_t s);
// exclusive scan of uint32 counts into uint32 offsets; returns total on request
int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n,
                       cudaStream_t s);

int tree_build(const float* pts, int64_t N, int rule, int32_t* tree_point,
               uint8_t* split_dim, int32_t* inorder, int32_t* node_at_inorder,
               cudaStream_t s);
int knn_query(const float* pts, const int32_t* tree_point,
              const uint8_t* split_dim, const int32_t* node_at_inorder,
              int64_t N, int k, int64_t n0, int32_t* nbr_tree, uint32_t* err,
              cudaStream_t s);

// levels, checks and whiten tiles; have_keys: tmp_vec holds in-order keys
int graph_finish_device(graphgp_graph_t g, cudaStream_t s, bool have_keys);

int dense_factor(graphgp_graph_t g, graphgp_factor_t f, const KernF& kp,
                 int type, cudaStream_t s);
int point_factor(graphgp_graph_t g, graphgp_factor_t f, const KernF& kp,
                 int type, cudaStream_t s);


bool valid_kernel(const graphgp_kernel* kern);

// Dense block of the on-the-fly forms into a temporary handle whose arrays
// live in the call's scratch (L0, L0^-1, sigma_0..n0-1); the block's
// log-determinant is added to *logdet and its floored pivots to *not_pd.
int dense_into(graphgp_graph_t g, const graphgp_kernel* kern, Scratch& sc, double* logdet,
               unsigned long long* not_pd, graphgp_factor_s& f, cudaStream_t s);

// y = M x for the n0 x n0 row-major lower-triangular M (the dense block's
// L0 or L0^-1); adds sum y_i^2 to *sq when sq is given.
int dense_matvec(const float* M, const float* x, float* y, int n0, double* sq, cudaStream_t s);

}  // namespace ggp
