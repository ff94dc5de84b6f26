// Preceding k-nearest-neighbour search (Sec. 2.1: c(i) = the k nearest
// preceding points; Sec. 2.2: every prefix of the tree order is itself a
// valid tree, so the points preceding tree index j are searched in the
// prefix tree {0..j-1}).
//
// One thread per query, queries taken in k-d in-order rank so that a warp
// holds spatially close queries.  Stack-free traversal of the implicit tree:
// the state (current node, previous node) decides whether we arrived from
// the parent, from the near child or from the far child.  A far subtree is
// skipped only if the FP32 square of the distance to the splitting plane is
// larger than the current k-th key; every point past the plane then has a
// larger FP32 key (IEEE rounding is monotone), so the result is exactly the
// brute-force definition: the k smallest (d2, tree index) keys with
// d2 = fma(dz,dz, fma(dy,dy, dx*dx)) computed with explicit round-to-nearest
// operations.
#include "common.cuh"

namespace ggp {
namespace {

__global__ void node_coords_kernel(const float* __restrict__ pts,
                                   const int32_t* __restrict__ tree_point,
                                   const uint8_t* __restrict__ split_dim,
                                   int64_t N, float4* __restrict__ xt) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = tree_point[j];
    xt[j] = make_float4(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2],
                        __int_as_float((int)split_dim[j]));
  }
}

__device__ __forceinline__ float key_d2(float4 a, float4 b) {
  float dx = __fsub_rn(a.x, b.x);
  float dy = __fsub_rn(a.y, b.y);
  float dz = __fsub_rn(a.z, b.z);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

__device__ __forceinline__ float pick(float4 v, int d) {
  return d == 0 ? v.x : (d == 1 ? v.y : v.z);
}

// Candidate list of KM entries sorted ascending.  The first KM-k entries are
// fillers (-1, -1) that precede every real key, so the k real entries always
// sit in the last k slots and the current k-th key is entry KM-1.
template <int KM>
__device__ __forceinline__ void insert_key(float (&bd)[KM], int32_t (&bi)[KM],
                                           float d, int32_t i) {
  if (d < bd[KM - 1] || (d == bd[KM - 1] && i < bi[KM - 1])) {
    bd[KM - 1] = d;
    bi[KM - 1] = i;
#pragma unroll
    for (int m = KM - 1; m > 0; m--) {
      bool sw = bd[m] < bd[m - 1] || (bd[m] == bd[m - 1] && bi[m] < bi[m - 1]);
      float td = sw ? bd[m - 1] : bd[m];
      int32_t ti = sw ? bi[m - 1] : bi[m];
      bd[m - 1] = sw ? bd[m] : bd[m - 1];
      bi[m - 1] = sw ? bi[m] : bi[m - 1];
      bd[m] = td;
      bi[m] = ti;
    }
  }
}

template <int KM>
__global__ void __launch_bounds__(128) knn_kernel(
    const float4* __restrict__ xt, const int32_t* __restrict__ node_at_inorder,
    int64_t N, int k, int64_t n0, int32_t* __restrict__ nbr_tree, uint32_t* __restrict__ err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = node_at_inorder[r];
    if (j < n0) continue;
    float4 q = xt[j];
    float bd[KM];
    int32_t bi[KM];
#pragma unroll
    for (int a = 0; a < KM; a++) {
      bool filler = a < KM - k;
      bd[a] = filler ? -1.0f : __int_as_float(0x7f800000);
      bi[a] = filler ? -1 : 0x7fffffff;
    }
    int64_t curr = 0, prev = -1;
    while (true) {
      float4 nd = xt[curr];
      int dim = __float_as_int(nd.w);
      int l = 63 - __clzll((unsigned long long)(curr + 1));
      int64_t lc = curr + (int64_t(1) << l), rc = curr + (int64_t(2) << l);
      int64_t parent = -1;
      if (curr > 0) {
        int64_t half = int64_t(1) << (l - 1);
        parent = half - 1 + ((curr - ((int64_t(1) << l) - 1)) & (half - 1));
      }
      float qd = pick(q, dim), sd = pick(nd, dim);
      bool left_first = qd < sd;
      int64_t near_c = left_first ? lc : rc;
      int64_t far_c = left_first ? rc : lc;
      if (prev == parent) {  // arrived from above: visit the node
        insert_key<KM>(bd, bi, key_d2(nd, q), (int32_t)curr);
        if (near_c < j) {
          prev = curr;
          curr = near_c;
          continue;
        }
        prev = near_c;  // no near child: continue as if back from it
      }
      if (prev == near_c) {
        float diff = __fsub_rn(qd, sd);
        float plane = __fmul_rn(diff, diff);
        if (far_c < j && !(plane > bd[KM - 1])) {
          prev = curr;
          curr = far_c;
          continue;
        }
      }
      if (curr == 0) break;
      prev = curr;
      curr = parent;
    }
    int32_t* out = nbr_tree + (j - n0) * k;
#pragma unroll
    for (int a = 0; a < KM; a++)
      if (a >= KM - k) {
        int32_t id = bi[a];
        if (id < 0 || id >= j) {  // cannot happen for n0 >= k; guards later gathers
          id = 0;
          atomicOr(err, ERRBIT_INDEX);
        }
        out[a - (KM - k)] = id;
      }
  }
}

}  // namespace

int knn_query(const float* pts, const int32_t* tree_point,
              const uint8_t* split_dim, const int32_t* node_at_inorder,
              int64_t N, int k, int64_t n0, int32_t* nbr_tree, uint32_t* err,
              cudaStream_t s) {
  if (N <= n0) return GRAPHGP_OK;
  Scratch sc(s);
  float4* xt = nullptr;
  GGP_TRY(sc.alloc(&xt, N));
  node_coords_kernel<<<grid_for(N, 256), 256, 0, s>>>(pts, tree_point, split_dim, N, xt);
  GGP_CUDA(cudaGetLastError());
  const int B = 128;
  unsigned grid = (unsigned)((N + B - 1) / B);
  if (k <= 8)
    knn_kernel<8><<<grid, B, 0, s>>>(xt, node_at_inorder, N, k, n0, nbr_tree, err);
  else if (k <= 16)
    knn_kernel<16><<<grid, B, 0, s>>>(xt, node_at_inorder, N, k, n0, nbr_tree, err);
  else if (k <= 32)
    knn_kernel<32><<<grid, B, 0, s>>>(xt, node_at_inorder, N, k, n0, nbr_tree, err);
  else
    knn_kernel<64><<<grid, B, 0, s>>>(xt, node_at_inorder, N, k, n0, nbr_tree, err);
  GGP_CUDA(cudaGetLastError());
  return GRAPHGP_OK;
}

}  // namespace ggp
