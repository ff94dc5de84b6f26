// Left-balanced k-d tree in the bit-reversed layout (Sec. 2.2 "Tree
// ordering", "Bit-reversed ordering"; Sec. 2.3: sort-based GPU build).
//
// Design: the points are sorted once per dimension by (coordinate, input
// index).  The three sorted orders are kept, each restricted to every open
// subtree, in the subtree's in-order slot range.  Processing the tree one
// level at a time:
//   * the bounding box of a subtree is read off the ends of its three sorted
//     ranges (no reduction), which fixes the split dimension;
//   * the median of the split dimension is the element at offset m (the size
//     of the left subtree) of that dimension's range: no selection pass;
//   * the two other orders are stably partitioned (left part, node, right
//     part) with one exclusive scan each, so they stay sorted.
// Every step is a permutation fixed by the data, so the result is exactly
// the recursive definition: split on the widest FP32 extent (ties to the
// lowest dimension) or on level mod 3, median by (coordinate, input index).
#include "common.cuh"

namespace ggp {
namespace {

__device__ __forceinline__ int node_level(int64_t j) {
  return 63 - __clzll((unsigned long long)(j + 1));
}

// Number of existing nodes in the subtree of j: the descendants of the node
// at (level l, position p) on level m occupy positions p + t 2^l, t < 2^(m-l).
__device__ int64_t subtree_nodes(int64_t j, int64_t N) {
  if (j >= N) return 0;
  int l = node_level(j);
  int64_t p = j - ((int64_t(1) << l) - 1);
  int64_t stride = int64_t(1) << l;
  int64_t count = 0;
  for (int m = l; m < 63; m++) {
    int64_t lo = (int64_t(1) << m) - 1 + p;
    if (lo >= N) break;
    int64_t cap = int64_t(1) << (m - l);
    int64_t n = (N - lo + stride - 1) / stride;
    count += n < cap ? n : cap;
  }
  return count;
}

__device__ __forceinline__ uint32_t orderable(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void presort_keys_kernel(const float* __restrict__ pts, int64_t N,
                                    int dim, uint32_t* __restrict__ keys,
                                    uint32_t* __restrict__ ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = orderable(pts[3 * i + dim]);
    ids[i] = (uint32_t)i;
  }
}

struct Orders {
  const int32_t* o[3];
};

// One thread per node of level l: split dimension, median point, in-order
// rank, and the in-order start of both children.
__global__ void level_nodes_kernel(const float* __restrict__ pts, int64_t N,
                                   int l, int rule, Orders ord,
                                   int32_t* __restrict__ start,
                                   int32_t* __restrict__ msize,
                                   int32_t* __restrict__ tree_point,
                                   uint8_t* __restrict__ split_dim,
                                   int32_t* __restrict__ inorder,
                                   int32_t* __restrict__ node_at_inorder) {
  int64_t first = (int64_t(1) << l) - 1;
  int64_t count = int64_t(1) << l;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = first + t;
    if (j >= N) return;
    int64_t S = subtree_nodes(j, N);
    int64_t lc = j + (int64_t(1) << l), rc = j + (int64_t(2) << l);
    int64_t m = subtree_nodes(lc, N);
    int64_t st = start[j];
    int dim;
    if (rule == 0) {
      float ext[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        float lo = pts[3 * (int64_t)ord.o[d][st] + d];
        float hi = pts[3 * (int64_t)ord.o[d][st + S - 1] + d];
        ext[d] = __fsub_rn(hi, lo);
      }
      dim = 0;
      if (ext[1] > ext[dim]) dim = 1;
      if (ext[2] > ext[dim]) dim = 2;
    } else {
      dim = l % 3;
    }
    int32_t p = ord.o[dim][st + m];
    tree_point[j] = p;
    split_dim[j] = (uint8_t)dim;
    inorder[j] = (int32_t)(st + m);
    msize[j] = (int32_t)m;
    node_at_inorder[st + m] = (int32_t)j;
    if (lc < N) start[lc] = (int32_t)st;
    if (rc < N) start[rc] = (int32_t)(st + m + 1);
  }
}

// One thread per in-order slot: the side (0 left, 1 node, 2 right) of the
// element found in the split dimension's order, and the slot's subtree on
// the next level (-1 once it holds a finished node).
__global__ void slot_side_kernel(int64_t N, Orders ord,
                                 const int32_t* __restrict__ seg,
                                 int32_t* __restrict__ seg_next,
                                 const int32_t* __restrict__ start,
                                 const int32_t* __restrict__ msize,
                                 const uint8_t* __restrict__ split_dim,
                                 uint8_t* __restrict__ side) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = seg[x];
    if (j < 0) {
      seg_next[x] = -1;
      continue;
    }
    int64_t r = x - start[j];
    int64_t m = msize[j];
    int l = node_level(j);
    int32_t e = ord.o[split_dim[j]][x];
    uint8_t sd = r < m ? 0 : (r == m ? 1 : 2);
    side[e] = sd;
    seg_next[x] = sd == 0 ? (int32_t)(j + (int64_t(1) << l))
                          : (sd == 1 ? -1 : (int32_t)(j + (int64_t(2) << l)));
  }
}

// Flags of the elements that go left in the order of dimension A, inside
// subtrees that do not split on A; records the slot of each node element.
__global__ void part_flags_kernel(int64_t N, int A, const int32_t* __restrict__ ordA,
                                  const int32_t* __restrict__ seg,
                                  const uint8_t* __restrict__ split_dim,
                                  const uint8_t* __restrict__ side,
                                  uint32_t* __restrict__ flags,
                                  int32_t* __restrict__ node_slot) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = seg[x];
    uint32_t f = 0;
    if (j >= 0 && split_dim[j] != A) {
      uint8_t sd = side[ordA[x]];
      f = sd == 0;
      if (sd == 1) node_slot[j] = (int32_t)x;
    }
    flags[x] = f;
  }
}

__global__ void part_scatter_kernel(int64_t N, int A,
                                    const int32_t* __restrict__ ordA,
                                    int32_t* __restrict__ ordA_next,
                                    const int32_t* __restrict__ seg,
                                    const uint8_t* __restrict__ split_dim,
                                    const uint8_t* __restrict__ side,
                                    const uint32_t* __restrict__ pre,
                                    const int32_t* __restrict__ start,
                                    const int32_t* __restrict__ msize,
                                    const int32_t* __restrict__ node_slot) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = seg[x];
    int32_t e = ordA[x];
    int64_t dest = x;
    if (j >= 0 && split_dim[j] != A) {
      int64_t st = start[j];
      int64_t m = msize[j];
      int64_t lr = (int64_t)pre[x] - (int64_t)pre[st];
      uint8_t sd = side[e];
      if (sd == 0) {
        dest = st + lr;
      } else if (sd == 1) {
        dest = st + m;
      } else {
        int64_t nb = node_slot[j] < x ? 1 : 0;
        dest = st + m + 1 + ((x - st) - lr - nb);
      }
    }
    ordA_next[dest] = e;
  }
}

}  // namespace

int tree_build(const float* pts, int64_t N, int rule, int32_t* tree_point,
               uint8_t* split_dim, int32_t* inorder, int32_t* node_at_inorder,
               cudaStream_t s) {
  if (N <= 0) return GRAPHGP_OK;
  Scratch sc(s);
  int32_t* ord[3][2];
  uint32_t *keys = nullptr, *keys_sorted = nullptr, *ids = nullptr;
  for (int d = 0; d < 3; d++)
    for (int b = 0; b < 2; b++) GGP_TRY(sc.alloc(&ord[d][b], N));
  GGP_TRY(sc.alloc(&keys, N));
  GGP_TRY(sc.alloc(&keys_sorted, N));
  GGP_TRY(sc.alloc(&ids, N));
  const int B = 256;
  unsigned grid = grid_for(N, B);
  for (int d = 0; d < 3; d++) {
    presort_keys_kernel<<<grid, B, 0, s>>>(pts, N, d, keys, ids);
    GGP_CUDA(cudaGetLastError());
    GGP_TRY(radix_sort_pairs(keys, ids, keys_sorted, (uint32_t*)ord[d][0], N, 32, s));
  }
  int32_t *seg[2], *start = nullptr, *msize = nullptr, *node_slot = nullptr;
  uint8_t* side = nullptr;
  uint32_t *flags = nullptr, *pre = nullptr;
  GGP_TRY(sc.alloc(&seg[0], N));
  GGP_TRY(sc.alloc(&seg[1], N));
  GGP_TRY(sc.alloc(&start, N));
  GGP_TRY(sc.alloc(&msize, N));
  GGP_TRY(sc.alloc(&node_slot, N));
  GGP_TRY(sc.alloc(&side, N));
  GGP_TRY(sc.alloc(&flags, N));
  GGP_TRY(sc.alloc(&pre, N));
  GGP_CUDA(cudaMemsetAsync(seg[0], 0, N * sizeof(int32_t), s));  // all in root
  GGP_CUDA(cudaMemsetAsync(start, 0, sizeof(int32_t), s));
  int cur[3] = {0, 0, 0};
  int sg = 0;
  int levels = 0;
  while (((int64_t(1) << levels) - 1) < N) levels++;
  for (int l = 0; l < levels; l++) {
    Orders o;
    for (int d = 0; d < 3; d++) o.o[d] = ord[d][cur[d]];
    int64_t nodes = int64_t(1) << l;
    level_nodes_kernel<<<grid_for(nodes, B), B, 0, s>>>(pts, N, l, rule, o, start, msize,
                                                        tree_point, split_dim, inorder,
                                                        node_at_inorder);
    GGP_CUDA(cudaGetLastError());
    if (l == levels - 1) break;  // last level: every subtree is a single node
    slot_side_kernel<<<grid, B, 0, s>>>(N, o, seg[sg], seg[1 - sg], start, msize, split_dim,
                                        side);
    GGP_CUDA(cudaGetLastError());
    for (int A = 0; A < 3; A++) {
      part_flags_kernel<<<grid, B, 0, s>>>(N, A, ord[A][cur[A]], seg[sg], split_dim, side, flags,
                                           node_slot);
      GGP_CUDA(cudaGetLastError());
      GGP_TRY(scan_exclusive_u32(flags, pre, N, s));
      part_scatter_kernel<<<grid, B, 0, s>>>(N, A, ord[A][cur[A]], ord[A][1 - cur[A]], seg[sg],
                                             split_dim, side, pre, start, msize, node_slot);
      GGP_CUDA(cudaGetLastError());
      cur[A] = 1 - cur[A];
    }
    sg = 1 - sg;
  }
  return GRAPHGP_OK;
}

}  // namespace ggp
