// Graph construction entry points (Sec. 2.2 "Batch construction", Sec. 2.3
// last paragraph): canonicalised input, k-d tree, preceding kNN, depth by the
// parallel fixed point, depth-sorted graph order, relabelled neighbour rows,
// and the level tables of the sweeps.  Also import / export / save /
// load / info / destroy of graph handles.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

namespace ggp {
namespace {

// Points of dimension d <= 3 become 3-D points with zero in the missing
// coordinates: distances are unchanged (exact zero terms), and the widest-
// extent split never picks a zero-extent dimension while a real one has a
// positive extent (all extents zero: lowest dimension, as in d dimensions).
__global__ void canonicalise_kernel(const float* __restrict__ in, int d, float* __restrict__ out,
                                    int64_t n, unsigned long long* __restrict__ bad) {
  unsigned long long local = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * 3;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / 3;
    const int c = (int)(e - i * 3);
    float x = c < d ? in[i * d + c] : 0.0f;
    if (!isfinite(x)) local++;
    out[e] = (x == 0.0f) ? 0.0f : x;  // -0.0 becomes +0.0
  }
  if (local) atomicAdd(bad, local);
}

// Parallel depth update of Sec. 2.3: every point applies
// d_j = 1 + max over c(j) of d_i; repeated until nothing changes.  Depths only
// grow and never pass their final value, so the fixed point is the longest-
// path depth.  Points below the smallest index changed in a pass are final
// (their inputs did not change during the pass), so the next pass starts
// there.
__global__ void depth_pass_kernel(const int32_t* __restrict__ nbr_tree, int32_t* depth,
                                  int64_t N, int k, int64_t n0, int64_t first,
                                  unsigned long long* __restrict__ min_changed) {
  for (int64_t j = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* row = nbr_tree + (j - n0) * k;
    int32_t m = 0;
    for (int a = 0; a < k; a++) m = max(m, __ldcg(depth + row[a]));
    int32_t d = m + 1;
    if (d != __ldcg(depth + j)) {
      __stcg(depth + j, d);
      atomicMin(min_changed, (unsigned long long)j);
    }
  }
}

__global__ void max_reduce_kernel(const int32_t* __restrict__ x, int64_t n,
                                  int* __restrict__ out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, x[i]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Keys of the depth sort in in-order order, plus the level histogram (held in
// shared memory when the number of levels is small).
__global__ void depth_keys_kernel(const int32_t* __restrict__ node_at_inorder,
                                  const int32_t* __restrict__ depth, int64_t N, int nlev,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  unsigned long long* __restrict__ level_count) {
  extern __shared__ unsigned int hist[];
  bool local = nlev <= 8192;
  if (local)
    for (int i = threadIdx.x; i < nlev; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = node_at_inorder[r];
    int32_t d = depth[j];
    keys[r] = (uint32_t)d;
    vals[r] = (uint32_t)j;
    if (local)
      atomicAdd(hist + d, 1u);
    else
      atomicAdd(level_count + d, 1ull);
  }
  __syncthreads();
  if (local)
    for (int i = threadIdx.x; i < nlev; i += blockDim.x)
      if (hist[i]) atomicAdd(level_count + i, (unsigned long long)hist[i]);
}

__global__ void positions_kernel(const uint32_t* __restrict__ tree_of_pos,
                                 const int32_t* __restrict__ tree_point,
                                 const int32_t* __restrict__ inorder,
                                 const float* __restrict__ pts, int64_t N,
                                 int32_t* __restrict__ pos_of_tree, int32_t* __restrict__ order,
                                 float4* __restrict__ xs, int32_t* __restrict__ pos_key) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = (int32_t)tree_of_pos[p];
    pos_of_tree[j] = (int32_t)p;
    pos_key[p] = inorder[j];
    int64_t o = tree_point[j];
    order[p] = (int32_t)o;
    xs[p] = make_float4(pts[3 * o], pts[3 * o + 1], pts[3 * o + 2], 0.0f);
  }
}

__global__ void relabel_kernel(const uint32_t* __restrict__ tree_of_pos,
                               const int32_t* __restrict__ pos_of_tree,
                               const int32_t* __restrict__ nbr_tree, int64_t N, int k,
                               int kp, int64_t n0, int32_t* __restrict__ nbr) {
  int64_t total = (N - n0) * kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = e / kp;
    int a = (int)(e - row * kp);
    int32_t v = 0;
    if (a < k) {
      int64_t j = tree_of_pos[n0 + row];
      v = pos_of_tree[nbr_tree[(j - n0) * k + a]];
    }
    nbr[e] = v;
  }
}

__global__ void order_xs_kernel(const float* __restrict__ pts, const int32_t* __restrict__ order,
                                int64_t N, float4* __restrict__ xs) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = order[p];
    xs[p] = make_float4(pts[3 * o], pts[3 * o + 1], pts[3 * o + 2], 0.0f);
  }
}

// Every neighbour of a row must lie in an earlier depth level (Sec. 2.2:
// points of one batch never condition on each other).  Flags ERRBIT_INDEX.
__global__ void check_levels_kernel(const int32_t* __restrict__ nbr, int kp, int k, int64_t n0,
                                    const int64_t* __restrict__ level_off, int num_levels,
                                    int64_t N, uint32_t* __restrict__ err) {
  for (int64_t p = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int a0 = 1, b0 = num_levels - 1;  // level of p: last l with level_off[l] <= p
    while (a0 < b0) {
      int mid = (a0 + b0 + 1) / 2;
      if (level_off[mid] <= p) a0 = mid; else b0 = mid - 1;
    }
    int64_t start = level_off[a0];
    const int32_t* row = nbr + (p - n0) * kp;
    for (int a = 0; a < k; a++)
      if (row[a] < 0 || row[a] >= start) atomicOr(err, ERRBIT_INDEX);
  }
}

// Spatial key of a position when no k-d tree is known (imported graphs):
// its rank inside its level scaled to [0, N), so every level spans the same
// key range.
__global__ void proportional_keys_kernel(const int64_t* __restrict__ level_off, int num_levels,
                                         int64_t N, int32_t* __restrict__ key) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int a0 = 0, b0 = num_levels - 1;
    while (a0 < b0) {
      int mid = (a0 + b0 + 1) / 2;
      if (level_off[mid] <= p) a0 = mid; else b0 = mid - 1;
    }
    int64_t lo = level_off[a0], n = level_off[a0 + 1] - lo;
    key[p] = (int32_t)((p - lo) * N / n);
  }
}

// tile_start[t * L + l] = first position of level l whose key is >= t R (keys
// are ascending inside every level).
__global__ void tile_table_kernel(const int32_t* __restrict__ key,
                                  const int64_t* __restrict__ level_off, int num_levels,
                                  int64_t n_tiles, int64_t R, int32_t* __restrict__ tile_start) {
  int64_t total = (n_tiles + 1) * num_levels;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = e / num_levels;
    int l = (int)(e - t * num_levels);
    int64_t a0 = level_off[l], b0 = level_off[l + 1];
    int64_t target = t * R;
    while (a0 < b0) {
      int64_t mid = (a0 + b0) / 2;
      if ((int64_t)key[mid] < target) a0 = mid + 1; else b0 = mid;
    }
    tile_start[e] = (int32_t)a0;
  }
}

int alloc_common(graphgp_graph_t g) {
  GGP_TRY(g->mem.alloc(&g->pts_in, g->N * 3));
  GGP_TRY(g->mem.alloc(&g->xs, g->N));
  GGP_TRY(g->mem.alloc(&g->order, g->N));
  GGP_TRY(g->mem.alloc(&g->nbr, (g->N - g->n0) * g->kp));
  GGP_TRY(g->mem.alloc(&g->err, 1));
  GGP_TRY(g->mem.alloc(&g->tmp_vec, g->N));
  GGP_TRY(g->mem.alloc(&g->tmp_vec2, g->N));
  return GRAPHGP_OK;
}

}  // namespace

// Level offsets on the device, the sweep barrier counters, and a check that
// every neighbour lies in an earlier level.
int graph_finish_device(graphgp_graph_t g, cudaStream_t s, bool have_keys) {
  g->max_level_size = 0;
  for (int l = 1; l < g->num_levels; l++)
    g->max_level_size = std::max<int64_t>(g->max_level_size, g->level_off_h[l + 1] - g->level_off_h[l]);
  GGP_TRY(g->mem.alloc(&g->level_off_d, g->num_levels + 1));
  GGP_TRY(g->mem.alloc(&g->level_bar, g->num_levels));
  GGP_CUDA(cudaMemcpyAsync(g->level_off_d, g->level_off_h.data(),
                           (g->num_levels + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (g->N > g->n0) {
    check_levels_kernel<<<grid_for(g->N - g->n0, 256), 256, 0, s>>>(
        g->nbr, g->kp, g->k, g->n0, g->level_off_d, g->num_levels, g->N, g->err);
    GGP_CUDA(cudaGetLastError());
  }
  // spatial tiles of the whiten sweep; the keys sit in tmp_vec
  int32_t* key = (int32_t*)g->tmp_vec;
  if (!have_keys) {
    proportional_keys_kernel<<<grid_for(g->N, 256), 256, 0, s>>>(g->level_off_d, g->num_levels,
                                                                 g->N, key);
    GGP_CUDA(cudaGetLastError());
  }
  g->tile_R = kTileR;
  g->n_tiles = (g->N + kTileR - 1) / kTileR;
  GGP_TRY(g->mem.alloc(&g->tile_start, (g->n_tiles + 1) * g->num_levels));
  tile_table_kernel<<<grid_for((g->n_tiles + 1) * g->num_levels, 256), 256, 0, s>>>(
      key, g->level_off_d, g->num_levels, g->n_tiles, kTileR, g->tile_start);
  GGP_CUDA(cudaGetLastError());
  GGP_CUDA(cudaStreamSynchronize(s));
  uint32_t err = 0;
  GGP_CUDA(cudaMemcpy(&err, g->err, 4, cudaMemcpyDeviceToHost));
  if (err & ERRBIT_INDEX) return GRAPHGP_ERR_INVALID;
  return GRAPHGP_OK;
}

}  // namespace ggp

using namespace ggp;

extern "C" int graphgp_build_graph(const float* points_d, int64_t N, int d, int k,
                                   const graphgp_build_opts* opts, void* stream,
                                   graphgp_graph_t* out) {
  if (!out) return GRAPHGP_ERR_INVALID;
  *out = nullptr;
  if (!points_d || N < 1 || N >= ((int64_t)1 << 31) || d < 1 || d > 3 || k < 1 || k > kMaxK)
    return GRAPHGP_ERR_INVALID;
  int n0 = opts && opts->n0 > 0 ? opts->n0 : (int)std::min<int64_t>(N, std::max(k, 256));
  int rule = opts ? opts->split_rule : 0;
  if (n0 < k || n0 > N || n0 > 2048 || (rule != 0 && rule != 1) || (rule == 1 && d != 3))
    return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  graphgp_graph_t g = new (std::nothrow) graphgp_graph_s();
  if (!g) return GRAPHGP_ERR_OOM;
  g->N = N;
  g->k = k;
  g->kp = row_stride(k);
  g->n0 = n0;
  g->max_spin = opts && opts->max_spin > 0 ? opts->max_spin : 20000000;
  auto fail = [&](int rc) {
    g->mem.free_all();
    delete g;
    return rc;
  };
  int rc = alloc_common(g);
  if (rc < 0) return fail(rc);
  rc = [&]() -> int {
    Scratch sc(s);
    unsigned long long* bad = nullptr;
    GGP_TRY(sc.alloc(&bad, 1));
    GGP_CUDA(cudaMemsetAsync(bad, 0, 8, s));
    GGP_CUDA(cudaMemsetAsync(g->err, 0, 4, s));
    canonicalise_kernel<<<grid_for(N * 3, 256), 256, 0, s>>>(points_d, d, g->pts_in, N, bad);
    GGP_CUDA(cudaGetLastError());
    unsigned long long nbad = 0;
    GGP_CUDA(cudaMemcpyAsync(&nbad, bad, 8, cudaMemcpyDeviceToHost, s));
    GGP_CUDA(cudaStreamSynchronize(s));
    if (nbad) return GRAPHGP_ERR_NAN;
    // tree
    GGP_TRY(g->mem.alloc(&g->tree_point, N));
    GGP_TRY(g->mem.alloc(&g->split_dim, N));
    GGP_TRY(g->mem.alloc(&g->inorder, N));
    GGP_TRY(g->mem.alloc(&g->depth_tree, N));
    GGP_TRY(g->mem.alloc(&g->nbr_tree, (N - n0) * k));
    g->has_tree = true;
    int32_t* node_at_inorder = nullptr;
    GGP_TRY(sc.alloc(&node_at_inorder, N));
    GGP_TRY(tree_build(g->pts_in, N, rule, g->tree_point, g->split_dim, g->inorder,
                       node_at_inorder, s));
    // preceding kNN
    GGP_TRY(knn_query(g->pts_in, g->tree_point, g->split_dim, node_at_inorder, N, k, n0,
                      g->nbr_tree, g->err, s));
    {
      uint32_t e = 0;
      GGP_CUDA(cudaMemcpyAsync(&e, g->err, 4, cudaMemcpyDeviceToHost, s));
      GGP_CUDA(cudaStreamSynchronize(s));
      if (e) return GRAPHGP_ERR_INVALID;
    }
    // depth
    GGP_CUDA(cudaMemsetAsync(g->depth_tree, 0, N * sizeof(int32_t), s));
    unsigned long long* minc = nullptr;
    GGP_TRY(sc.alloc(&minc, 1));
    // One k-d tree level at a time: a node's neighbours lie in its own or an
    // earlier tree level, so once the earlier levels are final a level needs
    // only as many passes as its own longest internal chain.
    int64_t passes = 0;
    for (int t = 0; ((int64_t(1) << t) - 1) < N; t++) {
      int64_t first = std::max<int64_t>(n0, (int64_t(1) << t) - 1);
      const int64_t end = std::min<int64_t>(N, (int64_t(2) << t) - 1);
      while (first < end) {
        const unsigned long long none = ~0ull;
        GGP_CUDA(cudaMemcpyAsync(minc, &none, 8, cudaMemcpyHostToDevice, s));
        depth_pass_kernel<<<grid_for(end - first, 256, 16), 256, 0, s>>>(
            g->nbr_tree, g->depth_tree, end, k, n0, first, minc);
        GGP_CUDA(cudaGetLastError());
        unsigned long long mc = 0;
        GGP_CUDA(cudaMemcpyAsync(&mc, minc, 8, cudaMemcpyDeviceToHost, s));
        GGP_CUDA(cudaStreamSynchronize(s));
        if (mc == none) break;
        first = (int64_t)mc;
        if (++passes > N) return GRAPHGP_ERR_TIMEOUT;
      }
    }
    int* dmax = nullptr;
    GGP_TRY(sc.alloc(&dmax, 1));
    GGP_CUDA(cudaMemsetAsync(dmax, 0, 4, s));
    max_reduce_kernel<<<grid_for(N, 256), 256, 0, s>>>(g->depth_tree, N, dmax);
    GGP_CUDA(cudaGetLastError());
    int maxd = 0;
    GGP_CUDA(cudaMemcpyAsync(&maxd, dmax, 4, cudaMemcpyDeviceToHost, s));
    GGP_CUDA(cudaStreamSynchronize(s));
    g->num_levels = maxd + 1;
    // depth-sorted order: stable by (depth, in-order rank)
    uint32_t *keys = nullptr, *vals = nullptr, *keys_s = nullptr, *tree_of_pos = nullptr;
    unsigned long long* cnt = nullptr;
    GGP_TRY(sc.alloc(&keys, N));
    GGP_TRY(sc.alloc(&vals, N));
    GGP_TRY(sc.alloc(&keys_s, N));
    GGP_TRY(sc.alloc(&tree_of_pos, N));
    GGP_TRY(sc.alloc(&cnt, g->num_levels));
    GGP_CUDA(cudaMemsetAsync(cnt, 0, g->num_levels * 8, s));
    size_t hsm = g->num_levels <= 8192 ? (size_t)g->num_levels * 4 : 0;
    depth_keys_kernel<<<grid_for(N, 256, 4), 256, hsm, s>>>(node_at_inorder, g->depth_tree, N,
                                                            g->num_levels, keys, vals, cnt);
    GGP_CUDA(cudaGetLastError());
    int bits = 0;
    while ((1u << bits) <= (unsigned)maxd) bits++;
    GGP_TRY(radix_sort_pairs(keys, vals, keys_s, tree_of_pos, N, bits, s));
    int32_t* pos_of_tree = nullptr;
    GGP_TRY(sc.alloc(&pos_of_tree, N));
    positions_kernel<<<grid_for(N, 256), 256, 0, s>>>(tree_of_pos, g->tree_point, g->inorder,
                                                      g->pts_in, N, pos_of_tree, g->order, g->xs,
                                                      (int32_t*)g->tmp_vec);
    GGP_CUDA(cudaGetLastError());
    if (N > n0) {
      relabel_kernel<<<grid_for((N - n0) * g->kp, 256), 256, 0, s>>>(
          tree_of_pos, pos_of_tree, g->nbr_tree, N, k, g->kp, n0, g->nbr);
      GGP_CUDA(cudaGetLastError());
    }
    std::vector<unsigned long long> counts(g->num_levels);
    GGP_CUDA(cudaMemcpyAsync(counts.data(), cnt, g->num_levels * 8, cudaMemcpyDeviceToHost, s));
    GGP_CUDA(cudaStreamSynchronize(s));
    g->level_off_h.assign(g->num_levels + 1, 0);
    for (int l = 0; l < g->num_levels; l++) g->level_off_h[l + 1] = g->level_off_h[l] + counts[l];
    if (g->level_off_h[1] != n0) return GRAPHGP_ERR_INVALID;
    return GRAPHGP_OK;
  }();
  if (rc < 0) return fail(rc);
  rc = graph_finish_device(g, s, true);
  if (rc < 0) return fail(rc);
  *out = g;
  return GRAPHGP_OK;
}

extern "C" int graphgp_graph_import(const float* points_h, int64_t N, int k, int n0,
                                    const int32_t* order_h, const int32_t* nbr_h,
                                    const int64_t* level_offsets_h, int num_levels,
                                    void* stream, graphgp_graph_t* out) {
  if (!out) return GRAPHGP_ERR_INVALID;
  *out = nullptr;
  if (!points_h || !order_h || !level_offsets_h || N < 1 || N >= ((int64_t)1 << 31) || k < 1 ||
      k > kMaxK || n0 < k || n0 > N || n0 > 2048 || num_levels < 1 || (N > n0 && !nbr_h))
    return GRAPHGP_ERR_INVALID;
  // validation on the host: order is a permutation, levels are consistent,
  // every neighbour lies in an earlier level
  if (level_offsets_h[0] != 0 || level_offsets_h[num_levels] != N) return GRAPHGP_ERR_INVALID;
  if (num_levels >= 2 && level_offsets_h[1] != n0) return GRAPHGP_ERR_INVALID;
  if (num_levels == 1 && N != n0) return GRAPHGP_ERR_INVALID;
  for (int l = 0; l < num_levels; l++)
    if (level_offsets_h[l + 1] <= level_offsets_h[l]) return GRAPHGP_ERR_INVALID;
  {
    std::vector<uint8_t> seen(N, 0);
    for (int64_t p = 0; p < N; p++) {
      int32_t o = order_h[p];
      if (o < 0 || o >= N || seen[o]) return GRAPHGP_ERR_INVALID;
      seen[o] = 1;
    }
    int l = 1;
    for (int64_t p = n0; p < N; p++) {
      while (p >= level_offsets_h[l + 1]) l++;
      for (int a = 0; a < k; a++) {
        int32_t c = nbr_h[(p - n0) * k + a];
        if (c < 0 || c >= level_offsets_h[l]) return GRAPHGP_ERR_INVALID;
      }
    }
    for (int64_t i = 0; i < N * 3; i++)
      if (!std::isfinite(points_h[i])) return GRAPHGP_ERR_NAN;
  }
  cudaStream_t s = (cudaStream_t)stream;
  graphgp_graph_t g = new (std::nothrow) graphgp_graph_s();
  if (!g) return GRAPHGP_ERR_OOM;
  g->N = N;
  g->k = k;
  g->kp = row_stride(k);
  g->n0 = n0;
  g->num_levels = num_levels;
  g->max_spin = 20000000;
  g->level_off_h.assign(level_offsets_h, level_offsets_h + num_levels + 1);
  auto fail = [&](int rc) {
    g->mem.free_all();
    delete g;
    return rc;
  };
  int rc = alloc_common(g);
  if (rc < 0) return fail(rc);
  rc = [&]() -> int {
    std::vector<float> pts(points_h, points_h + N * 3);
    for (auto& x : pts)
      if (x == 0.0f) x = 0.0f;
    std::vector<int32_t> nbrp((size_t)(N - n0) * g->kp, 0);
    for (int64_t r = 0; r < N - n0; r++)
      std::memcpy(&nbrp[r * g->kp], nbr_h + r * k, k * sizeof(int32_t));
    GGP_CUDA(cudaMemsetAsync(g->err, 0, 4, s));
    GGP_CUDA(cudaMemcpyAsync(g->pts_in, pts.data(), N * 12, cudaMemcpyHostToDevice, s));
    GGP_CUDA(cudaMemcpyAsync(g->order, order_h, N * 4, cudaMemcpyHostToDevice, s));
    if (N > n0)
      GGP_CUDA(cudaMemcpyAsync(g->nbr, nbrp.data(), nbrp.size() * 4, cudaMemcpyHostToDevice, s));
    order_xs_kernel<<<grid_for(N, 256), 256, 0, s>>>(g->pts_in, g->order, N, g->xs);
    GGP_CUDA(cudaGetLastError());
    GGP_CUDA(cudaStreamSynchronize(s));
    return GRAPHGP_OK;
  }();
  if (rc < 0) return fail(rc);
  rc = graph_finish_device(g, s, false);
  if (rc < 0) return fail(rc);
  *out = g;
  return GRAPHGP_OK;
}

extern "C" int graphgp_graph_info(graphgp_graph_t g, int64_t* N, int* k, int* n0,
                                  int* num_levels, size_t* bytes) {
  if (!g) return GRAPHGP_ERR_INVALID;
  if (N) *N = g->N;
  if (k) *k = g->k;
  if (n0) *n0 = g->n0;
  if (num_levels) *num_levels = g->num_levels;
  if (bytes) *bytes = g->mem.bytes;
  return GRAPHGP_OK;
}

extern "C" int graphgp_graph_export(graphgp_graph_t g, int32_t* order_d, int32_t* nbr_d,
                                    int64_t* level_offsets_h, void* stream) {
  if (!g) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (order_d)
    GGP_CUDA(cudaMemcpyAsync(order_d, g->order, g->N * 4, cudaMemcpyDeviceToDevice, s));
  if (nbr_d && g->N > g->n0)
    GGP_CUDA(cudaMemcpy2DAsync(nbr_d, g->k * 4, g->nbr, g->kp * 4, g->k * 4, g->N - g->n0,
                               cudaMemcpyDeviceToDevice, s));
  if (level_offsets_h)
    std::memcpy(level_offsets_h, g->level_off_h.data(), (g->num_levels + 1) * sizeof(int64_t));
  return GRAPHGP_OK;
}

extern "C" int graphgp_graph_export_tree(graphgp_graph_t g, int32_t* tree_point_d,
                                         uint8_t* split_dim_d, int32_t* inorder_d,
                                         int32_t* depth_d, int32_t* nbr_tree_d, void* stream) {
  if (!g || !g->has_tree) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t N = g->N;
  if (tree_point_d)
    GGP_CUDA(cudaMemcpyAsync(tree_point_d, g->tree_point, N * 4, cudaMemcpyDeviceToDevice, s));
  if (split_dim_d)
    GGP_CUDA(cudaMemcpyAsync(split_dim_d, g->split_dim, N, cudaMemcpyDeviceToDevice, s));
  if (inorder_d)
    GGP_CUDA(cudaMemcpyAsync(inorder_d, g->inorder, N * 4, cudaMemcpyDeviceToDevice, s));
  if (depth_d)
    GGP_CUDA(cudaMemcpyAsync(depth_d, g->depth_tree, N * 4, cudaMemcpyDeviceToDevice, s));
  if (nbr_tree_d && N > g->n0)
    GGP_CUDA(cudaMemcpyAsync(nbr_tree_d, g->nbr_tree, (N - g->n0) * g->k * 4,
                             cudaMemcpyDeviceToDevice, s));
  return GRAPHGP_OK;
}

namespace {
const char kMagic[8] = {'G', 'G', 'P', 'G', 'R', 'A', 'F', '1'};
}

extern "C" int graphgp_graph_save(graphgp_graph_t g, const char* path, void* stream) {
  if (!g || !path) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t N = g->N, rows = g->N - g->n0;
  std::vector<float> pts(N * 3);
  std::vector<int32_t> order(N), nbr(rows * g->k);
  GGP_CUDA(cudaMemcpyAsync(pts.data(), g->pts_in, N * 12, cudaMemcpyDeviceToHost, s));
  GGP_CUDA(cudaMemcpyAsync(order.data(), g->order, N * 4, cudaMemcpyDeviceToHost, s));
  if (rows)
    GGP_CUDA(cudaMemcpy2DAsync(nbr.data(), g->k * 4, g->nbr, g->kp * 4, g->k * 4, rows,
                               cudaMemcpyDeviceToHost, s));
  GGP_CUDA(cudaStreamSynchronize(s));
  FILE* f = std::fopen(path, "wb");
  if (!f) return GRAPHGP_ERR_IO;
  int32_t hdr[4] = {1, g->k, g->n0, g->num_levels};
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&N, 8, 1, f) == 1 &&
            std::fwrite(hdr, 4, 4, f) == 4 &&
            std::fwrite(pts.data(), 4, pts.size(), f) == pts.size() &&
            std::fwrite(order.data(), 4, order.size(), f) == order.size() &&
            std::fwrite(nbr.data(), 4, nbr.size(), f) == nbr.size() &&
            std::fwrite(g->level_off_h.data(), 8, g->level_off_h.size(), f) ==
                g->level_off_h.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? GRAPHGP_OK : GRAPHGP_ERR_IO;
}

extern "C" int graphgp_graph_load(const char* path, void* stream, graphgp_graph_t* out) {
  if (!path || !out) return GRAPHGP_ERR_INVALID;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return GRAPHGP_ERR_IO;
  char magic[8];
  int64_t N = 0;
  int32_t hdr[4];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(&N, 8, 1, f) == 1 && std::fread(hdr, 4, 4, f) == 4 && hdr[0] == 1 &&
            N >= 1 && N < ((int64_t)1 << 31) && hdr[1] >= 1 && hdr[1] <= kMaxK && hdr[2] >= 1 &&
            hdr[2] <= N && hdr[3] >= 1 && hdr[3] <= N;
  if (!ok) {
    std::fclose(f);
    return GRAPHGP_ERR_IO;
  }
  int k = hdr[1], n0 = hdr[2], nl = hdr[3];
  std::vector<float> pts(N * 3);
  std::vector<int32_t> order(N), nbr((N - n0) * k);
  std::vector<int64_t> lo(nl + 1);
  ok = std::fread(pts.data(), 4, pts.size(), f) == pts.size() &&
       std::fread(order.data(), 4, order.size(), f) == order.size() &&
       std::fread(nbr.data(), 4, nbr.size(), f) == nbr.size() &&
       std::fread(lo.data(), 8, lo.size(), f) == lo.size();
  std::fclose(f);
  if (!ok) return GRAPHGP_ERR_IO;
  return graphgp_graph_import(pts.data(), N, k, n0, order.data(), nbr.data(), lo.data(), nl,
                              stream, out);
}

extern "C" void graphgp_graph_destroy(graphgp_graph_t g) {
  if (!g) return;
  cudaDeviceSynchronize();
  g->mem.free_all();
  delete g;
}
