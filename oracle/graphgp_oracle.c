/*
 * graphgp_oracle.c -- plain, slow, obviously-correct FP64 CPU reference for
 * the GraphGP Vecchia hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two are compared on
 * the same seeded inputs.
 *
 * Every function cites the passage of the GraphGP paper it follows.  Where
 * the paper is silent the reading used is stated in the comment.  Compiled
 * with -ffp-contract=off so that every FP32 expression below rounds exactly
 * as written (the kNN key is an FP32-defined function).
 *
 * Layouts: points float[N][3]; tree arrays are indexed by tree index j
 * (bit-reversed level order); graph arrays by position (depth-sorted order).
 * Neighbour rows hold k entries; -1 marks an absent entry (rows of points
 * with fewer than k predecessors, used by the full-conditioning checks).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR -1
/* Pivot floor relative to the original diagonal entry (reading of the paper,
 * which is silent on non-positive-definite matrices). */
#define ORC_PD_FLOOR 1e-7

/* ------------------------------------------------------------------------ */
/* Tree shape: Sec. 2.2, "Bit-reversed ordering".  Level l holds tree indices
 * [2^l - 1, 2^(l+1) - 1); node j at level l has left child j + 2^l and right
 * child j + 2^(l+1).                                                        */
/* ------------------------------------------------------------------------ */

int oracle_level(int64_t j) {
  int l = 0;
  while ((((int64_t)2) << l) - 1 <= j) l++;
  return l;
}

int64_t oracle_left(int64_t j) { return j + (((int64_t)1) << oracle_level(j)); }

int64_t oracle_right(int64_t j) { return j + (((int64_t)2) << oracle_level(j)); }

/* The left child of (l, p) sits at (l+1, p) and the right child at
 * (l+1, p + 2^l), so the parent of (l, q) is (l-1, q mod 2^(l-1)). */
int64_t oracle_parent(int64_t j) {
  if (j <= 0) return -1;
  int l = oracle_level(j);
  int64_t q = j - ((((int64_t)1) << l) - 1);
  int64_t half = ((int64_t)1) << (l - 1);
  return (half - 1) + (q % half);
}

/* Number of nodes (< N) in the subtree of j, by walking the subtree level
 * by level: the descendants of (l, p) at level m are the positions p + t*2^l,
 * t < 2^(m-l). */
int64_t oracle_subtree_size(int64_t j, int64_t N) {
  if (j < 0 || j >= N) return 0;
  int l = oracle_level(j);
  int64_t p = j - ((((int64_t)1) << l) - 1);
  int64_t step = ((int64_t)1) << l;
  int64_t total = 0;
  for (int m = l;; m++) {
    int64_t first = ((((int64_t)1) << m) - 1) + p;
    if (first >= N) break;
    int64_t slots = ((int64_t)1) << (m - l);
    int64_t fit = (N - first + step - 1) / step;
    total += (fit < slots) ? fit : slots;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Input canonicalisation: -0.0 is read as +0.0 so that coordinate order and
 * numeric comparison agree.  Returns the number of non-finite values.       */
/* ------------------------------------------------------------------------ */
int64_t oracle_canonicalise(float* pts, int64_t n_values) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n_values; i++) {
    if (!isfinite(pts[i])) bad++;
    if (pts[i] == 0.0f) pts[i] = 0.0f;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Tree fill: Sec. 2.2 "Tree ordering" + Sec. 2.3 (left-balanced k-d tree).
 * build(j, S): split dimension = widest FP32 bounding-box extent of S (ties
 * to the lowest dimension) or level mod 3; sort S by (x[dim], input index);
 * node j receives the element whose rank equals the size of j's left
 * subtree; the smaller elements fill the left subtree, the larger the right.
 * inorder[j] is j's rank in the left-node-right traversal.                  */
/* ------------------------------------------------------------------------ */

static int key_less(const float* pts, int dim, int32_t a, int32_t b) {
  float xa = pts[3 * (int64_t)a + dim], xb = pts[3 * (int64_t)b + dim];
  if (xa < xb) return 1;
  if (xa > xb) return 0;
  return a < b;
}

static void merge_sort(int32_t* a, int32_t* tmp, int64_t n, const float* pts,
                       int dim) {
  if (n < 2) return;
  int64_t h = n / 2;
  merge_sort(a, tmp, h, pts, dim);
  merge_sort(a + h, tmp, n - h, pts, dim);
  int64_t i = 0, j = h, o = 0;
  while (i < h && j < n) tmp[o++] = key_less(pts, dim, a[j], a[i]) ? a[j++] : a[i++];
  while (i < h) tmp[o++] = a[i++];
  while (j < n) tmp[o++] = a[j++];
  memcpy(a, tmp, (size_t)n * sizeof(int32_t));
}

static int build_node(const float* pts, int64_t N, int rule, int64_t j,
                      int32_t* S, int32_t* tmp, int64_t n, int64_t base,
                      int32_t* tree_point, uint8_t* split_dim,
                      int64_t* inorder) {
  if (n == 0) return (j >= N || oracle_subtree_size(j, N) == 0) ? ORC_OK : ORC_ERR;
  if (j >= N || oracle_subtree_size(j, N) != n) return ORC_ERR;
  int dim;
  if (rule == 0) {
    float lo[3], hi[3], ext[3];
    for (int d = 0; d < 3; d++) lo[d] = hi[d] = pts[3 * (int64_t)S[0] + d];
    for (int64_t s = 1; s < n; s++)
      for (int d = 0; d < 3; d++) {
        float x = pts[3 * (int64_t)S[s] + d];
        if (x < lo[d]) lo[d] = x;
        if (x > hi[d]) hi[d] = x;
      }
    for (int d = 0; d < 3; d++) ext[d] = hi[d] - lo[d]; /* FP32 subtraction */
    dim = 0;
    if (ext[1] > ext[dim]) dim = 1;
    if (ext[2] > ext[dim]) dim = 2;
  } else {
    dim = oracle_level(j) % 3;
  }
  merge_sort(S, tmp, n, pts, dim);
  int64_t m = oracle_subtree_size(oracle_left(j), N);
  tree_point[j] = S[m];
  split_dim[j] = (uint8_t)dim;
  inorder[j] = base + m;
  if (build_node(pts, N, rule, oracle_left(j), S, tmp, m, base, tree_point,
                 split_dim, inorder) != ORC_OK)
    return ORC_ERR;
  return build_node(pts, N, rule, oracle_right(j), S + m + 1, tmp, n - m - 1,
                    base + m + 1, tree_point, split_dim, inorder);
}

int oracle_tree_build(const float* pts, int64_t N, int rule,
                      int32_t* tree_point, uint8_t* split_dim,
                      int64_t* inorder) {
  if (N <= 0) return ORC_OK;
  int32_t* S = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  int32_t* tmp = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  if (!S || !tmp) { free(S); free(tmp); return ORC_ERR; }
  for (int64_t i = 0; i < N; i++) S[i] = (int32_t)i;
  int rc = build_node(pts, N, rule, 0, S, tmp, N, 0, tree_point, split_dim, inorder);
  free(S);
  free(tmp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Preceding k nearest neighbours: Sec. 2.1 (c(i) = k nearest preceding
 * points) and Sec. 2.2 (preceding points in tree order).  Key of candidate
 * i for query j: (d2(x_i, x_j), i), lexicographic, with the FP32 squared
 * distance dx = x_i - x_j (rounded), d2 = fma(dz,dz, fma(dy,dy, dx*dx)).   */
/* ------------------------------------------------------------------------ */

float oracle_d2(const float* a, const float* b) {
  float dx = a[0] - b[0];
  float dy = a[1] - b[1];
  float dz = a[2] - b[2];
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

typedef struct {
  int k, count;
  float* d;
  int32_t* i;
} cand_list;

static void cand_try(cand_list* c, float d, int32_t idx) {
  int k = c->k;
  if (c->count == k) {
    float wd = c->d[k - 1];
    int32_t wi = c->i[k - 1];
    if (!(d < wd || (d == wd && idx < wi))) return;
  } else {
    c->count++;
  }
  int p = c->count - 1;
  while (p > 0 && (c->d[p - 1] > d || (c->d[p - 1] == d && c->i[p - 1] > idx))) {
    c->d[p] = c->d[p - 1];
    c->i[p] = c->i[p - 1];
    p--;
  }
  c->d[p] = d;
  c->i[p] = idx;
}

/* Brute force: the definition.  Row j-n0 of nbr receives the tree indices of
 * c(j) nearest first; rows with fewer than k predecessors are padded with -1. */
static void knn_brute_one(const float* pts, const int32_t* tree_point, int64_t j, int k,
                          float* d, int32_t* ix, int32_t* out) {
  cand_list c = {k, 0, d, ix};
  const float* q = pts + 3 * (int64_t)tree_point[j];
  for (int64_t i = 0; i < j; i++)
    cand_try(&c, oracle_d2(pts + 3 * (int64_t)tree_point[i], q), (int32_t)i);
  for (int a = 0; a < k; a++) out[a] = a < c.count ? c.i[a] : -1;
}

int oracle_knn_brute(const float* pts, const int32_t* tree_point, int64_t N,
                     int k, int64_t n0, int32_t* nbr) {
  float* d = (float*)malloc((size_t)k * sizeof(float));
  int32_t* ix = (int32_t*)malloc((size_t)k * sizeof(int32_t));
  if (!d || !ix) { free(d); free(ix); return ORC_ERR; }
  for (int64_t j = n0; j < N; j++) knn_brute_one(pts, tree_point, j, k, d, ix, nbr + (j - n0) * k);
  free(d);
  free(ix);
  return ORC_OK;
}

/* The same definition for a list of tree indices js[0..n_js) only (sampled
 * checks of large graphs); row r of nbr receives c(js[r]). */
int oracle_knn_brute_some(const float* pts, const int32_t* tree_point, const int64_t* js,
                          int64_t n_js, int k, int32_t* nbr) {
  float* d = (float*)malloc((size_t)k * sizeof(float));
  int32_t* ix = (int32_t*)malloc((size_t)k * sizeof(int32_t));
  if (!d || !ix) { free(d); free(ix); return ORC_ERR; }
  for (int64_t r = 0; r < n_js; r++) knn_brute_one(pts, tree_point, js[r], k, d, ix, nbr + r * k);
  free(d);
  free(ix);
  return ORC_OK;
}

/* Sequential search of the prefix tree {0..j-1} (Sec. 2.2: every prefix of
 * the order is a valid tree).  A far subtree is skipped only when the FP32
 * square of the plane distance exceeds the current k-th key distance; every
 * point beyond the plane has an FP32 key distance at least that large
 * (rounding is monotone), so the result equals the brute force. */
typedef struct {
  const float* pts;
  const int32_t* tree_point;
  const uint8_t* split_dim;
  int64_t limit;
  const float* q;
  cand_list* c;
} knn_ctx;

static void knn_visit(knn_ctx* x, int64_t node) {
  if (node >= x->limit) return;
  const float* p = x->pts + 3 * (int64_t)x->tree_point[node];
  cand_try(x->c, oracle_d2(p, x->q), (int32_t)node);
  int dim = x->split_dim[node];
  float diff = x->q[dim] - p[dim];
  int64_t near_child = (x->q[dim] < p[dim]) ? oracle_left(node) : oracle_right(node);
  int64_t far_child = (x->q[dim] < p[dim]) ? oracle_right(node) : oracle_left(node);
  knn_visit(x, near_child);
  float plane = diff * diff;
  float worst = (x->c->count == x->c->k) ? x->c->d[x->c->k - 1] : INFINITY;
  if (!(plane > worst)) knn_visit(x, far_child);
}

int oracle_knn_tree(const float* pts, const int32_t* tree_point,
                    const uint8_t* split_dim, int64_t N, int k, int64_t n0,
                    int32_t* nbr) {
  float* d = (float*)malloc((size_t)k * sizeof(float));
  int32_t* ix = (int32_t*)malloc((size_t)k * sizeof(int32_t));
  if (!d || !ix) { free(d); free(ix); return ORC_ERR; }
  for (int64_t j = n0; j < N; j++) {
    cand_list c = {k, 0, d, ix};
    knn_ctx x = {pts, tree_point, split_dim, j, pts + 3 * (int64_t)tree_point[j], &c};
    knn_visit(&x, 0);
    for (int a = 0; a < k; a++) nbr[(j - n0) * k + a] = a < c.count ? c.i[a] : -1;
  }
  free(d);
  free(ix);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Depth and graph order: Sec. 2.2 "Batch construction".  d_j = 0 for the
 * dense block j < n0, else d_j = 1 + max over c(j), in tree order.          */
/* ------------------------------------------------------------------------ */
int oracle_depth(const int32_t* nbr_tree, int64_t N, int k, int64_t n0,
                 int32_t* depth) {
  for (int64_t j = 0; j < N && j < n0; j++) depth[j] = 0;
  for (int64_t j = n0; j < N; j++) {
    int32_t m = 0;
    for (int a = 0; a < k; a++) {
      int32_t i = nbr_tree[(j - n0) * k + a];
      if (i < 0) continue;
      if (i >= j) return ORC_ERR;
      if (depth[i] > m) m = depth[i];
    }
    depth[j] = 1 + m;
  }
  return ORC_OK;
}

/* Positions: stable sort of the tree indices by (depth, in-order rank).
 * Reading: the paper only asks for a depth-sorted order; within a depth the
 * k-d in-order rank is used (any order gives the same conditioning).
 * level_offsets has max_depth+2 entries. */
int oracle_order(const int32_t* depth, const int64_t* inorder, int64_t N,
                 int32_t max_depth, int32_t* tree_of_pos, int32_t* pos_of_tree,
                 int64_t* level_offsets) {
  if (N <= 0 || max_depth < 0) return ORC_ERR;
  int32_t* by_rank = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  if (!by_rank) return ORC_ERR;
  for (int64_t j = 0; j < N; j++) {
    if (inorder[j] < 0 || inorder[j] >= N) { free(by_rank); return ORC_ERR; }
    by_rank[inorder[j]] = (int32_t)j;
  }
  for (int32_t l = 0; l <= max_depth + 1; l++) level_offsets[l] = 0;
  for (int64_t j = 0; j < N; j++) level_offsets[depth[j] + 1]++;
  for (int32_t l = 0; l <= max_depth; l++) level_offsets[l + 1] += level_offsets[l];
  int64_t* fill = (int64_t*)malloc((size_t)(max_depth + 1) * sizeof(int64_t));
  if (!fill) { free(by_rank); return ORC_ERR; }
  for (int32_t l = 0; l <= max_depth; l++) fill[l] = level_offsets[l];
  for (int64_t r = 0; r < N; r++) {
    int32_t j = by_rank[r];
    int64_t pos = fill[depth[j]]++;
    tree_of_pos[pos] = j;
    pos_of_tree[j] = (int32_t)pos;
  }
  free(fill);
  free(by_rank);
  return ORC_OK;
}

/* Neighbour lists relabelled from tree indices to positions, key order kept. */
int oracle_relabel(const int32_t* nbr_tree, const int32_t* tree_of_pos,
                   const int32_t* pos_of_tree, int64_t N, int k, int64_t n0,
                   int32_t* nbr_pos) {
  for (int64_t pos = n0; pos < N; pos++) {
    int64_t j = tree_of_pos[pos];
    if (j < n0) return ORC_ERR;
    for (int a = 0; a < k; a++) {
      int32_t t = nbr_tree[(j - n0) * k + a];
      nbr_pos[(pos - n0) * k + a] = t < 0 ? -1 : pos_of_tree[t];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Covariance kappa(r) (Sec. 2.1, stationary kernel) in FP64, and its
 * derivatives with respect to the lengthscale and the variance.             */
/* ------------------------------------------------------------------------ */
double oracle_kappa(int type, double s2, double ell, double r) {
  switch (type) {
    case 0: return s2 * exp(-r / ell);
    case 1: { double a = sqrt(3.0) * r / ell; return s2 * (1.0 + a) * exp(-a); }
    case 2: { double a = sqrt(5.0) * r / ell; return s2 * (1.0 + a + a * a / 3.0) * exp(-a); }
    case 3: return s2 * exp(-r * r / (2.0 * ell * ell));
  }
  return NAN;
}

double oracle_dkappa_dell(int type, double s2, double ell, double r) {
  switch (type) {
    case 0: return s2 * exp(-r / ell) * r / (ell * ell);
    case 1: { double a = sqrt(3.0) * r / ell; return s2 * a * a * exp(-a) / ell; }
    case 2: { double a = sqrt(5.0) * r / ell; return s2 * a * a * (1.0 + a) * exp(-a) / (3.0 * ell); }
    case 3: return s2 * exp(-r * r / (2.0 * ell * ell)) * r * r / (ell * ell * ell);
  }
  return NAN;
}

static double dist64(const float* a, const float* b) {
  double dx = (double)a[0] - (double)b[0];
  double dy = (double)a[1] - (double)b[1];
  double dz = (double)a[2] - (double)b[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Cholesky-Banachiewicz, row by row, in place on the lower triangle of the
 * n x n row-major matrix A (leading dimension lda).  Pivots below
 * ORC_PD_FLOOR * A_jj are raised to that value; returns how many were. */
static int chol_rows(double* A, int64_t n, int64_t lda) {
  int clamped = 0;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t j = 0; j <= i; j++) {
      double s = A[i * lda + j];
      for (int64_t m = 0; m < j; m++) s -= A[i * lda + m] * A[j * lda + m];
      if (i == j) {
        double floor_v = ORC_PD_FLOOR * A[i * lda + i];
        if (!(s > floor_v)) { s = floor_v; clamped++; }
        A[i * lda + i] = sqrt(s);
      } else {
        A[i * lda + j] = s / A[j * lda + j];
      }
    }
    for (int64_t j = i + 1; j < n; j++) A[i * lda + j] = 0.0;
  }
  return clamped;
}

/* Solve L y = r (forward) and L^T x = y (backward) for lower-triangular L. */
static void solve_lower(const double* L, int64_t n, int64_t lda, double* y) {
  for (int64_t i = 0; i < n; i++) {
    double s = y[i];
    for (int64_t m = 0; m < i; m++) s -= L[i * lda + m] * y[m];
    y[i] = s / L[i * lda + i];
  }
}

static void solve_upper_t(const double* L, int64_t n, int64_t lda, double* x) {
  for (int64_t i = n - 1; i >= 0; i--) {
    double s = x[i];
    for (int64_t m = i + 1; m < n; m++) s -= L[m * lda + i] * x[m];
    x[i] = s / L[i * lda + i];
  }
}

static int row_count(const int32_t* row, int k) {
  int c = 0;
  for (int a = 0; a < k; a++) if (row[a] >= 0) c++;
  return c;
}

/* ------------------------------------------------------------------------ */
/* Factor: Sec. 2.1 Eq. 2.  For position i >= n0 with c = c(i):
 *   K_cc[a][b] = kappa(|x_a - x_b|) + nugget [a == b],  K_ci, K_ii = kappa(0)
 *   + nugget;  L = chol(K_cc);  y = L^-1 K_ci;  b = L^-T y;
 *   sigma^2 = K_ii - y.y;  sigma = sqrt(sigma^2).
 * Dense block (the dense initial batch of Alg. 1): L0 = chol(K_00 + nugget I) over
 * positions 0..n0-1 and sigma_i = L0_ii.  logdet = 2 sum log sigma_i.
 * Distances are FP64 from the FP32 coordinates.                             */
/* ------------------------------------------------------------------------ */
/* One conditional (Sec. 2.1 Eq. 2) for point i of pts with neighbour list
 * row[0..k) (indices into pts, -1 for none): b (k entries, zero past the
 * list) and sigma.  K, y: k*k and k doubles of scratch.  Returns 1 when a
 * pivot or sigma^2 was floored. */
static int factor_row(const float* pts, int64_t i, const int32_t* row, int k, int type, double s2,
                      double ell, double nug, double* K, double* y, double* b, double* sigma) {
  double k0 = oracle_kappa(type, s2, ell, 0.0) + nug;
  int kc = row_count(row, k);
  const float* xi = pts + 3 * i;
  for (int a = 0; a < kc; a++) {
    for (int c = 0; c < kc; c++)
      K[a * kc + c] = (a == c) ? k0 : oracle_kappa(type, s2, ell, dist64(pts + 3 * (int64_t)row[a], pts + 3 * (int64_t)row[c]));
    y[a] = oracle_kappa(type, s2, ell, dist64(pts + 3 * (int64_t)row[a], xi));
  }
  int clamped = chol_rows(K, kc, kc);
  solve_lower(K, kc, kc, y);
  double s = k0;
  for (int a = 0; a < kc; a++) s -= y[a] * y[a];
  double floor_v = ORC_PD_FLOOR * k0;
  if (!(s > floor_v)) { s = floor_v; clamped++; }
  *sigma = sqrt(s);
  solve_upper_t(K, kc, kc, y);
  for (int a = 0; a < k; a++) b[a] = a < kc ? y[a] : 0.0;
  return clamped ? 1 : 0;
}

/* factor_row for the points idx[0..n) of pts (any order) with neighbour lists
 * nbr[r*k .. r*k+k) (indices into pts): sampled checks of large graphs. */
int oracle_factor_rows(const float* pts, const int64_t* idx, const int32_t* nbr, int64_t n, int k,
                       int type, double s2, double ell, double nug, double* b, double* sigma) {
  double* K = (double*)malloc((size_t)k * k * sizeof(double));
  double* y = (double*)malloc((size_t)k * sizeof(double));
  if (!K || !y) { free(K); free(y); return ORC_ERR; }
  for (int64_t r = 0; r < n; r++)
    factor_row(pts, idx[r], nbr + r * k, k, type, s2, ell, nug, K, y, b + r * k, sigma + r);
  free(K);
  free(y);
  return ORC_OK;
}

int oracle_factor(const float* pts_pos, const int32_t* nbr_pos, int64_t N,
                  int k, int64_t n0, int type, double s2, double ell,
                  double nug, double* b, double* sigma, double* L0,
                  double* logdet, int64_t* n_not_pd) {
  int64_t bad = 0;
  double k0 = oracle_kappa(type, s2, ell, 0.0) + nug;
  /* dense block */
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n0; j++)
      L0[i * n0 + j] = (i == j) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * i, pts_pos + 3 * j));
  bad += chol_rows(L0, n0, n0); /* one pivot per row: clamped pivots = rows */
  for (int64_t i = 0; i < n0; i++) sigma[i] = L0[i * n0 + i];
  double* K = (double*)malloc((size_t)k * k * sizeof(double));
  double* y = (double*)malloc((size_t)k * sizeof(double));
  if (!K || !y) { free(K); free(y); return ORC_ERR; }
  for (int64_t i = n0; i < N; i++)
    bad += factor_row(pts_pos, i, nbr_pos + (i - n0) * k, k, type, s2, ell, nug, K, y,
                      b + (i - n0) * k, sigma + i);
  free(K);
  free(y);
  double ld = 0.0;
  for (int64_t i = 0; i < N; i++) ld += log(sigma[i]);
  *logdet = 2.0 * ld;
  if (n_not_pd) *n_not_pd = bad;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sweeps: Alg. 1 (generate) and its inverse (whiten), Sec. 3.               */
/* ------------------------------------------------------------------------ */
void oracle_generate(const double* b, const double* sigma, const double* L0,
                     const int32_t* nbr_pos, int64_t N, int k, int64_t n0,
                     const double* xi, double* v) {
  for (int64_t i = 0; i < n0; i++) {
    double s = 0.0;
    for (int64_t m = 0; m <= i; m++) s += L0[i * n0 + m] * xi[m];
    v[i] = s;
  }
  for (int64_t i = n0; i < N; i++) {
    double s = 0.0;
    for (int a = 0; a < k; a++) {
      int32_t c = nbr_pos[(i - n0) * k + a];
      if (c >= 0) s += b[(i - n0) * k + a] * v[c];
    }
    v[i] = s + sigma[i] * xi[i];
  }
}

void oracle_whiten(const double* b, const double* sigma, const double* L0,
                   const int32_t* nbr_pos, int64_t N, int k, int64_t n0,
                   const double* v, double* xi) {
  for (int64_t i = 0; i < n0; i++) {
    double s = v[i];
    for (int64_t m = 0; m < i; m++) s -= L0[i * n0 + m] * xi[m];
    xi[i] = s / L0[i * n0 + i];
  }
  for (int64_t i = n0; i < N; i++) {
    double s = v[i];
    for (int a = 0; a < k; a++) {
      int32_t c = nbr_pos[(i - n0) * k + a];
      if (c >= 0) s -= b[(i - n0) * k + a] * v[c];
    }
    xi[i] = s / sigma[i];
  }
}

double oracle_logdet(const double* sigma, int64_t N) {
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) s += log(sigma[i]);
  return 2.0 * s;
}

/* Same sum over FP32 sigma values promoted to FP64. */
double oracle_logdet_f32(const float* sigma, int64_t N) {
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) s += log((double)sigma[i]);
  return 2.0 * s;
}

/* Alg. 1 taken literally: per point, the (k+1)x(k+1) joint covariance of
 * [c(i), i], its Cholesky factor L, and
 *   v_i = L[k][0:k] . (L[0:k][0:k]^-1 v_c) + L[k][k] xi_i.
 * Positions are visited in increasing order, which respects the batches. */
int oracle_generate_alg1(const float* pts_pos, const int32_t* nbr_pos,
                         int64_t N, int k, int64_t n0, int type, double s2,
                         double ell, double nug, const double* xi, double* v) {
  double k0 = oracle_kappa(type, s2, ell, 0.0) + nug;
  if (n0 > 0) {
    double* A = (double*)malloc((size_t)n0 * n0 * sizeof(double));
    if (!A) return ORC_ERR;
    for (int64_t i = 0; i < n0; i++)
      for (int64_t j = 0; j < n0; j++)
        A[i * n0 + j] = (i == j) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * i, pts_pos + 3 * j));
    chol_rows(A, n0, n0);
    for (int64_t i = 0; i < n0; i++) {
      double s = 0.0;
      for (int64_t m = 0; m <= i; m++) s += A[i * n0 + m] * xi[m];
      v[i] = s;
    }
    free(A);
  }
  int64_t m1 = (int64_t)k + 1;
  double* J = (double*)malloc((size_t)m1 * m1 * sizeof(double));
  double* w = (double*)malloc((size_t)m1 * sizeof(double));
  int64_t* idx = (int64_t*)malloc((size_t)m1 * sizeof(int64_t));
  if (!J || !w || !idx) { free(J); free(w); free(idx); return ORC_ERR; }
  for (int64_t i = n0; i < N; i++) {
    const int32_t* row = nbr_pos + (i - n0) * k;
    int kc = row_count(row, k);
    for (int a = 0; a < kc; a++) idx[a] = row[a];
    idx[kc] = i;
    int64_t n = kc + 1;
    for (int64_t a = 0; a < n; a++)
      for (int64_t c = 0; c < n; c++)
        J[a * n + c] = (a == c) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * idx[a], pts_pos + 3 * idx[c]));
    chol_rows(J, n, n);
    for (int a = 0; a < kc; a++) w[a] = v[idx[a]];
    solve_lower(J, kc, n, w);
    double s = 0.0;
    for (int a = 0; a < kc; a++) s += J[kc * n + a] * w[a];
    v[i] = s + J[kc * n + kc] * xi[i];
  }
  free(J);
  free(w);
  free(idx);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense rows in conditional form (Sec. 2.1: with c(i) = all preceding points
 * the approximation is the dense Cholesky factorisation).  Row i < n0 of the
 * strictly lower n0 x n0 matrix bd holds b_i = K_<i^-1 K_<i,i, obtained from
 * L0 as L0[:i,:i]^-T L0[i,:i]; sigma_i = L0_ii.                             */
/* ------------------------------------------------------------------------ */
int oracle_dense_rows(const double* L0, int64_t n0, double* bd) {
  double* t = (double*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(double));
  if (!t) return ORC_ERR;
  for (int64_t i = 0; i < n0; i++) {
    for (int64_t m = 0; m < i; m++) t[m] = L0[i * n0 + m];
    solve_upper_t(L0, i, n0, t);
    for (int64_t m = 0; m < n0; m++) bd[i * n0 + m] = m < i ? t[m] : 0.0;
  }
  free(t);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoints (Sec. 2.3: derivatives of the conditioning steps).  With every
 * row written as v_i = b_i . v_c(i) + sigma_i xi_i (dense rows with
 * c(i) = {0..i-1}, weights bd), the vector-Jacobian products are:
 *  whiten  (xi_i = (v_i - b_i.v_c)/sigma_i), w_i = xibar_i / sigma_i:
 *     vbar_i += w_i,  vbar_c -= w_i b_i,  bbar_i = -w_i v_c,
 *     sigbar_i = -w_i xi_i + 2 logdetbar / sigma_i
 *  generate: u_j = vbar_j + sum over rows i with j in c(i) of b_ij u_i, taken
 *     in decreasing position order; xibar_i = sigma_i u_i, bbar_i = u_i v_c,
 *     sigbar_i = u_i xi_i.                                                 */
/* ------------------------------------------------------------------------ */
void oracle_whiten_vjp(const double* b, const double* bd, const double* sigma,
                       const int32_t* nbr_pos, int64_t N, int k, int64_t n0,
                       const double* v, const double* xi, const double* xibar,
                       double logdetbar, double* vbar, double* bbar,
                       double* bdbar, double* sigbar) {
  for (int64_t i = 0; i < N; i++) vbar[i] = 0.0;
  for (int64_t i = 0; i < N; i++) {
    double w = xibar[i] / sigma[i];
    vbar[i] += w;
    sigbar[i] = -w * xi[i] + 2.0 * logdetbar / sigma[i];
    if (i < n0) {
      for (int64_t m = 0; m < n0; m++) {
        bdbar[i * n0 + m] = m < i ? -w * v[m] : 0.0;
        if (m < i) vbar[m] -= w * bd[i * n0 + m];
      }
    } else {
      for (int a = 0; a < k; a++) {
        int32_t c = nbr_pos[(i - n0) * k + a];
        bbar[(i - n0) * k + a] = c >= 0 ? -w * v[c] : 0.0;
        if (c >= 0) vbar[c] -= w * b[(i - n0) * k + a];
      }
    }
  }
}

void oracle_generate_vjp(const double* b, const double* bd,
                         const double* sigma, const int32_t* nbr_pos,
                         int64_t N, int k, int64_t n0, const double* xi,
                         const double* v, const double* vbar, double* xibar,
                         double* bbar, double* bdbar, double* sigbar) {
  double* u = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
  if (!u) return;
  for (int64_t i = 0; i < N; i++) u[i] = vbar[i];
  for (int64_t i = N - 1; i >= 0; i--) {
    /* u[i] is final here: every row that reads v_i has a larger position */
    xibar[i] = sigma[i] * u[i];
    sigbar[i] = u[i] * xi[i];
    if (i < n0) {
      for (int64_t m = 0; m < n0; m++) {
        bdbar[i * n0 + m] = m < i ? u[i] * v[m] : 0.0;
        if (m < i) u[m] += bd[i * n0 + m] * u[i];
      }
    } else {
      for (int a = 0; a < k; a++) {
        int32_t c = nbr_pos[(i - n0) * k + a];
        bbar[(i - n0) * k + a] = c >= 0 ? u[i] * v[c] : 0.0;
        if (c >= 0) u[c] += b[(i - n0) * k + a] * u[i];
      }
    }
  }
  free(u);
}

/* Factor backward, per row, from b = K_cc^-1 K_ci and s = sigma^2 =
 * K_ii - K_ic b:  sbar = sigbar / (2 sigma),  g = K_cc^-1 bbar,
 *   Kbar_cc[a][c] = -g_a b_c + sbar b_a b_c,  Kbar_ci = g - 2 sbar b,
 *   Kbar_ii = sbar,
 * then thetabar += sum Kbar * dK/dtheta with theta = (lengthscale, sigma2,
 * nugget).  Dense rows use c(i) = {0..i-1}; chol(K_<i) is the leading block
 * of L0.  Everything is recomputed in FP64. */
int oracle_factor_backward(const float* pts_pos, const int32_t* nbr_pos,
                           int64_t N, int k, int64_t n0, int type, double s2,
                           double ell, double nug, const double* bbar,
                           const double* bdbar, const double* sigbar,
                           double* thetabar) {
  double b_s = 0, b_l = 0, b_n = 0; /* d/dsigma2, d/dlengthscale, d/dnugget */
  double k0 = oracle_kappa(type, s2, ell, 0.0) + nug;
  int64_t kmax = (k > n0) ? k : n0;
  double* L = (double*)malloc((size_t)(kmax > 0 ? kmax * kmax : 1) * sizeof(double));
  double* L0 = (double*)malloc((size_t)(n0 > 0 ? n0 * n0 : 1) * sizeof(double));
  double* bb = (double*)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(double));
  double* g = (double*)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(double));
  int64_t* idx = (int64_t*)malloc((size_t)(kmax + 1) * sizeof(int64_t));
  if (!L || !L0 || !bb || !g || !idx) { free(L); free(L0); free(bb); free(g); free(idx); return ORC_ERR; }
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n0; j++)
      L0[i * n0 + j] = (i == j) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * i, pts_pos + 3 * j));
  chol_rows(L0, n0, n0);
  for (int64_t i = 0; i < N; i++) {
    int64_t kc;
    const double* Lc;
    int64_t ldl;
    if (i < n0) {
      kc = i;
      for (int64_t m = 0; m < kc; m++) idx[m] = m;
      Lc = L0;
      ldl = n0;
      for (int64_t m = 0; m < kc; m++) g[m] = bdbar[i * n0 + m];
    } else {
      const int32_t* row = nbr_pos + (i - n0) * k;
      kc = row_count(row, k);
      for (int64_t a = 0; a < kc; a++) idx[a] = row[a];
      for (int64_t a = 0; a < kc; a++)
        for (int64_t c = 0; c < kc; c++)
          L[a * kc + c] = (a == c) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * idx[a], pts_pos + 3 * idx[c]));
      chol_rows(L, kc, kc);
      Lc = L;
      ldl = kc;
      for (int64_t a = 0; a < kc; a++) g[a] = bbar[(i - n0) * k + a];
    }
    /* b = K_cc^-1 K_ci and sigma^2, recomputed */
    for (int64_t a = 0; a < kc; a++)
      bb[a] = oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * idx[a], pts_pos + 3 * i));
    solve_lower(Lc, kc, ldl, bb);
    double s = k0;
    for (int64_t a = 0; a < kc; a++) s -= bb[a] * bb[a];
    double sigma = sqrt(s);
    solve_upper_t(Lc, kc, ldl, bb);
    double sbar = sigbar[i] / (2.0 * sigma);
    solve_lower(Lc, kc, ldl, g);
    solve_upper_t(Lc, kc, ldl, g); /* g = K_cc^-1 bbar */
    /* K_ii term */
    b_s += sbar * oracle_kappa(type, 1.0, ell, 0.0);
    b_l += sbar * oracle_dkappa_dell(type, s2, ell, 0.0);
    b_n += sbar;
    for (int64_t a = 0; a < kc; a++) {
      const float* xa = pts_pos + 3 * idx[a];
      double r = dist64(xa, pts_pos + 3 * i);
      double kb = g[a] - 2.0 * sbar * bb[a]; /* Kbar_ci[a] */
      b_s += kb * oracle_kappa(type, 1.0, ell, r);
      b_l += kb * oracle_dkappa_dell(type, s2, ell, r);
      for (int64_t c = 0; c < kc; c++) {
        double kbar = -g[a] * bb[c] + sbar * bb[a] * bb[c];
        double rac = (a == c) ? 0.0 : dist64(xa, pts_pos + 3 * idx[c]);
        b_s += kbar * oracle_kappa(type, 1.0, ell, rac);
        b_l += kbar * oracle_dkappa_dell(type, s2, ell, rac);
        if (a == c) b_n += kbar;
      }
    }
  }
  thetabar[0] += b_l;
  thetabar[1] += b_s;
  thetabar[2] += b_n;
  free(L);
  free(L0);
  free(bb);
  free(g);
  free(idx);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Derivative of the covariance with respect to the distance, divided by the
 * distance: h(r) = kappa'(r) / r, so that d kappa(|x_a - x_b|) / d x_a =
 * h(r) (x_a - x_b).  Matern-1/2 is not differentiable at r = 0; there the
 * direction x_a - x_b vanishes and h is taken as 0.                        */
/* ------------------------------------------------------------------------ */
double oracle_kappa_h(int type, double s2, double ell, double r) {
  switch (type) {
    case 0: return r > 0.0 ? -s2 * exp(-r / ell) / (ell * r) : 0.0;
    case 1: { double a = sqrt(3.0) * r / ell; return -3.0 * s2 * exp(-a) / (ell * ell); }
    case 2: {
      double a = sqrt(5.0) * r / ell;
      return -5.0 * s2 * (1.0 + a) * exp(-a) / (3.0 * ell * ell);
    }
    case 3: return -s2 * exp(-r * r / (2.0 * ell * ell)) / (ell * ell);
  }
  return NAN;
}

/* Gradient with respect to the point coordinates (graph order), with the
 * graph held fixed, from the same per-row cotangents as
 * oracle_factor_backward: every covariance entry K_ab = kappa(|x_a - x_b|)
 * of row i (neighbour-neighbour and neighbour-point) passes its cotangent
 * Kbar_ab on to both of its points:  xbar_a += Kbar_ab h(r) (x_a - x_b),
 * xbar_b -= Kbar_ab h(r) (x_a - x_b).  xbar is [N][3], accumulated (+=).   */
int oracle_factor_backward_points(const float* pts_pos, const int32_t* nbr_pos,
                                  int64_t N, int k, int64_t n0, int type, double s2,
                                  double ell, double nug, const double* bbar,
                                  const double* bdbar, const double* sigbar,
                                  double* xbar) {
  double k0 = oracle_kappa(type, s2, ell, 0.0) + nug;
  int64_t kmax = (k > n0) ? k : n0;
  double* L = (double*)malloc((size_t)(kmax > 0 ? kmax * kmax : 1) * sizeof(double));
  double* L0 = (double*)malloc((size_t)(n0 > 0 ? n0 * n0 : 1) * sizeof(double));
  double* bb = (double*)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(double));
  double* g = (double*)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(double));
  int64_t* idx = (int64_t*)malloc((size_t)(kmax + 1) * sizeof(int64_t));
  if (!L || !L0 || !bb || !g || !idx) { free(L); free(L0); free(bb); free(g); free(idx); return ORC_ERR; }
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n0; j++)
      L0[i * n0 + j] = (i == j) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * i, pts_pos + 3 * j));
  chol_rows(L0, n0, n0);
  for (int64_t i = 0; i < N; i++) {
    int64_t kc;
    const double* Lc;
    int64_t ldl;
    if (i < n0) {
      kc = i;
      for (int64_t m = 0; m < kc; m++) idx[m] = m;
      Lc = L0;
      ldl = n0;
      for (int64_t m = 0; m < kc; m++) g[m] = bdbar[i * n0 + m];
    } else {
      const int32_t* row = nbr_pos + (i - n0) * k;
      kc = row_count(row, k);
      for (int64_t a = 0; a < kc; a++) idx[a] = row[a];
      for (int64_t a = 0; a < kc; a++)
        for (int64_t c = 0; c < kc; c++)
          L[a * kc + c] = (a == c) ? k0 : oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * idx[a], pts_pos + 3 * idx[c]));
      chol_rows(L, kc, kc);
      Lc = L;
      ldl = kc;
      for (int64_t a = 0; a < kc; a++) g[a] = bbar[(i - n0) * k + a];
    }
    for (int64_t a = 0; a < kc; a++)
      bb[a] = oracle_kappa(type, s2, ell, dist64(pts_pos + 3 * idx[a], pts_pos + 3 * i));
    solve_lower(Lc, kc, ldl, bb);
    double s = k0;
    for (int64_t a = 0; a < kc; a++) s -= bb[a] * bb[a];
    double sigma = sqrt(s);
    solve_upper_t(Lc, kc, ldl, bb);
    double sbar = sigbar[i] / (2.0 * sigma);
    solve_lower(Lc, kc, ldl, g);
    solve_upper_t(Lc, kc, ldl, g); /* g = K_cc^-1 bbar */
    const float* xi = pts_pos + 3 * i;
    for (int64_t a = 0; a < kc; a++) {
      const float* xa = pts_pos + 3 * idx[a];
      /* K_ci[a] = kappa(|x_a - x_i|), cotangent g_a - 2 sbar b_a */
      double w = (g[a] - 2.0 * sbar * bb[a]) * oracle_kappa_h(type, s2, ell, dist64(xa, xi));
      for (int d = 0; d < 3; d++) {
        double dd = (double)xa[d] - (double)xi[d];
        xbar[3 * idx[a] + d] += w * dd;
        xbar[3 * i + d] -= w * dd;
      }
      for (int64_t c = 0; c < kc; c++) {
        if (c == a) continue; /* kappa(0) + nugget does not move */
        const float* xc = pts_pos + 3 * idx[c];
        double kbar = -g[a] * bb[c] + sbar * bb[a] * bb[c];
        double wc = kbar * oracle_kappa_h(type, s2, ell, dist64(xa, xc));
        for (int d = 0; d < 3; d++) {
          double dd = (double)xa[d] - (double)xc[d];
          xbar[3 * idx[a] + d] += wc * dd;
          xbar[3 * idx[c] + d] -= wc * dd;
        }
      }
    }
  }
  free(L);
  free(L0);
  free(bb);
  free(g);
  free(idx);
  return ORC_OK;
}
