"""Checks of a graph that hold at any size, for workloads too large for the
oracle to rebuild in a test: the k-d tree invariants of Sec. 2.2 checked
node by node against every ancestor, the widest-extent split rule from
bottom-up bounding boxes, in-order ranks by recursion on the implicit tree,
the depth recurrence, the (depth, in-order) graph order, and exact preceding
kNN of sampled points from the FP32 key computed here in numpy (pinned
against the oracle's key in the CPU tests).  Nothing here calls the CUDA
library; the arrays come from the GPU's export and are only inspected."""
from __future__ import annotations

import numpy as np


def _fma_sq_f32(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Correctly rounded float32 fma(x, x, c) for float32 x, c.  x*x is exact
    in float64; the float64 sum's rounding error e comes from TwoSum; the only
    case where rounding the float64 sum to float32 differs from rounding the
    exact value is a sum that lands exactly on a float32 midpoint with e != 0,
    which is then resolved toward the sign of e."""
    p = x.astype(np.float64) * x.astype(np.float64)
    c64 = c.astype(np.float64)
    s = p + c64
    bb = s - p
    e = (p - (s - bb)) + (c64 - bb)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    below = np.where(r64 <= s, r, np.nextafter(r, np.float32(-np.inf)))
    above = np.nextafter(below, np.float32(np.inf))
    mid = (below.astype(np.float64) + above.astype(np.float64)) * 0.5
    tie = (s == mid) & (e != 0)
    return np.where(tie, np.where(e > 0, above, below), r).astype(np.float32)


def key_f32(a: np.ndarray, q: np.ndarray) -> np.ndarray:
    """FP32 kNN key of rows a [n, 3] against q [3]: dx = fl(a - q),
    t = fl(dx^2), t = fma(dy, dy, t), t = fma(dz, dz, t)."""
    a = np.asarray(a, np.float32)
    q = np.asarray(q, np.float32)
    d = a - q  # float32 subtraction, round to nearest
    t = (d[:, 0] * d[:, 0]).astype(np.float32)
    t = _fma_sq_f32(d[:, 1], t)
    return _fma_sq_f32(d[:, 2], t)


def knn_sample(X_tree: np.ndarray, j: int, k: int, chunk: int = 1 << 24) -> np.ndarray:
    """c(j): the k tree indices i < j with the smallest (key, i), scanning the
    candidates in chunks (each chunk keeps every entry tied with its k-th)."""
    q = X_tree[j]
    pool_k, pool_i = [], []
    for s in range(0, j, chunk):
        e = min(j, s + chunk)
        keys = key_f32(X_tree[s:e], q)
        m = min(k, e - s)
        kth = np.partition(keys, m - 1)[m - 1]
        cand = np.nonzero(keys <= kth)[0]
        pool_k.append(keys[cand])
        pool_i.append(cand + s)
    out = np.full(k, -1, np.int64)
    if pool_k:
        keys = np.concatenate(pool_k)
        idx = np.concatenate(pool_i)
        order = np.lexsort((idx, keys))[:k]
        out[:len(order)] = idx[order]
    return out


def _levels(N: int):
    l = 0
    while (1 << l) - 1 < N:
        yield l, (1 << l) - 1, min(N, (2 << l) - 1)
        l += 1


def subtree_sizes(N: int) -> np.ndarray:
    size = np.zeros(N + 1, np.int64)  # size[N] = 0 stands for "no child"
    lv = list(_levels(N))
    for l, a, b in reversed(lv):
        j = np.arange(a, b)
        lc = np.minimum(j + (1 << l), N)
        rc = np.minimum(j + (2 << l), N)
        size[a:b] = 1 + size[lc] + size[rc]
    return size[:N]


def inorder_ranks(N: int) -> np.ndarray:
    """In-order rank of every node of the implicit left-balanced tree."""
    size = np.append(subtree_sizes(N), 0)
    start = np.zeros(N, np.int64)  # first in-order rank of each subtree
    rank = np.zeros(N, np.int64)
    for l, a, b in _levels(N):
        j = np.arange(a, b)
        lc = j + (1 << l)
        rank[a:b] = start[a:b] + size[np.minimum(lc, N)]
        ok = lc < N
        start[lc[ok]] = start[j[ok]]
        rc = j + (2 << l)
        ok = rc < N
        start[rc[ok]] = rank[j[ok]] + 1
    return rank


def _node_level(nodes: np.ndarray) -> np.ndarray:
    nodes = np.asarray(nodes, np.int64)
    lvl = np.zeros_like(nodes)
    while True:
        up = ((np.int64(1) << (lvl + 1)) - 1) <= nodes
        if not up.any():
            return lvl
        lvl += up


def subtree_size_of(nodes: np.ndarray, N: int) -> np.ndarray:
    """Closed-form subtree sizes: the descendants of the node at (level l,
    position p) on level m sit at positions p + t 2^l, t < 2^(m - l)."""
    nodes = np.asarray(nodes, np.int64)
    out = np.zeros(len(nodes), np.int64)
    ok = nodes < N
    l = _node_level(np.where(ok, nodes, 0))
    p = nodes - ((np.int64(1) << l) - 1)
    m = l.copy()
    while True:
        first = (np.int64(1) << m) - 1 + p  # leftmost descendant on level m
        live = ok & (first < N)
        if not live.any():
            return out
        stride = np.int64(1) << l
        cnt = np.minimum((N - first + stride - 1) // stride, np.int64(1) << (m - l))
        out += np.where(live, cnt, 0)
        m += 1


def inorder_rank_of(nodes: np.ndarray, N: int) -> np.ndarray:
    """In-order rank of sampled nodes: the left subtree of the node plus, for
    every ancestor whose right subtree holds it, that ancestor and its left
    subtree."""
    nodes = np.asarray(nodes, np.int64)
    l = _node_level(nodes)
    p = nodes - ((np.int64(1) << l) - 1)
    rank = subtree_size_of(nodes + (np.int64(1) << l), N)
    for la in range(int(l.max()) if len(nodes) else 0):
        below = l > la
        a = (np.int64(1) << la) - 1 + (p % (np.int64(1) << la))
        right = (p % (np.int64(2) << la)) >= (np.int64(1) << la)
        add = subtree_size_of(a + (np.int64(1) << la), N) + 1
        rank += np.where(below & right, add, 0)
    return rank


def check_tree(pts: np.ndarray, tree_point: np.ndarray, split_dim: np.ndarray,
               nodes: np.ndarray | None = None, check_split_rule: bool = True):
    """Asserts the k-d invariants of the bit-reversed left-balanced tree:
    tree_point is a permutation; for every node u (or the given sample) and
    every ancestor a, u lies on a's left iff (x_u[s], idx_u) < (x_a[s], idx_a)
    with s = split_dim[a]; split_dim[j] is the widest FP32 extent of j's
    subtree (lowest dimension on ties)."""
    N = len(tree_point)
    tp = np.asarray(tree_point, np.int64)
    assert np.array_equal(np.sort(tp), np.arange(N))
    X = np.asarray(pts, np.float32)[tp]
    sd = np.asarray(split_dim, np.int64)
    if nodes is None:
        nodes = np.arange(N, dtype=np.int64)
    lvl = np.floor(np.log2(nodes + 1)).astype(np.int64)
    # exact integer level (log2 of float may be off by one at powers of two)
    lvl = np.where((1 << (lvl + 1)) - 1 <= nodes, lvl + 1, lvl)
    lvl = np.where((1 << lvl) - 1 > nodes, lvl - 1, lvl)
    pos = nodes - ((1 << lvl) - 1)
    for la in range(int(lvl.max()) if len(nodes) else 0):
        sel = lvl > la
        u = nodes[sel]
        pu = pos[sel]
        a = (1 << la) - 1 + (pu % (1 << la))
        right = (pu % (2 << la)) >= (1 << la)
        s = sd[a]
        xu, xa = X[u, s], X[a, s]
        less = (xu < xa) | ((xu == xa) & (tp[u] < tp[a]))
        assert np.array_equal(less, ~right), f"k-d order broken below level {la}"
    if check_split_rule:
        lo = X.copy()
        hi = X.copy()
        for l, a, b in reversed(list(_levels(N))):
            for off in (1 << l, 2 << l):
                j = np.arange(a, b)
                c = j + off
                ok = c < N
                lo[j[ok]] = np.minimum(lo[j[ok]], lo[c[ok]])
                hi[j[ok]] = np.maximum(hi[j[ok]], hi[c[ok]])
        ext = (hi - lo).astype(np.float32)
        assert np.array_equal(np.argmax(ext, axis=1), sd), "widest-extent split rule"


def check_depth_and_order(nbr_tree: np.ndarray, depth: np.ndarray, inorder: np.ndarray,
                          tree_point: np.ndarray, order: np.ndarray, level_offsets: np.ndarray,
                          nbr_pos: np.ndarray, n0: int):
    """d_j = 0 below n0, else 1 + max over c(j); positions sorted by
    (depth, in-order rank); level offsets; neighbours relabelled to
    positions in the same (nearest-first) order."""
    N = len(depth)
    d = np.asarray(depth, np.int64)
    assert np.all(d[:n0] == 0)
    if N > n0:
        nt = np.asarray(nbr_tree, np.int64)
        assert np.all(nt < np.arange(n0, N)[:, None])
        assert np.array_equal(d[n0:], 1 + d[nt].max(axis=1))
    key = d * N + np.asarray(inorder, np.int64)
    tree_of_pos = np.argsort(key, kind="stable")
    assert np.array_equal(np.asarray(order, np.int64), np.asarray(tree_point, np.int64)[tree_of_pos])
    lo = np.concatenate([[0], np.cumsum(np.bincount(d))])
    assert np.array_equal(np.asarray(level_offsets, np.int64), lo)
    if N > n0:
        pos_of_tree = np.empty(N, np.int64)
        pos_of_tree[tree_of_pos] = np.arange(N)
        rows = pos_of_tree[np.arange(n0, N)]
        want = np.empty((N - n0, nt.shape[1]), np.int64)
        want[rows - n0] = pos_of_tree[nt]
        assert np.array_equal(np.asarray(nbr_pos, np.int64), want)
