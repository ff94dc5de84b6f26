"""Pins of the oracle's preceding-kNN, depth and graph order (Sec. 2.1, 2.2)
against exact brute force and independent formulations."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads


def _round_f32(q: Fraction) -> np.float32:
    """Round an exact rational to the nearest float32, ties to even."""
    c = np.float32(float(q))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    best = None
    for x in cands:
        err = abs(Fraction(float(x)) - q)
        even = (np.array(x, np.float32).view(np.uint32) & 1) == 0
        key = (err, 0 if even else 1)
        if best is None or key < best[0]:
            best = (key, x)
    return np.float32(best[1])


def _exact_key(a, b):
    """FP32 key dx=fl(a-b), d2=fl(dz^2+fl(dy^2+fl(dx^2))) with every step an
    exactly rounded rational operation."""
    F = lambda x: Fraction(float(x))
    dx, dy, dz = (_round_f32(F(a[i]) - F(b[i])) for i in range(3))
    t = _round_f32(F(dx) * F(dx))
    t = _round_f32(F(dy) * F(dy) + F(t))
    return _round_f32(F(dz) * F(dz) + F(t))


def test_d2_matches_exact_rounding_and_is_symmetric():
    rng = np.random.default_rng(0)
    for _ in range(300):
        a = (rng.standard_normal(3) * 10.0 ** rng.integers(-4, 3)).astype(np.float32)
        b = (a + rng.standard_normal(3) * 10.0 ** rng.integers(-6, 1)).astype(np.float32)
        d = oracle.d2(a, b)
        assert d == _exact_key(a, b)
        assert d == oracle.d2(b, a)


@pytest.mark.parametrize("cloud", ["uniform", "grid", "dups"])
def test_knn_brute_equals_exact_rational_bruteforce(cloud):
    """The oracle's brute force equals a from-scratch rational-arithmetic
    brute force of the key (d2, tree index) on a tiny cloud."""
    N, k, n0 = 90, 5, 6
    rng = np.random.default_rng(1)
    if cloud == "uniform":
        pts = workloads.uniform_cube(N, 21)
    elif cloud == "grid":
        pts = rng.integers(0, 3, size=(N, 3)).astype(np.float32) * np.float32(0.1)
    else:
        base = workloads.uniform_cube(N // 3, 22)
        pts = np.concatenate([base, base, base])[:N]
    pts = oracle.canonicalise(pts)
    tp, sd, io = oracle.tree_build(pts)
    got = oracle.knn_brute(pts, tp, k, n0)
    for j in range(n0, N):
        keys = sorted((_exact_key(pts[tp[i]], pts[tp[j]]), i) for i in range(j))
        want = [i for _, i in keys[:k]]
        assert got[j - n0].tolist() == want


@pytest.mark.parametrize("cloud", ["uniform", "gaussian", "ldr", "grid", "blobs"])
@pytest.mark.parametrize("k", [1, 8, 16, 32])
def test_knn_tree_search_equals_bruteforce(cloud, k):
    """The pruned prefix-tree search returns exactly the brute-force lists."""
    N = 3000
    if cloud == "grid":
        pts = np.random.default_rng(2).integers(0, 6, size=(N, 3)).astype(np.float32)
    elif cloud == "blobs":
        pts = workloads.blobs(N, 23, n_blobs=20)
    else:
        pts = workloads.cloud(cloud, N, 24)
    pts = oracle.canonicalise(pts)
    n0 = max(k, 40)
    tp, sd, io = oracle.tree_build(pts)
    assert np.array_equal(oracle.knn_tree(pts, tp, sd, k, n0), oracle.knn_brute(pts, tp, k, n0))


def _depth_jacobi(nbr_tree, N, n0):
    """Sec. 2.3: apply the depth update to all points at once and iterate
    until nothing changes (independent of the oracle's sequential loop)."""
    d = np.zeros(N, np.int64)
    nb = nbr_tree.astype(np.int64)
    valid = nb >= 0
    while True:
        m = np.where(valid, d[np.where(valid, nb, 0)], -1).max(axis=1) if N > n0 else np.zeros(0)
        new = d.copy()
        new[n0:] = 1 + np.maximum(m, 0)
        if np.array_equal(new, d):
            return d
        d = new


@pytest.mark.parametrize("cloud", ["uniform", "gaussian", "ldr"])
def test_depth_and_order(cloud):
    N, k = 4096, 8
    g = oracle.build_graph(workloads.cloud(cloud, N, 25), k)
    n0 = g["n0"]
    dp = g["depth"]
    assert np.array_equal(dp, _depth_jacobi(g["nbr_tree"], N, n0))
    # order: a permutation sorted by (depth, in-order rank)
    top = g["tree_of_pos"]
    keys = list(zip(dp[top], g["inorder"][top]))
    assert keys == sorted(keys)
    assert sorted(top.tolist()) == list(range(N))
    lo = g["level_offsets"]
    assert lo[0] == 0 and lo[1] == n0 and lo[-1] == N
    lvl = np.repeat(np.arange(len(lo) - 1), np.diff(lo))
    assert np.array_equal(lvl, dp[top])
    # every neighbour sits in an earlier batch, and the relabelled list keeps
    # the tree-index list's entries in the same (nearest-first) order
    nbp = g["nbr_pos"]
    start_of_row = lo[lvl[n0:]]
    assert (nbp < start_of_row[:, None]).all()
    assert np.array_equal(top[nbp], g["nbr_tree"][top[n0:] - n0])


def _levels_for_order(pts, perm, k, n0):
    """Number of depth levels when generating in the order perm with
    k-nearest-preceding conditioning (numpy brute force, FP64 distances)."""
    x = pts[perm].astype(np.float64)
    N = len(perm)
    depth = np.zeros(N, np.int64)
    for j in range(n0, N):
        d = ((x[:j] - x[j]) ** 2).sum(axis=1)
        nb = np.argpartition(d, k - 1)[:k] if j > k else np.arange(j)
        depth[j] = 1 + depth[nb].max()
    return depth.max() + 1


def test_bitreversed_order_gives_fewer_batches():
    """Fig. 1 (centre), qualitatively: on a 3-D unit Gaussian cloud with k=16
    and n0=50 the GraphGP order needs the fewest batches, against the
    standard tree order, a random order and the x-sorted order."""
    N, k, n0 = 3000, 16, 50
    pts = oracle.canonicalise(workloads.unit_gaussian(N, 26))
    g = oracle.build_graph(pts, k, n0)
    ours = len(g["level_offsets"]) - 1
    # standard heap order of the same k-d tree: the node at heap position h
    heap = {}

    def walk(j, h):
        if j >= N:
            return
        heap[h] = j
        walk(oracle.left(j), 2 * h + 1)
        walk(oracle.right(j), 2 * h + 2)

    walk(0, 0)
    std_perm = g["tree_point"][[heap[h] for h in sorted(heap)]]
    rnd_perm = np.random.default_rng(3).permutation(N)
    x_perm = np.argsort(pts[:, 0], kind="stable")
    std, rnd, xs = (_levels_for_order(pts, p, k, n0) for p in (std_perm, rnd_perm, x_perm))
    # the same count through the numpy path, for the bit-reversed order itself
    assert _levels_for_order(pts, g["tree_point"], k, n0) == ours
    assert ours < min(std, rnd, xs)
    assert 1.5 * ours < std and 1.5 * ours < xs


def _tree_d(pts, d):
    """The tree fill of Sec. 2.2 written directly in d dimensions: widest FP32
    extent among the d coordinates (ties to the lowest), median by
    (coordinate, input index), node j takes the entry after its left subtree."""
    N = pts.shape[0]
    level = lambda j: (j + 1).bit_length() - 1
    left = lambda j: j + 2 ** level(j)
    right = lambda j: j + 2 ** (level(j) + 1)
    size = {}

    def sz(j):
        if j >= N:
            return 0
        if j not in size:
            size[j] = 1 + sz(left(j)) + sz(right(j))
        return size[j]

    tp = np.full(N, -1, np.int64)

    def fill(j, S):
        if j >= N:
            assert not S
            return
        ext = [np.float32(max(pts[i, c] for i in S)) - np.float32(min(pts[i, c] for i in S))
               for c in range(d)]
        dim = int(np.argmax(ext))  # first maximum: lowest dimension on ties
        S = sorted(S, key=lambda i: (pts[i, dim], i))
        m = sz(left(j))
        tp[j] = S[m]
        fill(left(j), S[:m])
        fill(right(j), S[m + 1:])

    fill(0, list(range(N)))
    return tp


def _exact_key_d(a, b, d):
    """FP32 key in d dimensions: dx = fl(a - b), t = fl(dx^2), then
    t = fl(dy^2 + t) for the second coordinate."""
    F = lambda x: Fraction(float(x))
    t = None
    for c in range(d):
        dc = _round_f32(F(a[c]) - F(b[c]))
        t = _round_f32(F(dc) * F(dc) + (F(t) if t is not None else 0))
    return t


@pytest.mark.parametrize("d", [1, 2])
def test_lower_dimensions_equal_zero_padded_points(d):
    """Points of dimension d < 3 are handled as 3-D points with zero extra
    coordinates: the padded tree and neighbour lists equal the d-dimensional
    definitions (with ties: coordinates on a coarse grid)."""
    N, k, n0 = 120, 4, 5
    rng = np.random.default_rng(30 + d)
    pts_d = (rng.integers(0, 40, size=(N, d)) * 0.05).astype(np.float32)
    padded = np.zeros((N, 3), np.float32)
    padded[:, :d] = pts_d
    g = oracle.build_graph(padded, k, n0)
    tp = _tree_d(pts_d, d)
    assert np.array_equal(g["tree_point"], tp)
    for j in range(n0, N):
        keys = sorted((_exact_key_d(pts_d[tp[i]], pts_d[tp[j]], d), i) for i in range(j))
        assert g["nbr_tree"][j - n0].tolist() == [i for _, i in keys[:k]]
