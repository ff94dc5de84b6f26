"""The any-size graph checks of tests/fullsize.py, pinned on CPU: they accept
the oracle's graphs, agree with the oracle's FP32 key and brute force, and
reject planted mistakes."""
import numpy as np
import pytest

import oracle
import workloads
from fullsize import (check_depth_and_order, check_tree, inorder_rank_of, inorder_ranks, key_f32,
                      knn_sample, subtree_size_of, subtree_sizes)


def test_key_matches_oracle_fp32_key():
    rng = np.random.default_rng(5)
    for _ in range(40):
        q = (rng.standard_normal(3) * 10.0 ** rng.integers(-4, 3)).astype(np.float32)
        a = (q + rng.standard_normal((500, 3)) * 10.0 ** rng.integers(-7, 2, size=(500, 1))
             ).astype(np.float32)
        got = key_f32(a, q)
        want = np.array([oracle.d2(x, q) for x in a], np.float32)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("kind", ["uniform", "grid", "dups"])
def test_knn_sample_equals_oracle_brute_force(kind):
    N, k, n0 = 700, 6, 8
    rng = np.random.default_rng(6)
    if kind == "uniform":
        pts = workloads.uniform_cube(N, 3)
    elif kind == "grid":
        pts = rng.integers(0, 4, size=(N, 3)).astype(np.float32) * np.float32(0.3)
    else:
        base = workloads.unit_gaussian(N // 2, 4)
        pts = np.concatenate([base, base])
    pts = oracle.canonicalise(pts)
    tp, sd, io = oracle.tree_build(pts)
    want = oracle.knn_brute(pts, tp, k, n0)
    X = pts[tp]
    for j in list(range(n0, n0 + 20)) + list(range(N - 20, N)):
        assert knn_sample(X, j, k).tolist() == want[j - n0].tolist()
    js = np.array([n0, 100, N - 1], np.int64)
    assert np.array_equal(oracle.knn_brute_some(pts, tp, js, k), want[js - n0])


@pytest.mark.parametrize("kind", ["uniform", "gaussian", "ldr", "blobs"])
def test_tree_checks_accept_oracle_trees_and_reject_mistakes(kind):
    N = 3001
    pts = oracle.canonicalise(workloads.cloud(kind, N, 12))
    tp, sd, io = oracle.tree_build(pts)
    check_tree(pts, tp, sd)
    assert np.array_equal(inorder_ranks(N), io)
    assert np.array_equal(subtree_sizes(N), [oracle.subtree_size(j, N) for j in range(N)])
    bad = tp.copy()
    bad[[5, 9]] = bad[[9, 5]]
    with pytest.raises(AssertionError):
        check_tree(pts, bad, sd)
    bad_sd = sd.copy()
    bad_sd[0] = (bad_sd[0] + 1) % 3
    with pytest.raises(AssertionError):
        check_tree(pts, tp, bad_sd)


def test_depth_order_checks_accept_oracle_graph_and_reject_mistakes():
    pts = workloads.unit_gaussian(2500, 13)
    g = oracle.build_graph(pts, 8, 64)
    args = (g["nbr_tree"], g["depth"], g["inorder"], g["tree_point"], g["order"],
            g["level_offsets"], g["nbr_pos"], 64)
    check_depth_and_order(*args)
    d = g["depth"].copy()
    d[-1] += 1
    with pytest.raises(AssertionError):
        check_depth_and_order(args[0], d, *args[2:])
    nb = g["nbr_pos"].copy()
    nb[3, [0, 1]] = nb[3, [1, 0]]
    with pytest.raises(AssertionError):
        check_depth_and_order(*args[:6], nb, 64)


def test_factor_rows_equal_oracle_factor():
    pts = workloads.uniform_cube(1500, 14)
    g = oracle.build_graph(pts, 8, 64)
    K = oracle.Kernel(1, 1.0, 0.1, 1e-6)
    fo = oracle.factor(g["pts_pos"], g["nbr_pos"], 8, 64, K)
    rows = np.array([64, 65, 700, 1499], np.int64)
    b, s = oracle.factor_rows(g["pts_pos"], rows, g["nbr_pos"][rows - 64], K)
    assert np.array_equal(b, fo["b"][rows - 64]) and np.array_equal(s, fo["sigma"][rows])


@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 1000, 4097])
def test_closed_form_sizes_and_ranks(N):
    nodes = np.arange(N)
    assert np.array_equal(subtree_size_of(nodes, N), [oracle.subtree_size(j, N) for j in range(N)])
    assert np.array_equal(inorder_rank_of(nodes, N), inorder_ranks(N))
    if N > 1:
        _, _, io = oracle.tree_build(oracle.canonicalise(workloads.uniform_cube(N, 15)))
        assert np.array_equal(inorder_ranks(N), io)
