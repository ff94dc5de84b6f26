"""Pins of the oracle's tree layout and tree build (Sec. 2.2) against facts the
paper states and brute-force definitions -- no CUDA involved."""
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _heap_children(i):
    return 2 * i + 1, 2 * i + 2


def _bitrev(p, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (p & 1)
        p >>= 1
    return r


def test_golden_bitreversal_level3():
    """Sec. 2.2: with full levels the order is a per-level bit reversal."""
    rows = np.loadtxt(os.path.join(GOLDEN, "bitrev_level3_N15.txt"), dtype=int)
    # walk the bit-reversed tree (children from the oracle) and the standard
    # heap tree in lockstep from the root; record where each level-3 node sits
    pos_std = {}

    def walk(j, h):
        pos_std[j] = h
        if oracle.left(j) < 15:
            a, b = _heap_children(h)
            walk(oracle.left(j), a)
            walk(oracle.right(j), b)

    walk(0, 0)
    for p, want in rows:
        j = 7 + p
        assert pos_std[j] - 7 == want


@pytest.mark.parametrize("h", [1, 2, 3, 5, 8, 11])
def test_bitreversal_equivalence_full_levels(h):
    """Every full level l of the bit-reversed tree equals the standard heap
    level permuted by the l-bit reversal (Sec. 2.2)."""
    N = (1 << h) - 1
    pos_std = {}

    def walk(j, s):
        pos_std[j] = s
        if oracle.left(j) < N:
            a, b = _heap_children(s)
            walk(oracle.left(j), a)
            walk(oracle.right(j), b)

    walk(0, 0)
    assert len(pos_std) == N
    for l in range(h):
        for p in range(1 << l):
            j = (1 << l) - 1 + p
            assert pos_std[j] - ((1 << l) - 1) == _bitrev(p, l)


def test_children_and_parent_consistency():
    """Children lie one level down, left children of a level come before all
    right children, and parent() inverts both (Sec. 2.2)."""
    for j in range(0, 5000):
        l = oracle.level(j)
        assert (1 << l) - 1 <= j < (1 << (l + 1)) - 1
        L, R = oracle.left(j), oracle.right(j)
        assert oracle.level(L) == l + 1 and oracle.level(R) == l + 1
        assert oracle.parent(L) == j and oracle.parent(R) == j
        # all left children of level l precede all right children
        assert L - ((1 << (l + 1)) - 1) < (1 << l) <= R - ((1 << (l + 1)) - 1)
    assert oracle.parent(0) == -1


@pytest.mark.parametrize("N", [1, 2, 3, 7, 10, 100, 257, 1000, 4097])
def test_prefix_is_tree_and_subtree_sizes(N):
    """Every prefix is a valid tree (parents precede children), and the
    closed-form subtree size equals an explicit count by recursion."""
    for j in range(1, N):
        assert oracle.parent(j) < j

    def count(j):
        if j >= N:
            return 0
        return 1 + count(oracle.left(j)) + count(oracle.right(j))

    for j in range(min(N, 300)):
        assert oracle.subtree_size(j, N) == count(j)
    assert oracle.subtree_size(0, N) == N


def _subtree_nodes(j, N):
    out, stack = [], [j]
    while stack:
        x = stack.pop()
        if x < N:
            out.append(x)
            stack.append(oracle.left(x))
            stack.append(oracle.right(x))
    return out


def _inorder(N):
    rank = {}

    def rec(j, base):
        if j >= N:
            return base
        base = rec(oracle.left(j), base)
        rank[j] = base
        return rec(oracle.right(j), base + 1)

    rec(0, 0)
    return np.array([rank[j] for j in range(N)])


CLOUDS = {
    "uniform": lambda n: workloads.uniform_cube(n, 11),
    "gaussian": lambda n: workloads.unit_gaussian(n, 12),
    "ldr": lambda n: workloads.ldr_cloud(n, 13),
    # heavy ties: integer grid with duplicates, and one constant axis
    "grid": lambda n: np.random.default_rng(14).integers(0, 4, size=(n, 3)).astype(np.float32),
    "flat": lambda n: np.c_[np.random.default_rng(15).random((n, 2)), np.zeros(n)].astype(np.float32),
}


@pytest.mark.parametrize("cloud", sorted(CLOUDS))
@pytest.mark.parametrize("rule", [0, 1])
def test_tree_build_invariants(cloud, rule):
    """k-d property with the (coordinate, input index) key, the split-dimension
    rule, the median rank and the in-order rank, each checked by brute force."""
    N = 777
    pts = oracle.canonicalise(CLOUDS[cloud](N))
    tp, sd, io = oracle.tree_build(pts, rule)
    assert sorted(tp.tolist()) == list(range(N))
    assert np.array_equal(io, _inorder(N))
    for j in range(N):
        d = int(sd[j])
        sub = _subtree_nodes(j, N)
        ids = tp[sub]
        if rule == 0:
            ext = (pts[ids].max(axis=0) - pts[ids].min(axis=0)).astype(np.float32)
            assert d == int(np.argmax(ext))  # argmax takes the first maximum
        else:
            assert d == oracle.level(j) % 3
        key = (pts[tp[j], d], tp[j])
        for x in _subtree_nodes(oracle.left(j), N):
            assert (pts[tp[x], d], tp[x]) < key
        for x in _subtree_nodes(oracle.right(j), N):
            assert (pts[tp[x], d], tp[x]) > key


def test_canonicalise_negative_zero_and_nan():
    p = np.array([[-0.0, 1.0, 2.0]], np.float32)
    c = oracle.canonicalise(p)
    assert not np.signbit(c[0, 0])
    with pytest.raises(ValueError):
        oracle.canonicalise(np.array([[np.nan, 0, 0]], np.float32))
