"""Sharding by position range (paper_2606_11402_gb300/shard.py) on CPU: the
range split, the halo of a range, and the all-gather / all-reduce plumbing of
the sharded NLL and gradient with two gloo ranks.  Each rank's compute is a
CPU stand-in built from the FP64 oracle (the rows of its range, by masking
the oracle's per-row cotangents); the assembled result must equal the
oracle's whole-problem NLL and gradient."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2606_11402_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("N,n0,world", [(1000, 50, 2), (1000, 50, 3), (1000, 600, 4), (300, 300, 2),
                                        (10, 4, 8)])
def test_position_ranges(N, n0, world):
    r = shard.position_ranges(N, n0, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == N
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    assert all(b >= a for a, b in r)
    assert r[0][1] >= min(n0, N)
    assert all(b >= n0 for b, _ in r[1:])
    if n0 <= N // world:
        sizes = [e - b for b, e in r]
        assert max(sizes) - min(sizes) <= 1


def _graph(N=1500, k=8, n0=64, seed=3):
    pts = workloads.uniform_cube(N, seed)
    return oracle.build_graph(pts, k, n0)


def test_halo_positions_are_the_outside_neighbours():
    g = _graph()
    n0, N = g["n0"], g["N"]
    for p0, p1 in shard.position_ranges(N, n0, 3):
        h = shard.halo_positions(g["nbr_pos"], n0, p0, p1)
        lo, hi = max(p0, n0) - n0, max(p1 - n0, 0)
        want = sorted({int(c) for row in g["nbr_pos"][lo:hi] for c in row if not p0 <= c < p1})
        assert h.tolist() == want
        assert np.all(h < p1)  # neighbours always precede


class OracleRowOps:
    """CPU stand-in for one range: the oracle's whole-problem quantities,
    restricted to the rows [p0, p1) by masking the per-row cotangents."""

    def __init__(self, g, kern, p0, p1):
        self.g, self.kern, self.p0, self.p1 = g, kern, p0, p1
        self.fo = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
        self.own = np.zeros(g["N"], bool)
        self.own[p0:p1] = True

    def _xi(self, v):
        g = self.g
        return oracle.whiten(self.fo, g["nbr_pos"], g["k"], g["n0"], v)

    def nll(self, v_full):
        v = v_full.numpy().astype(np.float64)
        xi = self._xi(v)
        part = 0.5 * np.sum(xi[self.own] ** 2) + np.sum(np.log(self.fo["sigma"][self.own]))
        return torch.tensor([part], dtype=torch.float64)

    def nll_backward(self, v_full):
        g, fo = self.g, self.fo
        k, n0 = g["k"], g["n0"]
        v = v_full.numpy().astype(np.float64)
        xi = self._xi(v)
        xibar = np.where(self.own, xi, 0.0)
        a = oracle.whiten_vjp(fo, g["nbr_pos"], k, n0, v, xi, xibar, 0.5)
        sigbar = np.where(self.own, a["sigbar"], 0.0)
        bdbar = a["bdbar"] * self.own[:n0, None]
        tb = oracle.factor_backward(g["pts_pos"], g["nbr_pos"], k, n0, self.kern, a["bbar"], bdbar,
                                    sigbar)
        return torch.from_numpy(a["vbar"]), torch.from_numpy(tb)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    td.init_process_group("gloo", rank=rank, world_size=world)
    g = _graph()
    kern = oracle.Kernel(1, 1.0, 0.1, 1e-6)
    sh = shard.ShardedNLL(g["N"], g["n0"], lambda p0, p1: OracleRowOps(g, kern, p0, p1))
    v = workloads.white_noise(g["N"], 11).astype(np.float64)
    v_own = torch.from_numpy(v[sh.p0:sh.p1].copy())
    nll, vbar_own, tb = sh.value_and_grad(v_own)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), nll=nll.numpy(), vbar=vbar_own.numpy(),
             tb=tb.numpy(), p0=sh.p0, p1=sh.p1)
    td.barrier()
    td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_nll_and_gradient_gloo(tmp_path, world):
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    g = _graph()
    kern = oracle.Kernel(1, 1.0, 0.1, 1e-6)
    v = workloads.white_noise(g["N"], 11).astype(np.float64)
    fo = oracle.factor(g["pts_pos"], g["nbr_pos"], g["k"], g["n0"], kern)
    nll_or = oracle.nll(fo, g["nbr_pos"], g["k"], g["n0"], v)
    vbar_or, tb_or = oracle.nll_grad(g, kern, v)
    vbar = np.concatenate([r["vbar"] for r in res])
    assert [int(r["p0"]) for r in res] == [b for b, _ in shard.position_ranges(g["N"], g["n0"], world)]
    for r in res:
        assert abs(float(r["nll"][0]) - nll_or) <= 1e-12 * abs(nll_or)
        assert np.allclose(r["tb"], tb_or, rtol=1e-10, atol=0.0)
    assert np.allclose(vbar, vbar_or, rtol=1e-10, atol=1e-12 * np.abs(vbar_or).max())
