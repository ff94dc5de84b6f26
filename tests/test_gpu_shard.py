"""Position-range entry points on the GPU (graphgp_factor_rows,
graphgp_nll_rows, graphgp_nll_backward_rows): the ranges' parts add up to the
whole-graph factor, NLL and gradient, and the sharded NLL runs through
torch.distributed (NCCL, one rank) on them."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as td

import workloads
from gpu_util import np_, rel_norm, to_gpu
from paper_2606_11402_gb300 import shard

pytestmark = pytest.mark.gpu


def _setup(gg, N, k, kern, kind="gaussian"):
    pts = workloads.cloud(kind, N, 51)
    g = gg.build_graph(to_gpu(pts), k, n0=min(N, 128))
    K = gg.Kernel(*kern)
    f = gg.factor(g, K)
    v = gg.generate(g, f, to_gpu(workloads.white_noise(N, 52)))
    return g, K, f, v


@pytest.mark.parametrize("N,k,world,kern", [(20_011, 16, 2, (1, 1.0, 0.1, 1e-6)),
                                            (20_011, 8, 3, (3, 1.0, 0.05, 1e-4)),
                                            (9_000, 32, 2, (3, 1.0, 0.05, 1e-4)),
                                            (5_000, 48, 2, (0, 1.0, 0.1, 1e-4))])
def test_ranges_add_up_to_the_whole(gpu_lib, N, k, world, kern):
    g, K, f, v = _setup(gpu_lib, N, k, kern)
    b, sigma, _ = (np_(t) for t in f.export())
    ld = np_(gpu_lib.logdet(f))[0]
    nll = np_(gpu_lib.nll(g, f, v))[0]
    vbar, tb = (np_(t) for t in gpu_lib.nll_backward(g, f, v))
    parts, vb_sum, tb_sum, ld_sum = 0.0, np.zeros(N), np.zeros(3), 0.0
    n0 = g.n0
    for p0, p1 in shard.position_ranges(N, n0, world):
        fr = gpu_lib.factor_rows(g, K, p0, p1)
        br, sr, _ = (np_(t) for t in fr.export())
        lo, hi = max(p0, n0) - n0, max(p1 - n0, 0)
        # the range's rows are the whole factor's, bit for bit; the others zero
        assert np.array_equal(br[lo:hi].view(np.uint32), b[lo:hi].view(np.uint32))
        assert np.array_equal(sr[p0:p1].view(np.uint32), sigma[p0:p1].view(np.uint32))
        assert not br[:lo].any() and not br[hi:].any()
        ld_sum += np_(gpu_lib.logdet(fr))[0]
        parts += np_(gpu_lib.nll_rows(g, fr, v))[0]
        vb = torch.zeros(N, dtype=torch.float32, device="cuda")
        tbr = torch.zeros(3, dtype=torch.float64, device="cuda")
        gpu_lib.nll_backward_rows(g, fr, v, vb, tbr)
        vb_sum += np_(vb)
        tb_sum += np_(tbr)
        with pytest.raises(gpu_lib.GraphGPError):  # whole-graph calls refuse a range factor
            gpu_lib.whiten(g, fr, v)
    assert abs(ld_sum - ld) <= 1e-12 * abs(ld)
    assert abs(parts - nll) <= 1e-9 * abs(nll), (parts, nll)
    assert rel_norm(vb_sum, vbar) < 1e-5, rel_norm(vb_sum, vbar)
    assert np.all(np.abs(tb_sum - tb) <= 1e-7 * np.abs(tb)), (tb_sum, tb)


def test_factor_rows_rejects_bad_ranges(gpu_lib):
    g, K, f, v = _setup(gpu_lib, 3000, 8, (1, 1.0, 0.1, 1e-6))
    for p0, p1 in [(10, 2000), (0, 50), (2000, 1000), (0, 3001), (-1, 100)]:
        with pytest.raises(gpu_lib.GraphGPError):
            gpu_lib.factor_rows(g, K, p0, p1)


def test_sharded_nll_one_nccl_rank(gpu_lib):
    """ShardedNLL through NCCL with one rank: its collectives are identities,
    so it must return graphgp_nll and graphgp_nll_backward."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    td.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        g, K, f, v = _setup(gpu_lib, 20_011, 16, (1, 1.0, 0.1, 1e-6))
        sh = shard.ShardedNLL(g.N, g.n0, lambda p0, p1: shard.GpuRowOps(g, K, p0, p1))
        nll, vbar, tb = sh.value_and_grad(v.clone())
        want = np_(gpu_lib.nll(g, f, v))[0]
        vb_w, tb_w = (np_(t) for t in gpu_lib.nll_backward(g, f, v))
        assert abs(np_(nll)[0] - want) <= 1e-9 * abs(want)
        assert rel_norm(np_(vbar), vb_w) < 1e-5
        assert np.all(np.abs(np_(tb) - tb_w) <= 1e-7 * np.abs(tb_w))
    finally:
        td.destroy_process_group()
