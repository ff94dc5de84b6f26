"""graphgp_nll_noalloc, the allocation-free NLL entry point, against
graphgp_nll.

Callers that cannot allocate device memory while they run (a serving loop that
reserved all memory for resident graphs, a latency-critical path that must not
pay cudaMalloc's device-wide synchronisation) use graphgp_nll_noalloc, which
keeps its reduction scratch in a static array inside the library.  This file
calls it through the C ABI twice in a row and checks both results against
graphgp_nll.  The whitened values are computed with the same arithmetic and
only the FP64 summation order differs, so the tolerance is the FP64-reduction
tolerance of the other tests, 1e-9 relative.  The file is collected last so a
run that stops at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,k,kind", [(20_011, 16, "gaussian"), (3000, 8, "uniform"),
                                      (300, 8, "uniform"), (5000, 48, "uniform")])
def test_nll_noalloc_matches_nll_on_two_calls(gpu_lib, N, k, kind):
    pts = torch.from_numpy(workloads.cloud(kind, N, 77)).cuda()
    g = gpu_lib.build_graph(pts, k, n0=min(N, 256))
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    v = gpu_lib.generate(g, f, torch.from_numpy(workloads.white_noise(N, 78)).cuda())
    ref = gpu_lib.nll(g, f, v)
    torch.cuda.synchronize()
    lib = gpu_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.graphgp_nll_noalloc(g.handle, f.handle, ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, gpu_lib.status_string(rc)
        torch.cuda.synchronize()
        got, want = out.item(), ref.item()
        assert np.isfinite(got)
        assert abs(got - want) <= 1e-9 * abs(want), (got, want)


def _call(gpu_lib, g, f, v, out):
    lib = gpu_lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.graphgp_nll_noalloc(g.handle, f.handle, ctypes.c_void_p(v.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), stream)


def test_nll_noalloc_dense_only_and_no_device_allocation(gpu_lib):
    """N == n0: the whole field is the dense block (no tile slots).  A second
    call leaves the device's free memory unchanged: the call allocates
    nothing."""
    N = 200
    pts = torch.from_numpy(workloads.uniform_cube(N, 79)).cuda()
    g = gpu_lib.build_graph(pts, 8, n0=N)
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    v = gpu_lib.generate(g, f, torch.from_numpy(workloads.white_noise(N, 80)).cuda())
    want = gpu_lib.nll(g, f, v).item()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(gpu_lib, g, f, v, out) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out.fill_(float("nan"))
    assert _call(gpu_lib, g, f, v, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert abs(out.item() - want) <= 1e-9 * abs(want), (out.item(), want)


def test_nll_noalloc_rejects_too_many_levels(gpu_lib):
    """A chain graph (every point conditions on the one before it) has one
    depth level per point; beyond 8192 levels the call is refused with
    GRAPHGP_ERR_INVALID before any work, and the output is not written."""
    N = 9000
    pts = workloads.uniform_cube(N, 81)
    order = np.arange(N, dtype=np.int32)
    nbr = np.arange(N - 1, dtype=np.int32)          # position p >= 1 conditions on p - 1
    lo = np.arange(N + 1, dtype=np.int64)           # one point per level
    g = gpu_lib.graph_import(pts, 1, 1, order, nbr, lo)
    assert g.num_levels == N
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    v = torch.zeros(N, dtype=torch.float32, device="cuda")
    out = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
    assert _call(gpu_lib, g, f, v, out) == gpu_lib.ERR_INVALID
    torch.cuda.synchronize()
    assert out.item() == 123.0
