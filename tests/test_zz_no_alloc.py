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
