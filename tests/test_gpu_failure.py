"""Failure detection without faulting the GPU: bounded device waits give up,
record a timeout and leave the context usable; host-side errors are reported
as status codes."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(gpu_lib):
    rc = gpu_lib.selftest_wait_timeout(20000)
    assert rc == gpu_lib.ERR_TIMEOUT
    # the context still works: a normal build / factor / generate round trip
    pts = torch.from_numpy(workloads.uniform_cube(5000, 1)).cuda()
    g = gpu_lib.build_graph(pts, 8)
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    xi = torch.from_numpy(workloads.white_noise(5000, 2)).cuda()
    v = gpu_lib.generate(g, f, xi)
    back = gpu_lib.whiten(g, f, v)
    st, _ = gpu_lib.sync_status(g, f)
    assert st == 0
    assert torch.allclose(back, xi, rtol=1e-4, atol=1e-4)
    assert gpu_lib.selftest_wait_timeout(0) == gpu_lib.ERR_INVALID


def test_generate_rejects_overlapping_buffers(gpu_lib):
    """generate marks its output positions pending before the sweep, so an
    output that overlaps the input is refused before any work."""
    N = 5000
    pts = torch.from_numpy(workloads.uniform_cube(N, 1)).cuda()
    g = gpu_lib.build_graph(pts, 8)
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    buf = torch.from_numpy(workloads.white_noise(2 * N, 2)).cuda()
    keep = buf.clone()
    for a, b in [(0, 0), (0, N // 2), (N // 2, 0)]:
        with pytest.raises(gpu_lib.GraphGPError):
            gpu_lib.generate(g, f, buf[a:a + N], out=buf[b:b + N])
    assert torch.equal(buf, keep)
    v = gpu_lib.generate(g, f, buf[:N], out=buf[N:])  # adjacent, not overlapping
    assert torch.isfinite(v).all()


def test_server_wait_timeout_and_bad_requests(gpu_lib):
    from paper_2606_11402_gb300 import serve as sv
    pts = torch.from_numpy(workloads.unit_gaussian(200_000, 3)).cuda()
    g = gpu_lib.build_graph(pts, 16)
    f = gpu_lib.factor(g, gpu_lib.Kernel(gpu_lib.MATERN32, 1.0, 0.1, 1e-6))
    server = sv.Server(n_slots=2)
    iid = server.register(g, f)
    with pytest.raises(gpu_lib.GraphGPError):
        server.submit(iid, sv.GENERATE, None)  # not started yet
    server.start()
    x = torch.from_numpy(workloads.white_noise(g.N, 4)).pin_memory()
    with pytest.raises(gpu_lib.GraphGPError):
        server.submit(iid + 5, sv.GENERATE, x)
    with pytest.raises(gpu_lib.GraphGPError):
        server.submit(iid, 9, x)
    tickets = [server.submit(iid, sv.NLL_GRAD, x) for _ in range(4)]
    st, *_ = server.wait(tickets[-1], timeout=1e-6)
    assert st in (gpu_lib.ERR_TIMEOUT, 0)
    for t in tickets:
        st, arr, adm, done = server.wait(t, timeout=60)
        assert st == 0 and arr <= adm <= done
    assert server.stats()["errors"] == 0
    server.close()
