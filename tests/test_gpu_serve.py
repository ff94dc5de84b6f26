"""Serving engine: every result is the same alone and in a concurrent mix
(vectors bit-identical except the NLL gradient, whose atomic transposed sums
agree to rounding; FP64 scalars within 1e-9 relative), admission under a
tight HBM budget, and a short Poisson stream through the engine and through
the one-at-a-time form."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

SIZES = [(3000, 8, "uniform"), (20011, 16, "gaussian"), (60000, 32, "uniform"),
         (5000, 16, "blobs"), (12000, 8, "ldr"), (40000, 16, "uniform")]


def _instances(gg):
    out = []
    for i, (N, k, kind) in enumerate(SIZES):
        pts = torch.from_numpy(workloads.cloud(kind, N, 90 + i)).cuda()
        g = gg.build_graph(pts, k, n0=min(N, 256))
        f = gg.factor(g, gg.Kernel(gg.MATERN32, 1.0, 0.05 + 0.02 * i, 1e-5))
        out.append((g, f))
    return out


def _reference(gg, inst, op, x):
    from paper_2606_11402_gb300 import serve as sv
    g, f = inst
    xd = x.cuda()
    if op == sv.GENERATE:
        return gg.generate(g, f, xd).cpu(), None
    if op == sv.WHITEN:
        return gg.whiten(g, f, xd).cpu(), None
    if op == sv.LOGDET:
        return None, gg.logdet(f).cpu()
    sc = torch.zeros(4, dtype=torch.float64, device="cuda")
    gg.nll(g, f, xd, out=sc[:1])
    vb, _ = gg.nll_backward(g, f, xd, 1.0, thetabar=sc[1:])
    return vb.cpu(), sc.cpu()


def test_results_identical_alone_and_in_mix(gpu_lib):
    from paper_2606_11402_gb300 import serve as sv
    inst = _instances(gpu_lib)
    inputs = [torch.from_numpy(workloads.white_noise(g.N, 200 + i)).pin_memory()
              for i, (g, _) in enumerate(inst)]
    ref = {(i, op): _reference(gpu_lib, inst[i], op, inputs[i]) for i in range(len(inst))
           for op in sv.OPS}
    torch.cuda.synchronize()
    server = sv.Server(n_slots=4)
    ids = [server.register(g, f) for g, f in inst]
    server.start()
    rng = np.random.default_rng(0)
    reqs = [(int(rng.integers(len(inst))), int(rng.choice(sv.OPS))) for _ in range(64)]
    outs = []
    for i, op in reqs:
        out = torch.full((inst[i][0].N,), float("nan"), dtype=torch.float32).pin_memory()
        sc = torch.full((4,), float("nan"), dtype=torch.float64).pin_memory()
        t = server.submit(ids[i], op, inputs[i], out, sc)
        outs.append((t, i, op, out, sc))
    for t, i, op, out, sc in outs:
        st, arr, adm, done = server.wait(t)
        assert st == 0 and arr <= adm <= done
        vref, sref = ref[(i, op)]
        if vref is not None and op == sv.NLL_GRAD:
            # the gradient's transposed sums are atomic: equal to rounding
            d = (out.double() - vref.double()).norm() / vref.double().norm()
            assert d < 1e-6, (i, op, d)
        elif vref is not None:
            assert torch.equal(out, vref), (i, op)
        if op == sv.LOGDET:
            assert sc[0].item() == sref[0].item()
        if op == sv.NLL_GRAD:
            assert np.allclose(sc.numpy(), sref.numpy(), rtol=1e-9, atol=0)
    assert server.stats()["errors"] == 0
    server.close()


def test_admission_under_tight_budget_and_streams(gpu_lib):
    from paper_2606_11402_gb300 import serve as sv
    inst = _instances(gpu_lib)[:3]
    inputs = [torch.from_numpy(workloads.white_noise(g.N, 300 + i)).pin_memory()
              for i, (g, _) in enumerate(inst)]
    # a budget below one request's footprint still serves, one at a time
    server = sv.Server(n_slots=4, hbm_budget=1024)
    for g, f in inst:
        server.register(g, f)
    server.start()
    reqs = sv.poisson_stream(len(inst), rate=400.0, duration=0.5, seed=1)
    res = sv.run_stream(reqs, inputs, server=server)
    assert res["requests"] == len(reqs) and res["p99_ms"] > 0
    assert server.stats()["completed"] == len(reqs)
    server.close()
    base = sv.run_stream(reqs, inputs, instances=inst)
    assert base["requests"] == len(reqs)
