#!/usr/bin/env python3
"""Benchmark of the GraphGP Vecchia hot path on GB300.

One step = one generate sweep (v = L xi, Alg. 1) + one whiten sweep
(xi = L^-1 v, Sec. 3) + the log-determinant, over the whole headline
workload: N = 2^26 points from a 3-D unit Gaussian (the paper's benchmark
cloud), k = 16 preceding neighbours, Matern-3/2 (s2 = 1, l = 0.1, nugget
1e-6), n0 = 256.  The graph and the factor are built once before timing
(their throughput is reported beside the line).  Every operand (4 GiB of
neighbour rows, 4 GiB of weights, 256 MiB per vector) is larger than the
129 MB L2, so no flush is needed between steps.

value = points per second through one step (N / step time).
e2e   = the same through the public API from pinned HOST buffers: xi copied
        in, v and xi and logdet copied out, inside the timed region.

Beside the line: the graph build and factor rates, the on-the-fly sweeps,
the adjoints (NLL gradient, generate VJP, the one-pass NLL value and
gradient, the vector-only VJPs), the differentiation workload (N = 2^22,
k = 32, SE), the large-dynamic-range and scale legs, the serving stream and
the CPU oracle's per-stage baseline.

Multi-GPU: the headline step contains generate, which does not shard (every
depth level would need an exchange); under torchrun every rank runs an
independent replica and value sums the ranks' points over the slowest
rank's time (weak scaling).  The NLL and its gradient shard by position
range (shard.py).

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "generate/whiten points/s at N=2^26,k=16 (%HBM peak); serving p50/p99 latency"
UNIT = "points/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _measured_traffic(kernel: str, N: int):
    """DRAM bytes per launch of `kernel` from profiles/sweeps_traffic_N2e26.txt,
    or None when the capture does not cover this N or the kernel sources have
    changed since it was taken (sha256 recorded in the file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "sweeps_traffic_N2e26.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    want, n_cap, traffic = {}, None, None
    for line in text.splitlines():
        if line.startswith("source_sha256 "):
            f, h = line[len("source_sha256 "):].split(":")
            want[f.strip()] = h.strip()
        elif line.startswith("N:"):
            n_cap = int(line.split(":")[1])
        elif line.startswith(kernel + ":"):
            for kv in line.split()[1:]:
                if kv.startswith("traffic_bytes="):
                    traffic = int(kv.split("=")[1])
    if n_cap != N or traffic is None or not want:
        return None
    for f, h in want.items():
        with open(os.path.join(ROOT, f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != h:
                return None
    return traffic


def _cpulist(text):
    out = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        out.update(range(int(lo), int(hi or lo) + 1))
    return out


def _near_gpu_cpus(dev):
    """Host cores of the GPU's NUMA node (sysfs local_cpulist of its PCI
    address) among those this process may use, or None where the topology is
    not exposed or every usable core is already local."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        addr = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open(f"/sys/bus/pci/devices/{addr}/local_cpulist") as fh:
            cpus = _cpulist(fh.read())
        avail = os.sched_getaffinity(0)
        cpus &= avail
        return cpus if cpus and cpus != avail else None
    except Exception:
        return None


def _clock_sampler(out_path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(out_path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def _clock_summary(path, gpu_index):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            sm.append(float(parts[1]))
            mx = float(parts[2])
            for n, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
    except Exception:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def replica_rate(total_ms, steps, points_per_rank, world, reduce_max):
    """Whole-job rate of `world` independent replicas (the path does not
    shard across GPUs): every rank processes points_per_rank points per step
    and the job takes as long as its slowest rank.  reduce_max(x) returns the
    maximum of x over the ranks.  Returns (ms per step, points/s)."""
    ms_step = reduce_max(total_ms) / steps
    return ms_step, points_per_rank * world / (ms_step / 1e3)


def replica_seed(base, rank):
    """Each replica draws its own cloud and noise."""
    return base + rank


def _cpu_model():
    """Host CPU model name and logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        import platform
        name = platform.processor() or platform.machine()
    return name, os.cpu_count() or 1


def _oracle_cloud(kind, N, seed):
    import workloads
    return {"gaussian": workloads.unit_gaussian, "ldr": workloads.ldr_cloud,
            "uniform": workloads.uniform_cube}[kind](N, seed)


def _oracle_stages(kind, N, k, kern, seed, xi_seed, reps=3):
    """Seconds of each stage of the FP64 oracle, as it stands, on one thread:
    graph build (sequential tree search for the k preceding neighbours),
    factor, generate, whiten, logdet (medians of `reps` passes for the
    sweeps)."""
    import numpy as np
    import oracle
    import workloads
    pts = _oracle_cloud(kind, N, seed)
    t0 = time.perf_counter()
    g = oracle.build_graph(pts, k, 256, knn="tree")
    t_graph = time.perf_counter() - t0
    K = oracle.Kernel(*kern)
    t0 = time.perf_counter()
    fo = oracle.factor(g["pts_pos"], g["nbr_pos"], k, g["n0"], K)
    t_factor = time.perf_counter() - t0
    xi = workloads.white_noise(N, xi_seed).astype(np.float64)
    tg, tw, tl = [], [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        v = oracle.generate(fo, g["nbr_pos"], k, g["n0"], xi)
        t1 = time.perf_counter()
        oracle.whiten(fo, g["nbr_pos"], k, g["n0"], v)
        t2 = time.perf_counter()
        oracle.logdet(fo["sigma"])
        t3 = time.perf_counter()
        tg.append(t1 - t0)
        tw.append(t2 - t1)
        tl.append(t3 - t2)
    return {"N": N, "k": k, "graph_s": t_graph, "factor_s": t_factor,
            "generate_s": statistics.median(tg), "whiten_s": statistics.median(tw),
            "logdet_s": statistics.median(tl)}


def _replica_step_rate(args):
    """One replica of the headline sample on one host core: points/s of
    generate + whiten + logdet (graph and factor untimed)."""
    N, seed, reps = args
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    w = workloads.WORKLOADS["metric"]
    pts = workloads.unit_gaussian(N, seed)
    g = oracle.build_graph(pts, w["k"], 256, knn="tree")
    fo = oracle.factor(g["pts_pos"], g["nbr_pos"], w["k"], 256, oracle.Kernel(*w["kernel"]))
    xi = workloads.white_noise(N, w["xi_seed"]).astype("float64")
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        v = oracle.generate(fo, g["nbr_pos"], w["k"], 256, xi)
        oracle.whiten(fo, g["nbr_pos"], w["k"], 256, v)
        oracle.logdet(fo["sigma"])
        times.append(time.perf_counter() - t0)
    return N / statistics.median(times)


def cpu_baseline(N_sample=1 << 18, reps=10, stages=False):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    one thread, and (stages=True) every host core running an independent
    replica, plus the per-stage times of the tiny, large-dynamic-range and
    headline-sample workloads on one thread."""
    import numpy as np
    import oracle
    import workloads
    w = workloads.WORKLOADS["metric"]
    pts = workloads.unit_gaussian(N_sample, w["seed"])
    t0 = time.perf_counter()
    g = oracle.build_graph(pts, w["k"], 256, knn="tree")
    t_graph = time.perf_counter() - t0
    K = oracle.Kernel(*w["kernel"])
    t0 = time.perf_counter()
    fo = oracle.factor(g["pts_pos"], g["nbr_pos"], w["k"], 256, K)
    t_factor = time.perf_counter() - t0
    xi = workloads.white_noise(N_sample, w["xi_seed"]).astype(np.float64)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        v = oracle.generate(fo, g["nbr_pos"], w["k"], 256, xi)
        oracle.whiten(fo, g["nbr_pos"], w["k"], 256, v)
        oracle.logdet(fo["sigma"])
        times.append(time.perf_counter() - t0)
    t_step = statistics.median(times)
    model, ncpu = _cpu_model()
    out = {"value": N_sample / t_step, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"unit-Gaussian cloud of {N_sample} points, k={w['k']}, n0=256, same kernel; "
                      f"median of {reps} generate+whiten+logdet passes (FP64, 1 thread of "
                      f"{ncpu}, {model}); oracle graph build {t_graph:.1f} s and factor "
                      f"{t_factor:.1f} s untimed"),
           "ms_per_step": t_step * 1e3, "host_cores": ncpu, "cpu_model": model,
           "graph_points_per_s": N_sample / t_graph, "factor_points_per_s": N_sample / t_factor}
    if stages:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        n_rep = 1 << 16
        with ctx.Pool(ncpu) as pool:
            rates = pool.map(_replica_step_rate, [(n_rep, 100 + r, 5) for r in range(ncpu)])
        out["all_cores"] = {"value": float(sum(rates)), "unit": UNIT, "cores": ncpu,
                            "sample": (f"{ncpu} independent replicas of a {n_rep}-point "
                                       "unit-Gaussian sample, one per host core; generate + "
                                       "whiten + logdet, median of 5 passes each")}
        tiny = workloads.WORKLOADS["tiny"]
        ldr = workloads.WORKLOADS["ldr"]
        out["stages_1_thread"] = {
            "tiny": _oracle_stages("uniform", tiny["N"], tiny["k"], tiny["kernel"], tiny["seed"],
                                   tiny["xi_seed"]),
            "large_dynamic_range": _oracle_stages("ldr", ldr["N"], ldr["k"], ldr["kernel"],
                                                  ldr["seed"], ldr["xi_seed"], reps=1),
            "headline_sample": {"N": N_sample, "k": w["k"], "graph_s": t_graph,
                                "factor_s": t_factor, "step_s": t_step},
        }
    return out


def serving_bench(n_inst=64, rate=2000.0, duration=5.0, seed=8, n_slots=8):
    """Poisson stream of generate / whiten / logdet / NLL-gradient requests over
    a pool of resident instances: N log-uniform in [1e3, 1e6], k in {8, 16, 32},
    Matern-3/2 with l log-uniform in [0.01, 0.2], half uniform and half
    clustered clouds.  Returns the engine's and the one-at-a-time form's
    p50/p99 latency and throughput on the same arrivals."""
    import numpy as np
    import torch

    import paper_2606_11402_gb300 as gg
    import workloads
    from paper_2606_11402_gb300 import serve as sv
    rng = np.random.Generator(np.random.PCG64(seed))
    inst, inputs, total_pts = [], [], 0
    t0 = time.perf_counter()
    for i in range(n_inst):
        N = int(10 ** rng.uniform(3.0, 6.0))
        k = int(rng.choice([8, 16, 32]))
        ell = float(10 ** rng.uniform(-2.0, np.log10(0.2)))
        pts = (workloads.uniform_cube(N, seed * 1000 + i) if i % 2 == 0 else
               workloads.blobs(N, seed * 1000 + i, n_blobs=100))
        g = gg.build_graph(torch.from_numpy(pts).cuda(), k, n0=min(N, 256))
        f = gg.factor(g, gg.Kernel(gg.MATERN32, 1.0, ell, 1e-6))
        inst.append((g, f))
        inputs.append(torch.from_numpy(workloads.white_noise(N, seed * 1000 + i)).pin_memory())
        total_pts += N
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    reqs = sv.poisson_stream(n_inst, rate, duration, seed + 1)
    warm = sv.poisson_stream(n_inst, rate, 0.5, seed + 2)
    server = sv.Server(n_slots=n_slots)
    for g, f in inst:
        server.register(g, f)
    server.start()
    # capture every (instance, op, slot) graph before timing
    for _ in range(n_slots):
        tks = [server.submit(i, op, inputs[i]) for i in range(n_inst) for op in sv.OPS]
        for t in tks:
            server.wait(t)
    sv.run_stream(warm, inputs, server=server)
    eng = sv.run_stream(reqs, inputs, server=server)
    # saturation: 2000 requests arriving within 1 ms, completion rate
    burst = sv.poisson_stream(n_inst, 2.0e6, 1.0e-3, seed + 3)
    eng_sat = sv.run_stream(burst, inputs, server=server)
    server.close()
    sv.run_stream(warm, inputs, instances=inst)
    one = sv.run_stream(reqs, inputs, instances=inst)
    one_sat = sv.run_stream(burst, inputs, instances=inst)
    pts_req = float(np.mean([inst[r.inst][0].N for r in reqs])) if reqs else 0.0
    return {"workload": (f"Poisson {rate:.0f} req/s for {duration:.0f} s over {n_inst} resident "
                         "instances (N log-uniform 1e3..1e6, k in {8,16,32}, Matern-3/2 "
                         "l log-uniform 0.01..0.2, uniform/clustered), ops uniform over "
                         "generate/whiten/logdet/nll-gradient"),
            "engine": eng, "one_at_a_time": one, "slots": n_slots,
            "saturation": {"requests": len(burst),
                           "engine_rps": eng_sat["throughput_rps"],
                           "one_at_a_time_rps": one_sat["throughput_rps"],
                           "engine_p99_ms": eng_sat["p99_ms"],
                           "one_at_a_time_p99_ms": one_sat["p99_ms"]},
            "mean_points_per_request": pts_req, "setup_s": t_setup,
            "instances_points": total_pts}


def differentiation_bench(stream, reps=3):
    """The differentiation workload (N = 2^22 uniform in [0,1]^3, k = 32,
    squared exponential l = 0.03, nugget 1e-4, v drawn from the model): the
    NLL and its gradient with respect to (l, s2, nugget) and v, the factor
    recomputed in the backward pass."""
    import torch

    import paper_2606_11402_gb300 as gg
    import workloads
    w = workloads.WORKLOADS["diff"]
    N, k = w["N"], w["k"]
    pts = torch.from_numpy(workloads.uniform_cube(N, w["seed"])).cuda()
    kern = gg.Kernel(*w["kernel"])
    g = gg.build_graph(pts, k)
    f = gg.factor(g, kern)
    v = gg.generate(g, f, torch.from_numpy(workloads.white_noise(N, w["xi_seed"])).cuda())
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    vbar = torch.empty_like(v)
    tbar = torch.zeros(3, dtype=torch.float64, device="cuda")

    def step():
        gg.nll(g, f, v, out=out)
        gg.nll_backward(g, f, v, vbar=vbar, thetabar=tbar)
    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    # on-the-fly forms (no stored factor: theta may change every step)
    xi_d = torch.from_numpy(workloads.white_noise(N, w["xi_seed"])).cuda()
    vf = torch.empty_like(v)
    gg.generate_fused(g, kern, xi_d, out=vf)
    gg.nll_fused(g, kern, v, out=out)
    torch.cuda.synchronize()
    a.record(stream)
    gg.generate_fused(g, kern, xi_d, out=vf)
    b.record(stream)
    torch.cuda.synchronize()
    fused_gen_ms = a.elapsed_time(b)
    a.record(stream)
    gg.nll_fused(g, kern, v, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    fused_nll_ms = a.elapsed_time(b)
    del vf, xi_d
    # one pass: NLL value and gradient with the factors recomputed
    gg.nll_grad_fused(g, kern, v, out=out, vbar=vbar, thetabar=tbar)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        gg.nll_grad_fused(g, kern, v, out=out, vbar=vbar, thetabar=tbar)
    b.record(stream)
    torch.cuda.synchronize()
    fused_grad_ms = a.elapsed_time(b) / reps
    pbar = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    gg.nll_backward_points(g, f, v, out=pbar)
    torch.cuda.synchronize()
    a.record(stream)
    gg.nll_backward_points(g, f, v, out=pbar)
    b.record(stream)
    torch.cuda.synchronize()
    pts_ms = a.elapsed_time(b)
    del f
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f2 = gg.factor(g, kern)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    st, _ = gg.sync_status(g, f2)
    return {"workload": "differentiation: N=2^22 uniform [0,1]^3, k=32, squared exponential "
                        "l=0.03 nugget 1e-4; NLL + gradient (l, s2, nugget, v)",
            "nll_and_gradient_ms": ms, "points_per_s": N / (ms / 1e3),
            "point_gradient_ms": pts_ms, "fused_generate_ms": fused_gen_ms,
            "fused_nll_ms": fused_nll_ms, "fused_nll_and_gradient_ms": fused_grad_ms,
            "factor_ms": t_factor * 1e3, "status": st}


def config_leg(name, stream, hbm, reps=5):
    """Throughput of one configured workload on its own (graph, factor,
    generate, whiten, logdet), with its sweeps against the HBM roofline:
    the large-dynamic-range cloud (N = 2^20, k = 16, Matern-3/2 l = 0.05, no
    nugget, FP64 rescue threshold 2^-10) or the scale cloud (N = 2^29,
    10^4 blobs + 10 % background, k = 16, Matern-3/2 l = 0.02, nugget 1e-6)."""
    import torch

    import paper_2606_11402_gb300 as gg
    import workloads
    w = workloads.WORKLOADS[name]
    N, k = w["N"], w["k"]
    tol = 2.0 ** -10 if name == "ldr" else 0.0
    kern = gg.Kernel(*w["kernel"], rescue_tol=tol)
    t0 = time.perf_counter()
    pts_h = workloads.cloud(w["cloud"], N, w["seed"])
    t_gen = time.perf_counter() - t0
    pts = torch.from_numpy(pts_h).cuda()
    del pts_h
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = gg.build_graph(pts, k, n0=256)
    torch.cuda.synchronize()
    t_graph = time.perf_counter() - t0
    del pts
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    f = gg.factor(g, kern)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    st, nbad = gg.sync_status(g, f)
    xi = torch.from_numpy(workloads.white_noise(N, w["xi_seed"])).cuda()
    v = torch.empty_like(xi)
    xo = torch.empty_like(xi)
    ld = torch.empty(1, dtype=torch.float64, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    gen_ms = timed(lambda: gg.generate(g, f, xi, out=v))
    wh_ms = timed(lambda: gg.whiten(g, f, v, out=xo))
    ld_ms = timed(lambda: gg.logdet(f, out=ld))
    rt = float(torch.linalg.vector_norm((xo - xi).double()) / torch.linalg.vector_norm(xi.double()))
    alg = (N - g.n0) * (8 * k + 16)
    out = {"workload": name, "N": N, "k": k, "levels": g.num_levels, "rescue_tol": tol or 2.0 ** -7,
           "host_cloud_s": t_gen, "graph_build_s": t_graph, "graph_points_per_s": N / t_graph,
           "factor_s": t_factor, "factor_points_per_s": N / t_factor, "not_pd_rows": nbad,
           "generate_ms": gen_ms, "generate_points_per_s": N / (gen_ms / 1e3),
           "generate_hbm_frac": alg / (gen_ms / 1e3) / 1e9 / hbm,
           "whiten_ms": wh_ms, "whiten_points_per_s": N / (wh_ms / 1e3),
           "whiten_hbm_frac": alg / (wh_ms / 1e3) / 1e9 / hbm,
           "logdet_ms": ld_ms, "whiten_generate_roundtrip_rel": rt, "status": st}
    del g, f, xi, v, xo
    torch.cuda.empty_cache()
    return out


def headline_config(N=1 << 26, k=16, n0=256, world=1):
    """The benchmark workload, as both arms name it in their JSON line."""
    lg = N.bit_length() - 1
    size = f"2^{lg}" if N == 1 << lg else str(N)
    return {"workload": (f"metric: unit Gaussian 3-D cloud, N={size}, k={k}, Matern-3/2 "
                         f"s2=1 l=0.1 nugget 1e-6, n0={n0}; step = generate + whiten + logdet"),
            "N": N, "k": k, "n0": n0, "l2": "inputs larger than L2 (no flush)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    reps = max(1, args.steps)
    cb = cpu_baseline(reps=reps + args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(headline_config(), sample=cb["sample"]),
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2606_11402_gb300 as gg
    import workloads

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    gg.load()
    w = dict(workloads.WORKLOADS["metric"])
    if args.N:
        w["N"] = args.N
    N, k = w["N"], w["k"]
    kern = gg.Kernel(*w["kernel"])
    stream = torch.cuda.current_stream()

    pts = torch.from_numpy(workloads.unit_gaussian(N, replica_seed(w["seed"], rank))).cuda()
    xi_h = workloads.white_noise(N, replica_seed(w["xi_seed"], rank))
    xi = torch.from_numpy(xi_h).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = gg.build_graph(pts, k, n0=256)
    torch.cuda.synchronize()
    t_graph = time.perf_counter() - t0
    del pts
    f = gg.factor(g, kern)  # first call loads the factor kernels
    del f
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = gg.factor(g, kern)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    st, nbad = gg.sync_status(g, f)
    v = torch.empty_like(xi)
    xo = torch.empty_like(xi)
    ld = torch.empty(1, dtype=torch.float64, device="cuda")

    def step():
        gg.generate(g, f, xi, out=v)
        gg.whiten(g, f, v, out=xo)
        gg.logdet(f, out=ld)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-sweep timing on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler, sf = _clock_sampler(os.path.join("/tmp", f"ggp_clocks_{rank}.csv"))
    time.sleep(0.3 if sampler else 0)
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for e0, e1, e2 in ev:
        e0.record(stream)
        gg.generate(g, f, xi, out=v)
        e1.record(stream)
        gg.whiten(g, f, v, out=xo)
        e2.record(stream)
        gg.logdet(f, out=ld)
    end.record(stream)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    if sampler:
        time.sleep(0.2)
        sampler.terminate()
        sampler.wait()
        sf.close()
    total_ms = start.elapsed_time(end)
    gen_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    wh_ms = statistics.mean(b.elapsed_time(c) for _, b, c in ev)

    def reduce_max(x):
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        if dist:
            td.all_reduce(t, op=td.ReduceOp.MAX)
        return t.item()

    ms_step, value = replica_rate(total_ms, args.steps, N, world, reduce_max)
    st2, _ = gg.sync_status(g, f)
    assert st2 >= 0

    # end to end through the public API with pinned host buffers: every step
    # copies its xi in, runs generate + whiten + logdet and copies v, xi and
    # logdet out.  Copies run on their own streams and overlap the sweeps of
    # the neighbouring steps (device vectors double-buffered; a buffer is
    # reused only after the copies that read it have finished).
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    # the pinned buffers are allocated from the host cores nearest the GPU, so
    # their pages sit in the GPU's local memory node (affinity restored after)
    near = _near_gpu_cpus(local)
    all_cpus = os.sched_getaffinity(0)
    if near:
        os.sched_setaffinity(0, near)
    xi_pin = torch.from_numpy(xi_h).pin_memory()
    v_pin = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(2)]
    xo_pin = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(2)]
    ld_pin = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    if near:
        os.sched_setaffinity(0, all_cpus)
    xi_d = [torch.empty_like(xi) for _ in range(2)]
    v_d, xo_d, ld_d = [v, torch.empty_like(v)], [xo, torch.empty_like(xo)], [ld, torch.empty_like(ld)]
    gen_done, out_done = [None, None], [None, None]

    def e2e_step(t):
        b = t % 2
        if gen_done[b] is not None:  # xi_d[b] was read by the generate of step t - 2
            s_in.wait_event(gen_done[b])
        with torch.cuda.stream(s_in):
            xi_d[b].copy_(xi_pin, non_blocking=True)
        e_in = torch.cuda.Event()
        e_in.record(s_in)
        stream.wait_event(e_in)
        if out_done[b] is not None:  # v_d[b], xo_d[b], ld_d[b] copied out at step t - 2
            stream.wait_event(out_done[b])
        gg.generate(g, f, xi_d[b], out=v_d[b])
        e_gen = torch.cuda.Event()
        e_gen.record(stream)
        gen_done[b] = e_gen
        gg.whiten(g, f, v_d[b], out=xo_d[b])
        gg.logdet(f, out=ld_d[b])
        e_comp = torch.cuda.Event()
        e_comp.record(stream)
        s_out.wait_event(e_gen)
        with torch.cuda.stream(s_out):
            v_pin[b].copy_(v_d[b], non_blocking=True)
            s_out.wait_event(e_comp)
            xo_pin[b].copy_(xo_d[b], non_blocking=True)
            ld_pin[b].copy_(ld_d[b], non_blocking=True)
        e_out = torch.cuda.Event()
        e_out.record(s_out)
        out_done[b] = e_out

    for t in range(2):
        e2e_step(t)
    torch.cuda.synchronize()
    s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    s_in.wait_event(s2)
    s_out.wait_event(s2)
    for t in range(args.steps):
        e2e_step(t)
    for e in out_done:
        stream.wait_event(e)
    e2.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_value = replica_rate(s2.elapsed_time(e2), args.steps, N, world, reduce_max)
    assert np.isfinite(v_pin[0].numpy()).all() and np.isfinite(xo_pin[0].numpy()).all()
    assert np.isfinite(ld_pin[0].numpy()).all()

    # on-the-fly sweeps (factors recomputed in the pass, nothing stored)
    fused = {}
    if g.k <= 32:
        def timed(fn, reps=3):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps
        fused["generate_ms"] = timed(lambda: gg.generate_fused(g, kern, xi, out=v))
        fused["whiten_ms"] = timed(lambda: gg.whiten_fused(g, kern, v, out=xo, logdet=ld))
        fused["generate_points_per_s"] = N / (fused["generate_ms"] / 1e3)
        fused["whiten_points_per_s"] = N / (fused["whiten_ms"] / 1e3)

    # adjoints on the same workload
    def timed_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    nll_out = torch.empty(1, dtype=torch.float64, device="cuda")
    vbar = torch.empty_like(v)
    tbar = torch.zeros(3, dtype=torch.float64, device="cuda")
    adj = {"nll_ms": timed_ms(lambda: gg.nll(g, f, v, out=nll_out)),
           "nll_backward_ms": timed_ms(lambda: gg.nll_backward(g, f, v, vbar=vbar, thetabar=tbar)),
           "generate_backward_ms": timed_ms(
               lambda: gg.generate_backward(g, f, xi, v, v, xibar=xo, thetabar=tbar)),
           # the factors recomputed: value and gradient of the NLL in one pass
           "nll_grad_fused_ms": timed_ms(
               lambda: gg.nll_grad_fused(g, kern, v, out=nll_out, vbar=vbar, thetabar=tbar)),
           # vector cotangent only (fixed kernel: no per-row factor backward)
           "nll_backward_vec_ms": timed_ms(
               lambda: gg.nll_backward(g, f, v, vbar=vbar, theta=False)),
           "generate_backward_vec_ms": timed_ms(
               lambda: gg.generate_backward(g, f, xi, v, v, xibar=xo, theta=False))}
    for key in list(adj):
        adj[key.replace("_ms", "_points_per_s")] = N / (adj[key] / 1e3)
    diff = differentiation_bench(stream) if args.diff else None
    hbm, peak_kind = _peaks()
    legs = {}
    if args.legs and not args.N:
        # the headline instance is released first: the scale leg holds ~150 GB
        rows_h, levels_h, n0_h = N - g.n0, g.num_levels, g.n0
        del f, g, v, xo, vbar, xi_d, v_d, xo_d
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        for name in ("ldr", "scale"):
            legs[name] = config_leg(name, stream, hbm)
    else:
        rows_h, levels_h, n0_h = N - g.n0, g.num_levels, g.n0

    rows = rows_h
    bytes_per_point = 8 * k + 16
    alg_bytes = rows * bytes_per_point
    dom = "generate" if gen_ms >= wh_ms else "whiten"
    dom_ms = max(gen_ms, wh_ms)
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(headline_config(N, k, n0_h, world), levels=levels_h),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": _measured_traffic(
                         "generate_kernel" if dom == "generate" else "whiten_tiles_kernel", N),
                     "peak_kind": peak_kind,
                     "bytes_per_point": bytes_per_point, "points_per_launch": rows},
        "stages": {"generate_ms": gen_ms, "whiten_ms": wh_ms,
                   "generate_points_per_s": N / (gen_ms / 1e3),
                   "whiten_points_per_s": N / (wh_ms / 1e3),
                   "generate_hbm_frac": alg_bytes / (gen_ms / 1e3) / 1e9 / hbm,
                   "whiten_hbm_frac": alg_bytes / (wh_ms / 1e3) / 1e9 / hbm,
                   "graph_build_s": t_graph, "graph_points_per_s": N / t_graph,
                   "factor_s": t_factor, "factor_points_per_s": N / t_factor,
                   "not_pd_rows": nbad, "fused": fused, "adjoints": adj},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 8 * N + 8,
                "copies": "pinned host buffers, own streams, overlapping neighbouring steps",
                "host_buffers": ("allocated from the %d host cores local to the GPU" % len(near))
                if near else "allocated without a NUMA preference"},
        # per step: generate = dense mat-vec + the two single-block runs of
        # small levels + the cooperative level sweep; whiten = dense mat-vec +
        # tile sweep; logdet is a device-to-device copy of the factor's sum
        "gpu_launches": 6 * args.steps,
        "clocks": _clock_summary(os.path.join("/tmp", f"ggp_clocks_{rank}.csv"), local),
    }
    if diff is not None:
        line["differentiation"] = diff
    if legs:
        line["configs"] = legs
    if rank == 0 and not args.no_serve:
        sb = serving_bench(duration=args.serve_duration)
        line["serving"] = sb
        line["serving_p50_ms"] = sb["engine"]["p50_ms"]
        line["serving_p99_ms"] = sb["engine"]["p99_ms"]
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(stages=True)
        line["cpu_baseline"] = {kk: vv for kk, vv in cb.items()
                                if kk in ("value", "unit", "cores", "kind", "sample")}
        line["cpu_baseline_detail"] = {kk: cb[kk] for kk in
                                       ("host_cores", "cpu_model", "all_cores", "stages_1_thread")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        td.barrier()
        td.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=0, help="override N (profiling a smaller case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--serve-duration", type=float, default=5.0)
    ap.add_argument("--no-diff", dest="diff", action="store_false",
                    help="skip the differentiation-workload timing")
    ap.add_argument("--no-legs", dest="legs", action="store_false",
                    help="skip the large-dynamic-range and scale workload legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
