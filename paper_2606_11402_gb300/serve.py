"""Serving over resident GraphGP instances (binding of graphgp_server_*).

``Server`` wraps the native continuous-batching engine: register instances
(graph + factor), start, submit requests with their arrival time, wait for
tickets.  ``run_stream`` drives a request stream with given arrival times
through either the engine or the one-request-at-a-time form (plain library
calls on one stream, each request copied in, computed and copied out before
the next starts) and returns per-request latencies.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import Factor, Graph, _check, _stream, load

GENERATE, WHITEN, LOGDET, NLL_GRAD = 0, 1, 2, 3
OPS = (GENERATE, WHITEN, LOGDET, NLL_GRAD)

_P = ctypes.c_void_p
_declared = False


def _lib():
    global _declared
    L = load()
    if not _declared:
        L.graphgp_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, _P]
        L.graphgp_server_register.argtypes = [_P, _P, _P, _P]
        L.graphgp_server_start.argtypes = [_P]
        L.graphgp_server_submit.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                            ctypes.c_double, _P]
        L.graphgp_server_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_double, _P]
        L.graphgp_server_stats.argtypes = [_P, _P, _P, _P, _P]
        L.graphgp_server_destroy.argtypes = [_P]
        L.graphgp_server_destroy.restype = None
        for n in ("graphgp_server_create", "graphgp_server_register", "graphgp_server_start",
                  "graphgp_server_submit", "graphgp_server_wait", "graphgp_server_stats"):
            getattr(L, n).restype = ctypes.c_int
        _declared = True
    return L


class Server:
    def __init__(self, n_slots: int = 8, hbm_budget: int = 0, use_graphs: bool = True):
        self._h = ctypes.c_void_p()
        _check(_lib().graphgp_server_create(n_slots, hbm_budget, int(use_graphs),
                                            ctypes.byref(self._h)), "server_create")
        self._keep = []

    def register(self, graph: Graph, fac: Factor) -> int:
        iid = ctypes.c_int()
        _check(_lib().graphgp_server_register(self._h, graph.handle, fac.handle, ctypes.byref(iid)),
               "server_register")
        self._keep.append((graph, fac))
        return iid.value

    def start(self):
        _check(_lib().graphgp_server_start(self._h), "server_start")

    def submit(self, inst: int, op: int, in_h=None, out_h=None, scal_h=None,
               arrival: float = 0.0) -> int:
        t = ctypes.c_uint64()
        ptr = lambda a: None if a is None else ctypes.c_void_p(a.data_ptr())
        _check(_lib().graphgp_server_submit(self._h, inst, op, ptr(in_h), ptr(out_h), ptr(scal_h),
                                            float(arrival), ctypes.byref(t)), "server_submit")
        return t.value

    def wait(self, ticket: int, timeout: float = 60.0):
        """(status, arrival, admit, done) of a ticket."""
        times = (ctypes.c_double * 3)()
        rc = _lib().graphgp_server_wait(self._h, ticket, float(timeout), times)
        return rc, times[0], times[1], times[2]

    def stats(self):
        c, e, q, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(_lib().graphgp_server_stats(self._h, ctypes.byref(c), ctypes.byref(e),
                                           ctypes.byref(q), ctypes.byref(b)), "server_stats")
        return dict(completed=c.value, errors=e.value, queued=q.value, bytes_in_flight=b.value)

    def close(self):
        if self._h:
            _lib().graphgp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Request:
    inst: int
    op: int
    arrival: float  # seconds from the start of the stream


def poisson_stream(n_inst: int, rate: float, duration: float, seed: int,
                   ops=OPS) -> list:
    """Poisson arrivals at `rate` per second; instance and operation uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append(Request(int(rng.integers(n_inst)), int(rng.choice(ops)), t))


def _percentiles(lat):
    a = np.asarray(lat)
    return dict(p50_ms=float(np.percentile(a, 50) * 1e3), p99_ms=float(np.percentile(a, 99) * 1e3),
                p999_ms=float(np.percentile(a, 99.9) * 1e3), mean_ms=float(a.mean() * 1e3),
                max_ms=float(a.max() * 1e3))


OP_NAMES = {GENERATE: "generate", WHITEN: "whiten", LOGDET: "logdet", NLL_GRAD: "nll_grad"}


def run_stream(reqs, inputs, server: Server | None = None, instances=None, stream=None):
    """Drives `reqs` in real time.  inputs[i] is a pinned host float32 tensor
    (the request input of instance i).  With `server`, requests go to the
    engine; otherwise `instances[i] = (graph, factor)` are served one at a time
    on one stream with the plain API.  Returns latency percentiles (overall
    and per operation), the split of each latency into queue wait (arrival
    to admission on a slot, or to the start of service one at a time) and
    service (admission to completion: copies in, device work, copies out),
    the number of failed requests, and the throughput."""
    from . import generate as gen, logdet as ld, nll, nll_backward, whiten as wh
    t0 = time.monotonic() + 0.05
    lat, done_at, queue, service, ops = [], [], [], [], []
    errors = 0
    if server is not None:
        tickets = []
        for r in reqs:
            wait = t0 + r.arrival - time.monotonic()
            if wait > 0:
                time.sleep(wait)
            tickets.append(server.submit(r.inst, r.op, inputs[r.inst], arrival=t0 + r.arrival))
        for r, tk in zip(reqs, tickets):
            st, arr, adm, done = server.wait(tk)
            if st != 0:
                errors += 1
                continue
            lat.append(done - arr)
            queue.append(adm - arr)
            service.append(done - adm)
            ops.append(r.op)
            done_at.append(done)
    else:
        s = torch.cuda.current_stream() if stream is None else stream
        dev = {}
        for i, (g, f) in enumerate(instances):
            dev[i] = (torch.empty(g.N, dtype=torch.float32, device="cuda"),
                      torch.empty(g.N, dtype=torch.float32, device="cuda"),
                      torch.empty(g.N, dtype=torch.float32).pin_memory())
        sc = torch.empty(4, dtype=torch.float64, device="cuda")
        sc_h = torch.empty(4, dtype=torch.float64).pin_memory()
        for r in reqs:
            wait = t0 + r.arrival - time.monotonic()
            if wait > 0:
                time.sleep(wait)
            start = time.monotonic()
            g, f = instances[r.inst]
            din, dout, hout = dev[r.inst]
            if r.op != LOGDET:
                din.copy_(inputs[r.inst], non_blocking=True)
            if r.op == GENERATE:
                gen(g, f, din, out=dout)
            elif r.op == WHITEN:
                wh(g, f, din, out=dout)
            elif r.op == LOGDET:
                ld(f, out=sc[:1])
            else:
                sc.zero_()
                nll(g, f, din, out=sc[:1])
                nll_backward(g, f, din, 1.0, vbar=dout, thetabar=sc[1:])
            if r.op != LOGDET:
                hout.copy_(dout, non_blocking=True)
            if r.op in (LOGDET, NLL_GRAD):
                sc_h.copy_(sc, non_blocking=True)
            s.synchronize()
            now = time.monotonic()
            lat.append(now - (t0 + r.arrival))
            queue.append(start - (t0 + r.arrival))
            service.append(now - start)
            ops.append(r.op)
            done_at.append(now)
    span = max(done_at) - t0 if done_at else 0.0
    res = _percentiles(lat) if lat else {}
    res.update(requests=len(lat), errors=errors,
               throughput_rps=len(lat) / span if span > 0 else 0.0, span_s=span)
    if lat:
        q, sv = np.asarray(queue), np.asarray(service)
        res["queue_p50_ms"] = float(np.percentile(q, 50) * 1e3)
        res["queue_p99_ms"] = float(np.percentile(q, 99) * 1e3)
        res["service_p50_ms"] = float(np.percentile(sv, 50) * 1e3)
        res["service_p99_ms"] = float(np.percentile(sv, 99) * 1e3)
        opa = np.asarray(ops)
        res["per_op"] = {}
        for op, name in OP_NAMES.items():
            m = opa == op
            if m.any():
                la = np.asarray(lat)[m]
                res["per_op"][name] = {
                    "requests": int(m.sum()), "p50_ms": float(np.percentile(la, 50) * 1e3),
                    "p99_ms": float(np.percentile(la, 99) * 1e3),
                    "service_p50_ms": float(np.percentile(sv[m], 50) * 1e3),
                    "service_p99_ms": float(np.percentile(sv[m], 99) * 1e3)}
    return res
