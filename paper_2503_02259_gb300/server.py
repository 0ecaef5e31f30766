"""Python client of the continuous-batching server in libgp.so (argument marshalling)."""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import _binding as B
from ._binding import check, lib


class Server:
    """gp_server on the current CUDA device with a device-memory budget and slots;
    max_batch > 1 lets a worker run up to that many compatible loss + gradient
    requests as one batched solve (grouped product launches)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, max_batch: int = 1):
        h = ctypes.c_void_p()
        if max_batch > 1:
            check(lib().gp_server_create_batched(int(hbm_budget_bytes), int(max_slots),
                                                 int(max_batch), ctypes.byref(h)),
                  "gp_server_create_batched")
        else:
            check(lib().gp_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)),
                  "gp_server_create")
        self.t0 = time.perf_counter()   # the server clock's origin (its times are relative to it)
        self._h = h
        self._keep = {}   # host arrays of queued requests stay alive until polled

    def close(self):
        if self._h:
            check(lib().gp_server_destroy(self._h), "gp_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def request(kind: int, X: np.ndarray, y: np.ndarray, kernel: int, theta, nprobe: int = 16,
                Xstar: np.ndarray | None = None, cg_maxit: int = 20, nlanczos: int = 20,
                cg_rtol: float = 1e-8, seed: int = 0, prec: int = B.PREC_FP32,
                slq_prec: int = B.PREC_FP32):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
        Xs = None if Xstar is None else np.ascontiguousarray(Xstar, dtype=np.float32)
        s, f, l = (float(v) for v in theta)
        r = B.gp_request(kind=int(kind), d=X.shape[1], n=X.shape[0], kernel=int(kernel),
                         nprobe=int(nprobe), theta=B.gp_theta(s, f, l), X=X.ctypes.data,
                         y=y.ctypes.data, Xstar=0 if Xs is None else Xs.ctypes.data,
                         m=0 if Xs is None else Xs.shape[0], cg_maxit=int(cg_maxit),
                         nlanczos=int(nlanczos), cg_rtol=float(cg_rtol), seed=int(seed) & (2**64 - 1),
                         prec=int(prec), slq_prec=int(slq_prec))
        return r, (X, y, Xs)

    def footprint(self, req) -> int:
        return lib().gp_server_footprint(ctypes.byref(req))

    def submit(self, req, keep) -> int:
        t = ctypes.c_uint64()
        check(lib().gp_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "gp_server_submit")
        self._keep[t.value] = (req, keep)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else a dict with the result (mu for predictions)."""
        req, keep = self._keep[ticket]
        res = B.gp_result()
        mu = None
        if req.kind == 1:
            mu = np.empty(req.m, dtype=np.float32)
            res.mu = mu.ctypes.data
        st = lib().gp_server_poll(self._h, ticket, ctypes.byref(res))
        if st == B.GP_ERR_TIMEOUT:
            return None
        check(st, "gp_server_poll")
        del self._keep[ticket]
        return {"status": res.status, "loss": res.loss, "grad": list(res.grad),
                "cg_iters": res.cg_iters, "relres": res.relres, "t_submit": res.t_submit_s,
                "t_start": res.t_start_s, "t_done": res.t_done_s, "mu": mu}

    def drain(self, timeout_s: float = 600.0) -> None:
        check(lib().gp_server_drain(self._h, float(timeout_s)), "gp_server_drain")

    def stats(self) -> dict:
        s = B.gp_server_stats()
        check(lib().gp_server_get_stats(self._h, ctypes.byref(s)), "gp_server_get_stats")
        return {k: getattr(s, k) for k, _ in B.gp_server_stats._fields_}


def replay(server: Server, requests, time_scale: float = 1.0, cg_maxit_train: int = 20,
           cg_maxit_pred: int = 50, **kw) -> list[dict]:
    """Submit requests at their arrival times (seconds x time_scale) and collect the
    results; returns one dict per request with its latency from submission
    (done - submit, server clock) and from its scheduled arrival time (which also
    counts any delay in submitting it).  The CG budgets default to a fixed 20
    iterations for loss+grad and 50 for predictions."""
    t0 = time.perf_counter()
    shift = t0 - server.t0   # server-clock time of the stream's start
    tickets = []
    for rq in requests:
        delay = rq.t_arrive * time_scale - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        p = rq.problem
        req, keep = Server.request(rq.kind, p.X, p.y, p.kind, p.theta, nprobe=rq.nprobe,
                                   Xstar=rq.Xstar,
                                   cg_maxit=cg_maxit_train if rq.kind == 0 else cg_maxit_pred, **kw)
        tickets.append(server.submit(req, keep))
    server.drain()
    out = []
    for t, rq in zip(tickets, requests):
        r = server.poll(t)
        r["latency_s"] = r["t_done"] - r["t_submit"]
        r["latency_from_arrival_s"] = r["t_done"] - (shift + rq.t_arrive * time_scale)
        out.append(r)
    return out
