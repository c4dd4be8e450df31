"""Binding of the continuous-batching server of libmasw (masw_server_*).

Argument marshalling only: admission, ticks, retirement and the trace replay
loop run natively in the library. ``Server.run_trace`` replays a request
trace (a ``workloads.Models`` with one model per request and arrival times)
and returns per-request latencies; ``latency_summary`` reduces them to
p50/p99 and throughput.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import masw


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_layers", ctypes.c_int32),
                ("max_lambda", ctypes.c_int32), ("mem_cap_bytes", ctypes.c_int64),
                ("chunks_per_tick", ctypes.c_int32), ("warps_per_block", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("in_flight", ctypes.c_int32), ("active_items", ctypes.c_int32),
                ("bytes_in_flight", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("completed", ctypes.c_int64)]


def _lib():
    lib = masw.load()
    if not getattr(lib, "_serving_sigs", False):
        p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "masw_server_create": [p, ctypes.POINTER(ServerConfig), p, ctypes.POINTER(p)],
            "masw_server_destroy": [p],
            "masw_server_submit": [p, i32, p, p, p, p, i32, p, ctypes.POINTER(i64)],
            "masw_server_tick": [p, ctypes.POINTER(i32)],
            "masw_server_poll": [p, i64, p, p, p],
            "masw_server_get_stats": [p, ctypes.POINTER(ServerStats)],
            "masw_server_run_trace": [p, i32, p, p, p, p, p, p, p, p, d, p, p, p, p, p],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib._serving_sigs = True
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Server:
    def __init__(self, grid, max_slots=2048, max_layers=30, max_lambda=400,
                 mem_cap_bytes=16 << 30, chunks_per_tick=8, warps_per_block=4, stream=None):
        self.cfg = ServerConfig(max_slots, max_layers, max_lambda, mem_cap_bytes,
                                chunks_per_tick, warps_per_block)
        g = (grid.c0, grid.dc, grid.n_c) if hasattr(grid, "c0") else tuple(grid)
        gd = masw.GridDesc(float(g[0]), float(g[1]), int(g[2]))
        out = ctypes.c_void_p()
        masw._check(_lib().masw_server_create(ctypes.byref(gd), ctypes.byref(self.cfg),
                                              masw._stream_handle(stream), ctypes.byref(out)),
                    "masw_server_create")
        self.handle = out.value

    def close(self):
        if self.handle:
            masw._check(_lib().masw_server_destroy(ctypes.c_void_p(self.handle)),
                        "masw_server_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, h, alpha, beta, rho, lam) -> int:
        h, alpha, beta, rho, lam = (_f64(x) for x in (h, alpha, beta, rho, lam))
        rid = ctypes.c_int64()
        masw._check(_lib().masw_server_submit(ctypes.c_void_p(self.handle), h.size, _p(h),
                                              _p(alpha), _p(beta), _p(rho), lam.size, _p(lam),
                                              ctypes.byref(rid)), "masw_server_submit")
        return rid.value

    def tick(self) -> int:
        n = ctypes.c_int32()
        masw._check(_lib().masw_server_tick(ctypes.c_void_p(self.handle), ctypes.byref(n)),
                    "masw_server_tick")
        return n.value

    def poll(self, rid: int, n_lambda: int):
        """(ct, idx, status) or None while the request is still running."""
        ct = np.empty(n_lambda)
        idx = np.empty(n_lambda, dtype=np.int32)
        st = np.empty(n_lambda, dtype=np.int32)
        rc = _lib().masw_server_poll(ctypes.c_void_p(self.handle), rid, _p(ct), _p(idx), _p(st))
        if rc == masw.EAGAIN:
            return None
        masw._check(rc, "masw_server_poll")
        return ct, idx, st

    def set_route(self, route: int):
        """Test routing through the slower paths (masw_server_set_route)."""
        f = _lib().masw_server_set_route
        f.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        f.restype = ctypes.c_int
        masw._check(f(ctypes.c_void_p(self.handle), int(route)), "masw_server_set_route")

    PROFILE_KEYS = ("ticks", "upload_scatter_ms", "count_kernel_ms", "tick_kernel_ms",
                    "check_kernel_ms", "readback_ms", "host_launch_ms", "host_finish_ms",
                    "host_admit_ms")

    def profile(self, enable: bool) -> dict:
        """masw_server_profile: start (and zero) or stop the per-tick profile;
        returns the totals so far (device and host milliseconds)."""
        f = _lib().masw_server_profile
        f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        f.restype = ctypes.c_int
        out = np.zeros(len(self.PROFILE_KEYS))
        masw._check(f(ctypes.c_void_p(self.handle), int(bool(enable)), _p(out)),
                    "masw_server_profile")
        return dict(zip(self.PROFILE_KEYS, out.tolist()))

    def stats(self) -> dict:
        s = ServerStats()
        masw._check(_lib().masw_server_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(s)),
                    "masw_server_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def run_trace(self, requests, arrival_s, timeout_s=600.0):
        """Replay the trace natively. Returns (latency_s, ct, idx, status, stats)."""
        nl, nw = _i32(requests.n_layers), _i32(requests.n_lambda)
        h, a, b, r, lam = (_f64(x) for x in (requests.h, requests.alpha, requests.beta,
                                             requests.rho, requests.lam))
        arr = _f64(arrival_s)
        n = nl.size
        lat = np.empty(n)
        ct = np.empty(lam.size)
        idx = np.empty(lam.size, dtype=np.int32)
        st = np.empty(lam.size, dtype=np.int32)
        stats = np.zeros(3, dtype=np.int64)
        masw._check(_lib().masw_server_run_trace(
            ctypes.c_void_p(self.handle), n, _p(nl), _p(h), _p(a), _p(b), _p(r), _p(nw), _p(lam),
            _p(arr), float(timeout_s), _p(lat), _p(ct), _p(idx), _p(st), _p(stats)),
            "masw_server_run_trace")
        return lat, ct, idx, st, {"ticks": int(stats[0]), "refused": int(stats[1]),
                                  "max_in_flight": int(stats[2])}


def latency_summary(lat, arrival_s, n_requests):
    lat = np.asarray(lat)
    span = float(np.max(np.asarray(arrival_s) + lat))
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(np.mean(lat)),
            "curves_per_s": n_requests / span if span > 0 else None}
