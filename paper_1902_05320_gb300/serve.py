"""Binding of the serving loop (kb_server_* in include/sha3gb.h).

Argument marshalling only; batching, admission and hashing run in the library.
Message and output buffers must be page-locked host memory (numpy arrays are
not: use torch.empty(..., pin_memory=True) or Server.pinned()).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_batch_requests", ctypes.c_uint32), ("max_batch_bytes", ctypes.c_uint64),
                ("long_threshold_perms", ctypes.c_uint64), ("long_lane_kernel", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("message_bytes", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("max_batch_requests_seen", ctypes.c_uint64), ("peak_arena_bytes", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("completion_ring", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("wall_s", ctypes.c_double), ("throughput_rps", ctypes.c_double),
                ("throughput_gbs", ctypes.c_double), ("lat_mean_us", ctypes.c_double),
                ("lat_p50_us", ctypes.c_double), ("lat_p90_us", ctypes.c_double), ("lat_p99_us", ctypes.c_double),
                ("lat_p999_us", ctypes.c_double), ("lat_max_us", ctypes.c_double),
                ("submit_lag_p50_us", ctypes.c_double), ("submit_lag_p99_us", ctypes.c_double),
                ("queue_wait_p50_us", ctypes.c_double), ("queue_wait_p99_us", ctypes.c_double),
                ("service_p50_us", ctypes.c_double), ("service_p99_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


def _lib():
    lib = binding.load()
    if not getattr(lib, "_serve_sigs", False):
        vp, u64 = ctypes.c_void_p, ctypes.c_uint64
        lib.kb_server_create.restype = vp
        lib.kb_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_int)]
        lib.kb_server_destroy.restype = None
        lib.kb_server_destroy.argtypes = [vp]
        lib.kb_server_submit.restype = ctypes.c_int
        lib.kb_server_submit.argtypes = [vp, vp, u64, ctypes.c_int, ctypes.c_uint32, vp,
                                         ctypes.POINTER(ctypes.c_uint64)]
        lib.kb_server_wait.restype = ctypes.c_int
        lib.kb_server_wait.argtypes = [vp, u64, ctypes.c_int]
        lib.kb_server_drain.restype = ctypes.c_int
        lib.kb_server_drain.argtypes = [vp, ctypes.c_int]
        lib.kb_server_replay.restype = ctypes.c_int
        lib.kb_server_replay.argtypes = [vp, vp, vp, vp, vp, vp, vp, u64, vp, vp, ctypes.POINTER(ServerStats)]
        lib._serve_sigs = True
    return lib


def _addr(x) -> int:
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Server:
    """A continuous-batching hash server on the current device."""

    def __init__(self, hbm_budget_bytes: int = 2 << 30, max_inflight: int = 48, max_batch_requests: int = 4096,
                 max_batch_bytes: int = 256 << 20, long_threshold_perms: int = 0,
                 long_lane_parallel: bool = True):
        cfg = ServerConfig(hbm_budget_bytes, max_inflight, max_batch_requests, max_batch_bytes,
                           long_threshold_perms, 0 if long_lane_parallel else 1, 0)
        st = ctypes.c_int(0)
        self._h = _lib().kb_server_create(ctypes.byref(cfg), ctypes.byref(st))
        if not self._h:
            raise binding.Sha3gbError(st.value, "kb_server_create")

    @staticmethod
    def pinned(nbytes: int):
        import torch

        return torch.empty(max(nbytes, 1), dtype=torch.uint8, pin_memory=True)

    def submit(self, msg_addr: int, length: int, variant: int, out_len: int, out_addr: int) -> int:
        ticket = ctypes.c_uint64(0)
        binding._check(_lib().kb_server_submit(self._h, msg_addr, length, variant, out_len, out_addr,
                                               ctypes.byref(ticket)), "kb_server_submit")
        return ticket.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> None:
        binding._check(_lib().kb_server_wait(self._h, ticket, timeout_ms), "kb_server_wait")

    def drain(self, timeout_ms: int = -1) -> None:
        binding._check(_lib().kb_server_drain(self._h, timeout_ms), "kb_server_drain")

    def replay(self, pool, offsets, lens, variants, out_lens, arrival_ns, outputs, latencies=None) -> dict:
        """Submits request i at arrival_ns[i] (ns from the start); pool and
        outputs are pinned tensors; returns the stats as a dict."""
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        lens = np.ascontiguousarray(lens, dtype=np.uint64)
        variants = np.ascontiguousarray(variants, dtype=np.uint8)
        out_lens = np.ascontiguousarray(out_lens, dtype=np.uint32)
        arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        n = offsets.size
        stats = ServerStats()
        lat_addr = None if latencies is None else latencies.ctypes.data
        binding._check(_lib().kb_server_replay(self._h, _addr(pool), offsets.ctypes.data, lens.ctypes.data,
                                               variants.ctypes.data, out_lens.ctypes.data, arrival_ns.ctypes.data,
                                               n, _addr(outputs), lat_addr, ctypes.byref(stats)),
                       "kb_server_replay")
        return stats.as_dict()

    def close(self) -> None:
        if self._h:
            _lib().kb_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
