"""Binding of the real-time request loop (supra_server_* in include/supra.h):
memory-admitted continuous batching of B-mode requests over resident plans,
by delay-and-sum, minimum variance or learned apodization.  Marshalling only;
the loop itself (admission, batching, streams, graphs, completion times) runs
in libsupra's native worker thread."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, load

KINDS = {"das": 0, "mv": 1, "apod": 2}


class _Config(ctypes.Structure):
    _fields_ = [("memory_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("plan", ctypes.c_void_p), ("ch", ctypes.c_void_p),
                ("ch_host", ctypes.c_void_p), ("out_host", ctypes.c_void_p), ("apod_params", ctypes.c_void_p),
                ("mv_subaperture", ctypes.c_int32), ("mv_loading", ctypes.c_float), ("tag", ctypes.c_int64)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("tag", ctypes.c_int64), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("out", ctypes.c_void_p), ("out_bytes", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("graph_instantiations", ctypes.c_int64),
                ("graph_updates", ctypes.c_int64), ("memory_used", ctypes.c_int64), ("memory_peak", ctypes.c_int64),
                ("pending", ctypes.c_int32), ("inflight", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _lib():
    lib = load()
    if not getattr(lib, "_server_types", False):
        P = ctypes.c_void_p
        lib.supra_server_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(P)]
        lib.supra_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]
        lib.supra_server_submit_trace.argtypes = [P, ctypes.c_int32, ctypes.POINTER(Request),
                                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.supra_server_poll.argtypes = [P, ctypes.POINTER(Completion), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]
        lib.supra_server_wait.argtypes = [P, ctypes.c_int64, ctypes.c_double]
        lib.supra_server_release.argtypes = [P, ctypes.c_int64]
        lib.supra_server_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        lib.supra_server_now.argtypes = [P]
        lib.supra_server_now.restype = ctypes.c_double
        lib.supra_server_destroy.argtypes = [P]
        lib.supra_server_destroy.restype = None
        lib._server_types = True
    return lib


class _DeviceBytes:
    """Zero-copy view of device bytes for torch.as_tensor."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(int(v) for v in shape), "typestr": "|u1",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Server:
    """A running request loop on the current CUDA device."""

    def __init__(self, memory_bytes: int, n_streams: int = 4, max_batch: int = 16, use_graphs: bool = True):
        self._h = ctypes.c_void_p()
        cfg = _Config(int(memory_bytes), int(n_streams), int(max_batch), 1 if use_graphs else 0)
        _check(_lib().supra_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "supra_server_create")
        self._keep = {}   # ticket -> objects the request refers to
        self.submitted = 0

    @staticmethod
    def request(kind, plan, ch=None, ch_host=None, out_host=None, apod_params=None, mv_subaperture=32,
                mv_loading=0.01, tag=0) -> Request:
        ptr = lambda t: None if t is None else t.data_ptr()
        return Request(KINDS[kind] if isinstance(kind, str) else int(kind), plan.handle.value, ptr(ch),
                       ptr(ch_host), ptr(out_host), ptr(apod_params), int(mv_subaperture), float(mv_loading),
                       int(tag))

    def submit(self, kind, plan, keep=(), **kw) -> int:
        r = self.request(kind, plan, **kw)
        t = ctypes.c_int64()
        _check(_lib().supra_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "supra_server_submit")
        self._keep[t.value] = (plan, kw, keep)
        self.submitted += 1
        return t.value

    def submit_trace(self, reqs, t_arrival, keep=()) -> list:
        """reqs: list of (kind, plan, kwargs); t_arrival: seconds from now."""
        n = len(reqs)
        arr = (Request * n)(*[self.request(k, p, **kw) for k, p, kw in reqs])
        ts = (ctypes.c_double * n)(*[float(x) for x in t_arrival])
        tk = (ctypes.c_int64 * n)()
        _check(_lib().supra_server_submit_trace(self._h, n, arr, ts, tk), "supra_server_submit_trace")
        tickets = list(tk)
        for t, r in zip(tickets, reqs):
            self._keep[t] = (r, keep)
        self.submitted += n
        return tickets

    def poll(self, max_n: int = 4096) -> list:
        buf = (Completion * max_n)()
        n = ctypes.c_int32()
        _check(_lib().supra_server_poll(self._h, buf, max_n, ctypes.byref(n)), "supra_server_poll")
        out = [buf[i].as_dict() for i in range(n.value)]
        for c in out:
            if c["out"] is None:
                self._keep.pop(c["ticket"], None)
        return out

    def wait(self, timeout_s: float = 600.0):
        _check(_lib().supra_server_wait(self._h, self.submitted, float(timeout_s)), "supra_server_wait")

    def release(self, ticket: int):
        _check(_lib().supra_server_release(self._h, int(ticket)), "supra_server_release")
        self._keep.pop(ticket, None)

    def result(self, completion: dict, shape):
        """Copy of a result kept on the device (uint8 tensor of `shape`)."""
        import torch

        n = int(np.prod(shape))
        if completion["out"] is None or completion["out_bytes"] != n:
            raise ValueError("no device result of that size")
        return torch.as_tensor(_DeviceBytes(completion["out"], shape), device="cuda").clone()

    def stats(self) -> dict:
        st = Stats()
        _check(_lib().supra_server_get_stats(self._h, ctypes.byref(st)), "supra_server_get_stats")
        return st.as_dict()

    def now(self) -> float:
        return float(_lib().supra_server_now(self._h))

    def close(self):
        if self._h is not None and self._h.value:
            _lib().supra_server_destroy(self._h)
            self._h = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
