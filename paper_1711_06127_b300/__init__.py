"""Python binding of libsupra, a B300-native (sm_103a) implementation of the
SUPRA real-time ultrasound chain (arXiv:1711.06127): receive delay-and-sum
beamforming, IQ envelope, log compression and 2D/3D scan conversion.

Argument marshalling only: every step runs in the CUDA kernels of
libsupra.so, reached through the C ABI of include/supra.h with ctypes.
PyTorch supplies device memory and streams.  There is no CPU fallback:
importing works without a GPU, but every compute call needs the built
library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SUPRA_LIBRARY selects another build of the library (the checked test variant,
# libsupra_checked.so); by default the in-tree libsupra.so.
LIB_PATH = os.environ.get("SUPRA_LIBRARY") or os.path.join(_HERE, "libsupra.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EINTERNAL, EWORKSPACE = 0, -1, -2, -3, -4, -5, -6
WINDOWS = {"rect": 0, "hann": 1, "hamming": 2}
GEOMETRIES = {"linear": 0, "sector": 1, "pyramid": 2}

EXPORTS = ("supra_plan_create", "supra_plan_destroy", "supra_plan_get_info", "supra_beamform", "supra_envelope",
           "supra_logcompress", "supra_scanconvert", "supra_bmode_workspace_size", "supra_bmode",
           "supra_bmode_batched", "supra_bmode_noalloc", "supra_mv", "supra_apod_features", "supra_apod_forward",
           "supra_apod_workspace_size", "supra_apod_grad", "supra_apod_adam", "supra_apod_step", "supra_apod_epoch", "supra_apod_mlp",
           "supra_render", "supra_plan_set_max_group", "supra_plan_get_max_group", "supra_autotune_bmode",
           "supra_plan_set_tile_shape", "supra_plan_get_tile_shape", "supra_autotune_tile_shape", "supra_server_create",
           "supra_server_submit", "supra_server_submit_trace", "supra_server_poll", "supra_server_wait",
           "supra_server_release", "supra_server_get_stats", "supra_server_now", "supra_server_destroy",
           "supra_selftest_bounded_wait", "supra_device_status", "supra_strerror", "supra_version")
APOD_PARAMS, APOD_INPUTS = 20736, 128


class SupraError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class _Probe(ctypes.Structure):
    _fields_ = [("n_el", ctypes.c_int32), ("elem_pos", ctypes.POINTER(ctypes.c_double))]


class _Scan(ctypes.Structure):
    _fields_ = [("n_tx", ctypes.c_int32), ("tx_origin", ctypes.POINTER(ctypes.c_double)),
                ("n_lines", ctypes.c_int32), ("line_origin", ctypes.POINTER(ctypes.c_double)),
                ("line_dir", ctypes.POINTER(ctypes.c_double)), ("line_tx", ctypes.POINTER(ctypes.c_int32)),
                ("n_depth", ctypes.c_int32), ("depth0", ctypes.c_double), ("depth_step", ctypes.c_double),
                ("geometry", ctypes.c_int32), ("lines_x", ctypes.c_int32), ("lines_y", ctypes.c_int32),
                ("tx_dir", ctypes.POINTER(ctypes.c_double)), ("compound", ctypes.c_int32)]


class _Rx(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("fs", ctypes.c_double), ("fc", ctypes.c_double),
                ("fnumber", ctypes.c_double), ("min_half_aperture", ctypes.c_double), ("window", ctypes.c_int32),
                ("n_samples", ctypes.c_int32), ("t0", ctypes.c_double)]


class _Post(ctypes.Structure):
    _fields_ = [("fir_taps", ctypes.c_int32), ("fir_cutoff", ctypes.c_double), ("dyn_range_db", ctypes.c_double),
                ("log_ref", ctypes.c_double), ("n_bands", ctypes.c_int32), ("band_step", ctypes.c_double)]


class _TileShape(ctypes.Structure):
    _fields_ = [("frames_per_group", ctypes.c_int32), ("elements_per_stage", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("depth_segments", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3)]


class _Camera(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 3), ("right", ctypes.c_double * 3), ("down", ctypes.c_double * 3),
                ("dir", ctypes.c_double * 3), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_steps", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("alpha", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_tx", ctypes.c_int64), ("n_el", ctypes.c_int64), ("n_samples", ctypes.c_int64),
                ("n_lines", ctypes.c_int64), ("n_depth", ctypes.c_int64), ("channel_bytes", ctypes.c_int64),
                ("aperture_element_samples", ctypes.c_int64), ("aperture_bytes", ctypes.c_int64),
                ("rf_bytes", ctypes.c_int64), ("bmode_bytes", ctypes.c_int64), ("image_bytes", ctypes.c_int64),
                ("has_grid", ctypes.c_int32), ("depth_tile", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsupra.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsupra.so not built at {path}: run `python -m paper_1711_06127_b300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.supra_plan_create.argtypes = [ctypes.POINTER(_Probe), ctypes.POINTER(_Scan), ctypes.POINTER(_Rx),
                                      ctypes.POINTER(_Post), ctypes.POINTER(_Grid), ctypes.POINTER(P)]
    lib.supra_plan_destroy.argtypes = [P]
    lib.supra_plan_destroy.restype = None
    lib.supra_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    for name in ("supra_beamform", "supra_envelope", "supra_logcompress", "supra_scanconvert"):
        getattr(lib, name).argtypes = [P, P, P, P]
    lib.supra_bmode_workspace_size.argtypes = [ctypes.c_int32, ctypes.POINTER(P)]
    lib.supra_bmode_workspace_size.restype = ctypes.c_size_t
    lib.supra_bmode.argtypes = [P, P, P, P, ctypes.c_size_t, P]
    lib.supra_bmode_batched.argtypes = [ctypes.c_int32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P,
                                        ctypes.c_size_t, P]
    lib.supra_bmode_noalloc.argtypes = [P, P, P, P]
    lib.supra_mv.argtypes = [P, ctypes.c_int32, ctypes.c_float, P, P, P]
    I64, F = ctypes.c_int64, ctypes.c_float
    lib.supra_apod_features.argtypes = [P, P, P, P, P, P]
    lib.supra_apod_forward.argtypes = [P, I64, I64, P, P, P, P, P]
    lib.supra_apod_workspace_size.argtypes = []
    lib.supra_apod_workspace_size.restype = ctypes.c_size_t
    lib.supra_apod_grad.argtypes = [P, I64, I64, P, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.supra_apod_adam.argtypes = [P, P, P, P, ctypes.c_int32, F, F, F, F, P]
    lib.supra_apod_step.argtypes = [P, P, P, ctypes.c_int32, F, F, F, F, I64, I64, P, P, P, P, P, P, P,
                                    ctypes.c_size_t, P]
    lib.supra_apod_epoch.argtypes = [P, P, P, ctypes.c_int32, F, F, F, F, I64, ctypes.c_int32, ctypes.c_int32, P,
                                     P, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.supra_apod_mlp.argtypes = [P, P, P, P, P]
    lib.supra_render.argtypes = [ctypes.POINTER(_Grid), P, ctypes.POINTER(_Camera), P, P]
    lib.supra_plan_set_max_group.argtypes = [P, ctypes.c_int32]
    lib.supra_plan_get_max_group.argtypes = [P]
    lib.supra_autotune_bmode.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P), ctypes.POINTER(P), P, ctypes.c_size_t,
                                         ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_float)]
    lib.supra_plan_set_tile_shape.argtypes = [P, ctypes.POINTER(_TileShape)]
    lib.supra_plan_get_tile_shape.argtypes = [P, ctypes.POINTER(_TileShape)]
    lib.supra_autotune_tile_shape.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P), ctypes.POINTER(P), P,
                                              ctypes.c_size_t, ctypes.c_int32, P, ctypes.POINTER(_TileShape),
                                              ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.supra_selftest_bounded_wait.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
    lib.supra_device_status.argtypes = [ctypes.c_int32]
    lib.supra_strerror.argtypes = [ctypes.c_int]
    lib.supra_strerror.restype = ctypes.c_char_p
    lib.supra_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().supra_strerror(code).decode()
    except Exception:
        return "unknown error"


def _check(code: int, what: str):
    if code != 0:
        raise SupraError(code, what)


def _stream_ptr(stream) -> Optional[int]:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_tensor(t, dtype, shape, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Plan:
    """A resident plan: geometry, delay bases, aperture bounds, taps and the
    scan-conversion map, built once (Sec. 2: parameters computed once for a
    fixed acquisition).  Keyword arguments as produced by
    phantom.Setup.params()."""

    def __init__(self, *, elem_pos, tx_origin, line_origin, line_dir, line_tx, n_depth, depth0, depth_step,
                 geometry="linear", lines_x=None, lines_y=1, c, fs, fc, fnumber, min_half_aperture, window="hann",
                 n_samples, t0=0.0, fir_taps=63, fir_cutoff=None, dyn_range_db=60.0, log_ref=16000.0, grid=None,
                 n_bands=1, band_step=0.0, tx_dir=None, compound=0, **_ignored):
        lib = load()
        self._keep = []

        def dp(a, dt=np.float64, cols=3):
            arr = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(arr)
            ct = ctypes.c_double if dt == np.float64 else ctypes.c_int32
            return arr, arr.ctypes.data_as(ctypes.POINTER(ct))

        ep, ep_p = dp(elem_pos)
        tx, tx_p = dp(tx_origin)
        lo, lo_p = dp(line_origin)
        ld, ld_p = dp(line_dir)
        lt, lt_p = dp(line_tx, np.int32)
        n_lines = lo.shape[0]
        self.n_el, self.n_tx, self.n_lines = ep.shape[0], tx.shape[0], n_lines
        self.n_depth, self.n_samples = int(n_depth), int(n_samples)
        self.probe = _Probe(ep.shape[0], ep_p)
        td_p = None
        if tx_dir is not None:
            td, td_p = dp(np.asarray(tx_dir, np.float64).reshape(-1, 3))
            if td.shape[0] != tx.shape[0]:
                raise ValueError("tx_dir must have one row per transmit")
        self.compound = int(compound or 0)
        self.scan = _Scan(tx.shape[0], tx_p, n_lines, lo_p, ld_p, lt_p, int(n_depth), float(depth0),
                          float(depth_step), GEOMETRIES[geometry] if isinstance(geometry, str) else int(geometry),
                          int(n_lines if lines_x is None else lines_x), int(lines_y), td_p, self.compound)
        self.rx = _Rx(float(c), float(fs), float(fc), float(fnumber), float(min_half_aperture),
                      WINDOWS[window] if isinstance(window, str) else int(window), int(n_samples), float(t0))
        self.post = _Post(int(fir_taps), float(fc / 2 if fir_cutoff is None else fir_cutoff), float(dyn_range_db),
                          float(log_ref), int(n_bands or 1), float(band_step or 0.0))
        self.grid = None
        gptr = None
        if grid is not None:
            n = grid["n"]
            self.grid = _Grid(int(n[0]), int(n[1]), int(n[2]), (ctypes.c_double * 3)(*grid["origin"]),
                              (ctypes.c_double * 3)(*grid["spacing"]))
            gptr = ctypes.byref(self.grid)
        h = ctypes.c_void_p()
        _check(lib.supra_plan_create(ctypes.byref(self.probe), ctypes.byref(self.scan), ctypes.byref(self.rx),
                                     ctypes.byref(self.post), gptr, ctypes.byref(h)), "supra_plan_create")
        self.handle = h
        inf = PlanInfo()
        _check(lib.supra_plan_get_info(h, ctypes.byref(inf)), "supra_plan_get_info")
        self.info = inf.as_dict()
        self.image_shape = None
        if grid is not None:
            nx, ny, nz = (int(v) for v in grid["n"])
            self.image_shape = (nz, nx) if ny == 1 else (nz, ny, nx)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().supra_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ch_shape(self):
        return (self.n_tx, self.n_el, self.n_samples)

    @property
    def line_shape(self):
        return (self.n_lines, self.n_depth)

    @property
    def out_shape(self):
        return self.image_shape if self.image_shape is not None else self.line_shape

    # ---- the four nodes of Table 1 ---------------------------------------
    def beamform(self, ch, rf=None, stream=None):
        import torch

        if rf is None:
            rf = torch.empty(self.line_shape, dtype=torch.float32, device=ch.device)
        _check(load().supra_beamform(self.handle, _dev_tensor(ch, torch.int16, self.ch_shape, "ch"),
                                     _dev_tensor(rf, torch.float32, self.line_shape, "rf"), _stream_ptr(stream)),
               "supra_beamform")
        return rf

    def envelope(self, rf, env=None, stream=None):
        import torch

        if env is None:
            env = torch.empty(self.line_shape, dtype=torch.float32, device=rf.device)
        _check(load().supra_envelope(self.handle, _dev_tensor(rf, torch.float32, self.line_shape, "rf"),
                                     _dev_tensor(env, torch.float32, self.line_shape, "env"), _stream_ptr(stream)),
               "supra_envelope")
        return env

    def logcompress(self, env, bm=None, stream=None):
        import torch

        if bm is None:
            bm = torch.empty(self.line_shape, dtype=torch.uint8, device=env.device)
        _check(load().supra_logcompress(self.handle, _dev_tensor(env, torch.float32, self.line_shape, "env"),
                                        _dev_tensor(bm, torch.uint8, self.line_shape, "bm"), _stream_ptr(stream)),
               "supra_logcompress")
        return bm

    def scanconvert(self, bm, img=None, stream=None):
        import torch

        if self.image_shape is None:
            raise ValueError("plan has no output grid")
        if img is None:
            img = torch.empty(self.image_shape, dtype=torch.uint8, device=bm.device)
        _check(load().supra_scanconvert(self.handle, _dev_tensor(bm, torch.uint8, self.line_shape, "bm"),
                                        _dev_tensor(img, torch.uint8, self.image_shape, "img"), _stream_ptr(stream)),
               "supra_scanconvert")
        return img

    def mv(self, ch, subaperture=32, loading=None, rf=None, stream=None):
        """Exact minimum-variance beamformer (supra_mv); loading (relative to the
        mean eigenvalue of the covariance) defaults to 0.01."""
        import torch

        if loading is None:
            loading = 0.01
        if rf is None:
            rf = torch.empty(self.line_shape, dtype=torch.float32, device=ch.device)
        _check(load().supra_mv(self.handle, int(subaperture), float(loading),
                               _dev_tensor(ch, torch.int16, self.ch_shape, "ch"),
                               _dev_tensor(rf, torch.float32, self.line_shape, "rf"), _stream_ptr(stream)), "supra_mv")
        return rf

    def apod(self, ch, params, rf=None, stream=None):
        """Learned-apodization beamformer (supra_apod_mlp): params float32
        [APOD_PARAMS] on the device."""
        import torch

        if rf is None:
            rf = torch.empty(self.line_shape, dtype=torch.float32, device=ch.device)
        _check(load().supra_apod_mlp(self.handle, _dev_tensor(params, torch.float32, (APOD_PARAMS,), "params"),
                                     _dev_tensor(ch, torch.int16, self.ch_shape, "ch"),
                                     _dev_tensor(rf, torch.float32, self.line_shape, "rf"), _stream_ptr(stream)),
               "supra_apod_mlp")
        return rf

    def apod_features(self, ch, feat=None, mask=None, norm=None, stream=None):
        """Network inputs of every pixel (supra_apod_features): feat bfloat16
        [n_lines * n_depth, 128] (x / ||x||), mask int32 [.., 4] (aperture
        bits), norm float32 [..]."""
        import torch

        P = self.n_lines * self.n_depth
        dev = ch.device
        feat = torch.empty((P, APOD_INPUTS), dtype=torch.bfloat16, device=dev) if feat is None else feat
        mask = torch.empty((P, 4), dtype=torch.int32, device=dev) if mask is None else mask
        norm = torch.empty((P,), dtype=torch.float32, device=dev) if norm is None else norm
        _check(load().supra_apod_features(self.handle, _dev_tensor(ch, torch.int16, self.ch_shape, "ch"),
                                          _dev_tensor(feat, torch.bfloat16, (P, APOD_INPUTS), "feat"),
                                          _dev_tensor(mask, torch.int32, (P, 4), "mask"),
                                          _dev_tensor(norm, torch.float32, (P,), "norm"), _stream_ptr(stream)),
               "supra_apod_features")
        return feat, mask, norm

    # ---- tuning ------------------------------------------------------------
    @property
    def tile_shape(self) -> dict:
        s = _TileShape()
        _check(load().supra_plan_get_tile_shape(self.handle, ctypes.byref(s)), "supra_plan_get_tile_shape")
        return {k: int(getattr(s, k)) for k, _ in _TileShape._fields_}

    @tile_shape.setter
    def tile_shape(self, shape: dict):
        cur = self.tile_shape
        cur.update(shape)
        s = _TileShape(**{k: int(v) for k, v in cur.items()})
        _check(load().supra_plan_set_tile_shape(self.handle, ctypes.byref(s)), "supra_plan_set_tile_shape")

    def autotune_shape(self, chs, outs=None, workspace=None, reps=3, stream=None):
        """Times the fused chain on these frames (device tensors of this plan)
        for the shape in effect and each candidate tile shape, keeps the
        fastest; returns (shape, ms, ms of the shape in effect before)."""
        import torch

        n = len(chs)
        outs = [torch.empty(self.out_shape, dtype=torch.uint8, device=c.device) for c in chs] if outs is None else outs
        need = workspace_size([self] * n)
        if need and workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=chs[0].device)
        PA = ctypes.c_void_p * n
        ca = PA(*[_dev_tensor(c, torch.int16, self.ch_shape, "ch") for c in chs])
        oa = PA(*[_dev_tensor(o, torch.uint8, self.out_shape, "out") for o in outs])
        s, ms, ms0 = _TileShape(), ctypes.c_float(), ctypes.c_float()
        _check(load().supra_autotune_tile_shape(self.handle, n, ca, oa,
                                                workspace.data_ptr() if workspace is not None else None, need,
                                                int(reps), _stream_ptr(stream), ctypes.byref(s), ctypes.byref(ms),
                                                ctypes.byref(ms0)), "supra_autotune_tile_shape")
        return {k: int(getattr(s, k)) for k, _ in _TileShape._fields_}, float(ms.value), float(ms0.value)

    @property
    def max_group(self) -> int:
        return int(load().supra_plan_get_max_group(self.handle))

    @max_group.setter
    def max_group(self, g: int):
        _check(load().supra_plan_set_max_group(self.handle, int(g)), "supra_plan_set_max_group")

    def autotune(self, chs, outs=None, workspace=None, reps=3, stream=None):
        """Times the fused chain on these frames (device tensors of this plan)
        for each frames-per-tile class, keeps the fastest; returns (G, ms)."""
        import torch

        n = len(chs)
        outs = [torch.empty(self.out_shape, dtype=torch.uint8, device=c.device) for c in chs] if outs is None else outs
        need = workspace_size([self] * n)
        if need and workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=chs[0].device)
        PA = ctypes.c_void_p * n
        ca = PA(*[_dev_tensor(c, torch.int16, self.ch_shape, "ch") for c in chs])
        oa = PA(*[_dev_tensor(o, torch.uint8, self.out_shape, "out") for o in outs])
        g, ms = ctypes.c_int32(), ctypes.c_float()
        _check(load().supra_autotune_bmode(self.handle, n, ca, oa, workspace.data_ptr() if workspace is not None else None,
                                           need, int(reps), _stream_ptr(stream), ctypes.byref(g), ctypes.byref(ms)),
               "supra_autotune_bmode")
        return int(g.value), float(ms.value)

    # ---- fused chain -----------------------------------------------------
    def bmode(self, ch, out=None, workspace=None, stream=None):
        return bmode_batched([self], [ch], None if out is None else [out], workspace, stream)[0]


def workspace_size(plans: Sequence[Plan]) -> int:
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    return int(load().supra_bmode_workspace_size(len(plans), arr))


def bmode_batched(plans: Sequence[Plan], chs, outs=None, workspace=None, stream=None):
    """Fused chain over n frames (frames of one plan that are adjacent are
    beamformed together).  Returns the output tensors."""
    import torch

    n = len(plans)
    if n != len(chs):
        raise ValueError("plans and chs differ in length")
    if outs is None:
        outs = [torch.empty(p.out_shape, dtype=torch.uint8, device=c.device) for p, c in zip(plans, chs)]
    need = workspace_size(plans)
    if need and workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=chs[0].device)
    wptr = workspace.data_ptr() if workspace is not None else None
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    P = ctypes.c_void_p * n
    pa = P(*[p.handle.value for p in plans])
    ca = P(*[_dev_tensor(c, torch.int16, p.ch_shape, "ch") for p, c in zip(plans, chs)])
    oa = P(*[_dev_tensor(o, torch.uint8, p.out_shape, "out") for p, o in zip(plans, outs)])
    _check(load().supra_bmode_batched(n, pa, ca, oa, wptr, wbytes, _stream_ptr(stream)), "supra_bmode_batched")
    return outs


def render(vol, grid: dict, camera: dict, width: int, height: int, mode: str = "mip", lo: float = 0.0,
           hi: float = 255.0, alpha: float = 1.0, image=None, stream=None):
    """Headless volume rendering (supra_render) of a uint8 volume [nz][ny][nx]
    on `grid` ({"n", "origin", "spacing"}); camera: centre, right, down, dir
    (3-vectors, metres), t0, dt, n_steps.  Returns float [height, width]."""
    import torch

    n = grid["n"]
    g = _Grid(int(n[0]), int(n[1]), int(n[2]), (ctypes.c_double * 3)(*grid["origin"]),
              (ctypes.c_double * 3)(*grid["spacing"]))
    v3 = lambda k: (ctypes.c_double * 3)(*[float(x) for x in camera[k]])
    cam = _Camera(v3("centre"), v3("right"), v3("down"), v3("dir"), float(camera["t0"]), float(camera["dt"]),
                  int(camera["n_steps"]), int(width), int(height), {"mip": 0, "ea": 1}[mode], float(lo), float(hi),
                  float(alpha))
    if image is None:
        image = torch.empty((height, width), dtype=torch.float32, device=vol.device)
    _check(load().supra_render(ctypes.byref(g), _dev_tensor(vol, torch.uint8, (int(n[2]), int(n[1]), int(n[0])), "vol"),
                               ctypes.byref(cam), _dev_tensor(image, torch.float32, (height, width), "image"),
                               _stream_ptr(stream)), "supra_render")
    return image


def device_status(clear: bool = True) -> int:
    """Device-side failure code since the last clear (0 = none); synchronizes."""
    return int(load().supra_device_status(1 if clear else 0))


def selftest_bounded_wait(budget_cycles: int = 1 << 20) -> tuple:
    """Runs the bounded-wait self-test (an mbarrier that never completes, waited on
    with a cycle budget and with the abort-word path); returns the two waits' timeout
    flags.  The device status word is left at ETIMEOUT for the caller to read."""
    out = (ctypes.c_int32 * 2)()
    _check(load().supra_selftest_bounded_wait(int(budget_cycles), out), "supra_selftest_bounded_wait")
    return int(out[0]), int(out[1])


def version() -> str:
    return load().supra_version().decode()
