"""Seeded synthetic acquisitions: probe and scan geometry plus raw int16
channel data of a scatterer phantom.

This module is the input generator shared by the tests, the benchmark and the
smoke check.  It holds the forward (acquisition) model only -- where the
echoes of a phantom arrive on each element -- and none of the beamforming,
envelope, compression or scan-conversion arithmetic.  The paper's own data
(in-vivo, CIRS phantom, wire tank, Sec. 3) are not available, so these seeded
phantoms stand in for them.

Geometry follows the acquisitions of Sec. 3 and the run-time table (Table 1):
a linear array with 0.3 mm pitch for 2D and a 32x32 matrix array for 3D.
Units: metres, seconds, Hz.  Probe frame: array in the z = 0 plane, x lateral,
y elevation, z depth.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

WINDOWS = {"rect": 0, "hann": 1, "hamming": 2}
GEOMETRIES = {"linear": 0, "sector": 1, "pyramid": 2}


@dataclasses.dataclass
class Setup:
    """A complete acquisition + processing description (plain arrays)."""

    elem_pos: np.ndarray            # [n_el, 3]
    tx_origin: np.ndarray           # [n_tx, 3]
    tx_focus: np.ndarray            # [n_tx, 3] (only the synthesizer uses it)
    line_origin: np.ndarray         # [n_lines, 3]
    line_dir: np.ndarray            # [n_lines, 3] unit
    line_tx: np.ndarray             # [n_lines] int32
    n_depth: int
    depth0: float
    depth_step: float
    geometry: str                   # linear | sector | pyramid
    lines_x: int
    lines_y: int
    c: float
    fs: float
    fc: float
    fnumber: float
    min_half_aperture: float
    window: str
    n_samples: int
    t0: float = 0.0
    fir_taps: int = 63
    fir_cutoff: float = 0.0         # Hz; 0 -> fc / 2
    n_bands: int = 1                # frequency-compounding bank size
    band_step: float = 0.0          # Hz between band centres
    dyn_range_db: float = 60.0
    log_ref: float = 16000.0
    grid: Optional[dict] = None     # {"n": (nx, ny, nz), "origin": (3,), "spacing": (3,)}
    name: str = ""
    tx_dir: Optional[np.ndarray] = None   # [n_tx, 3]: nonzero rows are plane-wave transmits
    compound: int = 0                     # 1: every line averages all transmits

    @property
    def n_el(self) -> int:
        return int(self.elem_pos.shape[0])

    @property
    def n_tx(self) -> int:
        return int(self.tx_origin.shape[0])

    @property
    def n_lines(self) -> int:
        return int(self.line_origin.shape[0])

    @property
    def cutoff(self) -> float:
        return self.fir_cutoff if self.fir_cutoff > 0 else self.fc / 2

    def params(self) -> dict:
        """Keyword arguments accepted by both the oracle and the library binding."""
        d = dict(
            elem_pos=self.elem_pos, tx_origin=self.tx_origin, line_origin=self.line_origin,
            line_dir=self.line_dir, line_tx=self.line_tx, n_depth=self.n_depth, depth0=self.depth0,
            depth_step=self.depth_step, geometry=self.geometry, lines_x=self.lines_x, lines_y=self.lines_y,
            c=self.c, fs=self.fs, fc=self.fc, fnumber=self.fnumber, min_half_aperture=self.min_half_aperture,
            window=self.window, n_samples=self.n_samples, t0=self.t0, fir_taps=self.fir_taps,
            fir_cutoff=self.cutoff, dyn_range_db=self.dyn_range_db, log_ref=self.log_ref, grid=self.grid,
            n_bands=self.n_bands, band_step=self.band_step, tx_dir=self.tx_dir, compound=self.compound)
        return d

    def replace(self, **kw) -> "Setup":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------- probes

def linear_probe(n_el: int, pitch: float) -> np.ndarray:
    x = (np.arange(n_el) - (n_el - 1) / 2.0) * pitch
    return np.stack([x, np.zeros(n_el), np.zeros(n_el)], axis=1)


def matrix_probe(nx: int, ny: int, pitch: float) -> np.ndarray:
    """Row-major: element e = iy * nx + ix."""
    x = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    y = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    xx, yy = np.meshgrid(x, y)
    return np.stack([xx.ravel(), yy.ravel(), np.zeros(nx * ny)], axis=1)


# ----------------------------------------------------------------------------- scans

def linear_setup(n_el=64, pitch=0.3e-3, n_lines=64, n_samples=1024, fc=5e6, fs=40e6, c=1540.0,
                 focus=30e-3, fnumber=1.5, window="hann", grid_n=None, n_depth=None, lines_per_tx=1,
                 name="linear") -> Setup:
    """Linear array, parallel scanlines along +z evenly spaced over the element
    span.  lines_per_tx > 1 reconstructs several lines from one transmit event
    (multi-line receive, Sec. 2 item 1 and Table 1's "(n / 2)" rows); the
    transmit sits at the centre of its lines."""
    elem = linear_probe(n_el, pitch)
    xs = np.linspace(elem[0, 0], elem[-1, 0], n_lines) if n_lines > 1 else np.array([0.0])
    line_origin = np.stack([xs, np.zeros(n_lines), np.zeros(n_lines)], axis=1)
    line_dir = np.tile(np.array([0.0, 0.0, 1.0]), (n_lines, 1))
    n_tx = (n_lines + lines_per_tx - 1) // lines_per_tx
    line_tx = (np.arange(n_lines) // lines_per_tx).astype(np.int32)
    tx_x = np.array([xs[line_tx == t].mean() for t in range(n_tx)])
    tx_origin = np.stack([tx_x, np.zeros(n_tx), np.zeros(n_tx)], axis=1)
    tx_focus = tx_origin + np.array([0.0, 0.0, focus])
    depth_step = c / (2 * fs)
    n_depth = n_samples if n_depth is None else n_depth
    grid = None
    if grid_n is not None:
        nx, nz = grid_n
        zmax = (n_depth - 1) * depth_step
        grid = {"n": (nx, 1, nz), "origin": (xs[0], 0.0, 0.0),
                "spacing": ((xs[-1] - xs[0]) / (nx - 1), 1.0, zmax / (nz - 1))}
    return Setup(elem_pos=elem, tx_origin=tx_origin, tx_focus=tx_focus, line_origin=line_origin,
                 line_dir=line_dir, line_tx=line_tx, n_depth=n_depth, depth0=0.0, depth_step=depth_step,
                 geometry="linear", lines_x=n_lines, lines_y=1, c=c, fs=fs, fc=fc, fnumber=fnumber,
                 min_half_aperture=pitch, window=window, n_samples=n_samples, grid=grid, name=name)


def sector_setup(n_el=64, pitch=0.3e-3, n_lines=64, half_angle_deg=30.0, n_samples=1024, fc=3.5e6, fs=20e6,
                 c=1540.0, focus=30e-3, fnumber=1.5, window="hann", grid_n=None, name="sector") -> Setup:
    """Phased linear array: lines from the array centre at evenly spaced angles
    in the xz plane."""
    elem = linear_probe(n_el, pitch)
    th = np.deg2rad(np.linspace(-half_angle_deg, half_angle_deg, n_lines))
    line_dir = np.stack([np.sin(th), np.zeros(n_lines), np.cos(th)], axis=1)
    line_origin = np.zeros((n_lines, 3))
    line_tx = np.arange(n_lines, dtype=np.int32)
    tx_origin = line_origin.copy()
    tx_focus = tx_origin + focus * line_dir
    depth_step = c / (2 * fs)
    grid = None
    if grid_n is not None:
        nx, nz = grid_n
        rmax = (n_samples - 1) * depth_step
        xh = rmax * math.sin(math.radians(half_angle_deg))
        grid = {"n": (nx, 1, nz), "origin": (-xh, 0.0, 0.0),
                "spacing": (2 * xh / (nx - 1), 1.0, rmax / (nz - 1))}
    return Setup(elem_pos=elem, tx_origin=tx_origin, tx_focus=tx_focus, line_origin=line_origin,
                 line_dir=line_dir, line_tx=line_tx, n_depth=n_samples, depth0=0.0, depth_step=depth_step,
                 geometry="sector", lines_x=n_lines, lines_y=1, c=c, fs=fs, fc=fc, fnumber=fnumber,
                 min_half_aperture=pitch, window=window, n_samples=n_samples, grid=grid, name=name)


def pyramid_setup(nx_el=32, ny_el=32, pitch=0.3e-3, lines_x=64, lines_y=64, half_angle_deg=30.0,
                  n_samples=1536, fc=3.5e6, fs=20e6, c=1540.0, focus=30e-3, fnumber=1.5, window="hann",
                  grid_n=None, name="pyramid") -> Setup:
    """Matrix array, lines from the array centre on a pyramidal sector:
    d = normalize(tan(theta_x), tan(theta_y), 1), line l = iy * lines_x + ix."""
    elem = matrix_probe(nx_el, ny_el, pitch)
    tx = np.deg2rad(np.linspace(-half_angle_deg, half_angle_deg, lines_x))
    ty = np.deg2rad(np.linspace(-half_angle_deg, half_angle_deg, lines_y))
    TY, TX = np.meshgrid(ty, tx, indexing="ij")
    v = np.stack([np.tan(TX).ravel(), np.tan(TY).ravel(), np.ones(lines_x * lines_y)], axis=1)
    line_dir = v / np.linalg.norm(v, axis=1, keepdims=True)
    n_lines = lines_x * lines_y
    line_origin = np.zeros((n_lines, 3))
    line_tx = np.arange(n_lines, dtype=np.int32)
    tx_origin = line_origin.copy()
    tx_focus = tx_origin + focus * line_dir
    depth_step = c / (2 * fs)
    grid = None
    if grid_n is not None:
        gx, gy, gz = grid_n
        zmax = (n_samples - 1) * depth_step
        h = zmax * math.tan(math.radians(half_angle_deg))
        grid = {"n": (gx, gy, gz), "origin": (-h, -h, 0.0),
                "spacing": (2 * h / (gx - 1), 2 * h / (gy - 1), zmax / (gz - 1))}
    return Setup(elem_pos=elem, tx_origin=tx_origin, tx_focus=tx_focus, line_origin=line_origin,
                 line_dir=line_dir, line_tx=line_tx, n_depth=n_samples, depth0=0.0, depth_step=depth_step,
                 geometry="pyramid", lines_x=lines_x, lines_y=lines_y, c=c, fs=fs, fc=fc, fnumber=fnumber,
                 min_half_aperture=pitch, window=window, n_samples=n_samples, grid=grid, name=name)


# ----------------------------------------------------------------------------- the workloads

def config1() -> Setup:
    """2D plain DAS, one frame: 64-element linear array, pitch 0.3 mm, fc 5 MHz,
    fs 40 MHz, 64 focused lines (one per transmit, focus 30 mm), 1024 samples,
    Hann, F# 1.5, RF 64x1024 then 60 dB B-mode (no scan conversion)."""
    return linear_setup(64, 0.3e-3, 64, 1024, fc=5e6, fs=40e6, focus=30e-3, fnumber=1.5,
                        name="2d-linear-64el-64lines-1024s")


def config2() -> Setup:
    """2D full pipeline: 128 elements, fc 7 MHz, fs 40 MHz, 256 lines, 2048
    samples, scan conversion to 512x512 (frames are batched 64 per launch)."""
    return linear_setup(128, 0.3e-3, 256, 2048, fc=7e6, fs=40e6, focus=30e-3, fnumber=1.5,
                        grid_n=(512, 512), name="2d-linear-128el-256lines-2048s-sc512")


def config3(lines=64) -> Setup:
    """3D: 32x32 matrix array, fc 3.5 MHz, fs 20 MHz, lines x lines scanlines on
    a +-30 deg pyramid (one per transmit), 1536 samples, 256^3 volume."""
    return pyramid_setup(32, 32, 0.3e-3, lines, lines, 30.0, 1536, fc=3.5e6, fs=20e6, focus=30e-3,
                         fnumber=1.5, grid_n=(256, 256, 256), name=f"3d-pyramid-1024el-{lines}x{lines}-1536s-vol256")


# ----------------------------------------------------------------------------- phantom

@dataclasses.dataclass
class Phantom:
    pos: np.ndarray   # [n, 3]
    amp: np.ndarray   # [n]


def make_phantom(setup: Setup, seed: int, n_scatter: int, n_points: int = 0, cysts=(),
                 point_amp: float = 30.0) -> Phantom:
    """Uniform random scatterers in the imaged region with Rayleigh(1)
    amplitudes, bright point targets of amplitude point_amp, and anechoic cysts
    (spheres / discs with their scatterers removed).

    2D (linear / sector): scatterers in the y = 0 plane.  3D: inside the
    pyramid.  Point targets: 2D on the central axis evenly over [0.25, 0.9] of
    the imaged depth; 3D a 5x5 lateral grid at half depth."""
    rng = np.random.default_rng(seed)
    zmax = setup.depth0 + (setup.n_depth - 1) * setup.depth_step
    zmin = 1e-3
    if setup.geometry == "linear":
        x0, x1 = setup.line_origin[:, 0].min(), setup.line_origin[:, 0].max()
        pos = np.stack([rng.uniform(x0, x1, n_scatter), np.zeros(n_scatter), rng.uniform(zmin, zmax, n_scatter)], 1)
    elif setup.geometry == "sector":
        th = np.arctan2(setup.line_dir[:, 0], setup.line_dir[:, 2])
        t = rng.uniform(th.min(), th.max(), n_scatter)
        r = np.sqrt(rng.uniform(zmin ** 2, zmax ** 2, n_scatter))
        pos = np.stack([r * np.sin(t), np.zeros(n_scatter), r * np.cos(t)], 1)
    else:
        tx = np.arctan(setup.line_dir[:, 0] / setup.line_dir[:, 2])
        ty = np.arctan(setup.line_dir[:, 1] / setup.line_dir[:, 2])
        ax = rng.uniform(tx.min(), tx.max(), n_scatter)
        ay = rng.uniform(ty.min(), ty.max(), n_scatter)
        r = np.cbrt(rng.uniform(zmin ** 3, zmax ** 3, n_scatter))
        v = np.stack([np.tan(ax), np.tan(ay), np.ones(n_scatter)], 1)
        pos = r[:, None] * v / np.linalg.norm(v, axis=1, keepdims=True)
    amp = rng.rayleigh(1.0, n_scatter)
    keep = np.ones(n_scatter, dtype=bool)
    for (cx, cz, rad) in cysts:
        keep &= (pos[:, 0] - cx) ** 2 + (pos[:, 2] - cz) ** 2 > rad ** 2
    pos, amp = pos[keep], amp[keep]
    if n_points:
        if setup.geometry == "pyramid":
            g = np.linspace(-0.5, 0.5, 5) * zmax * 0.5 * math.tan(math.radians(25))
            gx, gy = np.meshgrid(g, g)
            pts = np.stack([gx.ravel(), gy.ravel(), np.full(25, zmax / 2)], 1)
        else:
            zs = np.linspace(0.25, 0.9, n_points) * zmax
            pts = np.stack([np.zeros(n_points), np.zeros(n_points), zs], 1)
        pos = np.concatenate([pos, pts])
        amp = np.concatenate([amp, np.full(len(pts), point_amp)])
    return Phantom(pos=pos, amp=amp)


def default_phantom(setup: Setup, seed: int) -> Phantom:
    """The phantom of each workload: 2000 scatterers + 5 targets (64-element
    2D), 10000 scatterers + 3 anechoic 4 mm cysts (128-element 2D), 20000
    scatterers + a 5x5 target grid (3D)."""
    if setup.geometry == "pyramid":
        return make_phantom(setup, seed, 20000, n_points=25)
    if setup.n_el >= 128:
        cysts = ((-10e-3, 15e-3, 2e-3), (0.0, 25e-3, 2e-3), (10e-3, 32e-3, 2e-3))
        return make_phantom(setup, seed, 10000, n_points=0, cysts=cysts)
    return make_phantom(setup, seed, 2000, n_points=5)


def synth_channels(setup: Setup, phantom: Phantom, seed: int, device="cpu", snr_db: float = 30.0,
                   peak: float = 16000.0, beam_floor: float = 1e-3, chunk: int = 1 << 21):
    """Raw channel data int16 [n_tx, n_el, n_samples] (torch tensor on device).

    Each scatterer p returns, on element e after transmit t, the pulse
        a * b_t(p) * exp(-(t - T)^2 / (2 s^2)) * cos(2 pi fc (t - T)),
        T = (|p - o_t| + |p - x_e|) / c,  s = (2 / fc) / 2.3548 (FWHM 2 cycles),
    truncated at |t - T| <= 3.5 s.  b_t is a Gaussian transmit beam around the
    axis o_t -> focus: exp(-d^2 / (2 sb^2)), sb = lambda F_tx (1 + |z - z_f| / z_f),
    F_tx = z_f / array width; pairs with b_t < beam_floor are dropped.
    Gaussian noise at snr_db below the noise-free RMS, then scaling so the
    frame peak is `peak`, round half to even, saturation to int16.
    Spreading loss, attenuation and element directivity are left out."""
    import torch

    dev = torch.device(device)
    f64 = torch.float64 if dev.type == "cpu" else torch.float32
    n_tx, n_el, n_s = setup.n_tx, setup.n_el, setup.n_samples
    c, fs, fc = setup.c, setup.fs, setup.fc
    sig = (2.0 / fc) / 2.3548
    half = 3.5 * sig
    J = int(math.ceil(2 * half * fs)) + 2
    lam = c / fc
    width = max(np.ptp(setup.elem_pos[:, 0]), np.ptp(setup.elem_pos[:, 1]), lam)

    P = torch.as_tensor(phantom.pos, dtype=f64, device=dev)
    A = torch.as_tensor(phantom.amp, dtype=f64, device=dev)
    X = torch.as_tensor(setup.elem_pos, dtype=f64, device=dev)
    O = torch.as_tensor(setup.tx_origin, dtype=f64, device=dev)
    Fo = torch.as_tensor(setup.tx_focus, dtype=f64, device=dev)
    buf = torch.zeros(n_tx * n_el * n_s, dtype=torch.float32, device=dev)

    axis = Fo - O
    zf = torch.linalg.norm(axis, dim=1).clamp_min(1e-9)
    axis = axis / zf[:, None]
    Ftx = zf / width
    # plane-wave transmits: arrival n.(p - o_t), the whole field insonified (no focal beam)
    if setup.tx_dir is not None:
        ND = torch.as_tensor(np.asarray(setup.tx_dir, np.float64).reshape(-1, 3), dtype=f64, device=dev)
        nlen = torch.linalg.norm(ND, dim=1)
        plane = nlen > 0
        ND = torch.where(plane[:, None], ND / nlen.clamp_min(1e-30)[:, None], ND)
    else:
        ND = torch.zeros_like(O)
        plane = torch.zeros(n_tx, dtype=torch.bool, device=dev)
    gpu_lists = []   # (transmit, pair) lists for the GPU accumulation
    # transmit beam weight for every (transmit, scatterer), kept where significant
    tx_rows = max(1, (1 << 24) // max(1, P.shape[0]))
    for t0 in range(0, n_tx, tx_rows):
        t1 = min(n_tx, t0 + tx_rows)
        rel = P[None, :, :] - O[t0:t1, None, :]
        z = (rel * axis[t0:t1, None, :]).sum(-1)
        dperp2 = (rel * rel).sum(-1) - z * z
        sb = lam * Ftx[t0:t1, None] * (1 + (z - zf[t0:t1, None]).abs() / zf[t0:t1, None])
        b = torch.exp(-dperp2.clamp_min(0) / (2 * sb * sb))
        b = torch.where(plane[t0:t1, None], torch.ones_like(b), b)
        tt, ss = torch.nonzero(b > beam_floor, as_tuple=True)
        if tt.numel() == 0:
            continue
        amp = (A[ss] * b[tt, ss]).to(f64)
        tt = tt + t0
        if dev.type == "cuda":
            gpu_lists.append((tt, torch.cat([P[ss].float(), amp.float()[:, None]], dim=1)))
            continue
        dtx = torch.where(plane[tt], ((P[ss] - O[tt]) * ND[tt]).sum(-1), torch.linalg.norm(P[ss] - O[tt], dim=1))
        npair = tt.numel()
        pair_rows = max(1, chunk // (n_el * J))
        for p0 in range(0, npair, pair_rows):
            p1 = min(npair, p0 + pair_rows)
            pp = P[ss[p0:p1]]
            T = (dtx[p0:p1, None] + torch.linalg.norm(pp[:, None, :] - X[None, :, :], dim=2)) / c  # [p, e]
            k0 = torch.ceil((T - half) * fs)
            k = k0[..., None] + torch.arange(J, device=dev, dtype=f64)                         # [p, e, J]
            dt = k / fs - T[..., None]
            val = amp[p0:p1, None, None] * torch.exp(-dt * dt / (2 * sig * sig)) * torch.cos(2 * math.pi * fc * dt)
            ok = (k >= 0) & (k < n_s) & (dt.abs() <= half)
            base = (tt[p0:p1, None] * n_el + torch.arange(n_el, device=dev)[None, :]) * n_s     # [p, e]
            idx = base[..., None] + k.long()
            buf.index_add_(0, idx[ok], val[ok].to(torch.float32))

    if dev.type == "cuda" and gpu_lists:
        _gpu_echoes(setup, gpu_lists, sig, half, J, buf, ND.float())

    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 7919 + 17)
    rms = torch.sqrt(torch.mean(buf.double() ** 2)).item()
    if rms > 0 and snr_db is not None:
        sn = rms * 10 ** (-snr_db / 20)
        buf += sn * torch.randn(buf.shape, generator=gen, device=dev, dtype=torch.float32)
    pk = buf.abs().max().item()
    if pk > 0:
        buf *= peak / pk
    out = torch.round(buf).clamp_(-32768, 32767).to(torch.int16)
    return out.view(n_tx, n_el, n_s)


_synth_lib = None


def _gpu_echoes(setup, lists, sig, half, J, buf, tx_dir):
    """Accumulates the echoes of (transmit, scatterer) pairs on the GPU
    (synth_cuda.cu) into buf, float [n_tx * n_el * n_s]."""
    import ctypes

    import torch

    global _synth_lib
    if _synth_lib is None:
        from . import build

        _synth_lib = ctypes.CDLL(build.build())
        _synth_lib.phantom_echoes.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 5 + [ctypes.c_float] * 5 + \
            [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    dev = buf.device
    tt = torch.cat([l[0] for l in lists])
    pairs = torch.cat([l[1] for l in lists]).contiguous()
    order = torch.argsort(tt, stable=True)
    tt, pairs = tt[order], pairs[order].contiguous()
    counts = torch.bincount(tt, minlength=setup.n_tx)
    start = torch.zeros(setup.n_tx + 1, dtype=torch.int32, device=dev)
    start[1:] = torch.cumsum(counts, 0).to(torch.int32)
    elem = torch.as_tensor(setup.elem_pos, dtype=torch.float32, device=dev).contiguous()
    txo = torch.as_tensor(setup.tx_origin, dtype=torch.float32, device=dev).contiguous()
    txd = tx_dir.to(dev).contiguous()
    rc = _synth_lib.phantom_echoes(setup.n_tx, setup.n_el, setup.n_samples, elem.data_ptr(), txo.data_ptr(),
                                   txd.data_ptr(), start.data_ptr(), pairs.data_ptr(), setup.c, setup.fs, setup.fc,
                                   sig, half, J, buf.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    if rc != 0:
        raise RuntimeError(f"phantom_echoes failed with CUDA error {rc}")


def random_channels(setup: Setup, seed: int, amplitude: int = 8000):
    """Uniform random int16 records (no phantom): exercises every sample."""
    import torch

    g = torch.Generator().manual_seed(int(seed))
    return torch.randint(-amplitude, amplitude + 1, (setup.n_tx, setup.n_el, setup.n_samples),
                         generator=g, dtype=torch.int32).to(torch.int16)


# ----------------------------------------------------------------------------- learned apodization inputs

APOD_SIZES = ((64, 128), (64,), (64, 64), (64,), (128, 64), (128,))   # W1, b1, W2, b2, W3, b3


def apod_init(seed: int, out_scale: float = 0.0, bias_scale: float = 0.0) -> np.ndarray:
    """Seeded initial parameters of the per-pixel apodization network, float32
    flat vector in the order W1, b1, W2, b2, W3, b3 ([out][in] row-major).
    Hidden weights: He-normal (std sqrt(2 / fan_in)).  Output weights: normal
    with std out_scale / sqrt(64) (0 -> all-zero output layer, i.e. a uniform
    apodization over the aperture at the start).  Biases: normal with std
    bias_scale."""
    rng = np.random.default_rng(int(seed))
    parts = []
    for k, shape in enumerate(APOD_SIZES):
        if len(shape) == 2:
            std = math.sqrt(2.0 / shape[1]) if k < 4 else out_scale / math.sqrt(shape[1])
        else:
            std = bias_scale
        parts.append((rng.standard_normal(shape) * std).ravel())
    return np.concatenate(parts).astype(np.float32)


def apod_random_batch(seed: int, n: int, min_active: int = 2, n_el: int = 128):
    """Random network inputs for gradient checks: raw samples X[n,128] (bf16
    representable, zero off the mask), masks[n,128] (a contiguous run of at
    least min_active elements, as an F-number aperture gives), norms ||x|| and
    targets t in [-1, 1]."""
    rng = np.random.default_rng(int(seed))
    X = np.zeros((n, 128), np.float32)
    mask = np.zeros((n, 128), bool)
    for b in range(n):
        w = int(rng.integers(min_active, n_el + 1))
        s = int(rng.integers(0, n_el - w + 1))
        mask[b, s:s + w] = True
        X[b, s:s + w] = rng.normal(0.0, 1000.0, w)
    # round to bfloat16 (keep the top 16 bits, round to nearest even)
    u = X.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    X = u.astype(np.uint32).view(np.float32)
    norm = np.sqrt(np.sum(X.astype(np.float64) ** 2, axis=1))
    t = rng.uniform(-1.0, 1.0, n)
    return X, mask, norm, t


def random_cysts(seed: int, n: int = 3, x_mm=(-12.0, 12.0), z_mm=(10.0, 35.0), radius_mm: float = 2.0):
    """Seeded anechoic cyst layout (x, z, radius in metres) for the
    learned-apodization frames: n cysts at random positions, 2 mm radius."""
    rng = np.random.default_rng(int(seed) + 104729)
    xs = rng.uniform(x_mm[0], x_mm[1], n) * 1e-3
    zs = rng.uniform(z_mm[0], z_mm[1], n) * 1e-3
    return tuple((float(x), float(z), radius_mm * 1e-3) for x, z in zip(xs, zs))


def apod_frame(setup: Setup, seed: int, device="cuda"):
    """One frame of the learned-apodization workload: 10000 scatterers, three
    point targets and the seed's cysts.  Returns (channels, cysts)."""
    cysts = random_cysts(seed)
    ph = make_phantom(setup, seed, 10000, n_points=3, cysts=cysts)
    return synth_channels(setup, ph, seed, device=device), cysts


def table1_setup(n_tx: int, lines_per_tx: int, seed_name: str = "") -> Setup:
    """The 2D configurations of the run-time table (Table 1): a 64-channel
    linear array (0.3 mm pitch, fc 5 MHz, fs 40 MHz), 45 mm depth, output on
    a 0.0225 mm isotropic grid; "n_tx / k" = n_tx transmits with k receive
    lines each (multi-line: n_tx * k - (k - 1) lines evenly over the array)."""
    c, fs = 1540.0, 40e6
    n_s = int(math.ceil(45e-3 * 2 / c * fs))
    n_lines = n_tx * lines_per_tx - (lines_per_tx - 1)
    span = 63 * 0.3e-3
    zmax = (n_s - 1) * c / (2 * fs)
    grid_n = (int(round(span / 0.0225e-3)) + 1, int(round(zmax / 0.0225e-3)) + 1)
    return linear_setup(64, 0.3e-3, n_lines, n_s, fc=5e6, fs=fs, c=c, focus=30e-3, fnumber=1.5,
                        lines_per_tx=lines_per_tx, grid_n=grid_n,
                        name=f"2d-linear-64ch-{n_tx}tx-{lines_per_tx}lpt-45mm-grid0.0225mm")



def planewave_setup(n_el=128, pitch=0.3e-3, n_lines=128, n_samples=2048, angles_deg=(-10, -5, 0, 5, 10), fc=5e6,
                    fs=40e6, c=1540.0, fnumber=1.5, window="hann", grid_n=None, name="planewave") -> Setup:
    """Plane-wave imaging with coherent compounding: one plane wave per angle
    (direction (sin a, 0, cos a)), passing the array's first element (a >= 0)
    or last element (a < 0) at time 0 so every element fires at t >= 0; lines
    straight down, evenly over the array; every line averages all angles."""
    s = linear_setup(n_el, pitch, n_lines, n_samples, fc=fc, fs=fs, c=c, fnumber=fnumber, window=window,
                     grid_n=grid_n, name=name)
    th = np.deg2rad(np.asarray(angles_deg, np.float64))
    x0, x1 = s.elem_pos[0, 0], s.elem_pos[-1, 0]
    s.tx_origin = np.stack([np.where(th >= 0, x0, x1), np.zeros_like(th), np.zeros_like(th)], 1)
    s.tx_dir = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], 1)
    s.tx_focus = s.tx_origin + 30e-3 * s.tx_dir   # unused for plane waves
    s.line_tx = np.zeros(n_lines, np.int32)
    s.compound = 1
    return s
