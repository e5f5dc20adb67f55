"""GPU parity of every node of the chain against the FP64 oracle, through the
C ABI (Sec. 1 step list, Sec. 2 items 1-5, Table 1 nodes).  Sizes span several
depth tiles with ragged tails; edge cases: single element, multi-line
transmits, record start t0 > 0, coarse depth steps, unaligned records (the
plain-load staging path), sector and pyramid layouts, windows with a hard
aperture edge."""
import numpy as np
import pytest
import torch

import oracle
import paper_1711_06127_b300 as supra
import phantom
from _setups import small_linear, tiny
from gpu_util import ENV_TOL, RF_TOL, assert_gray, max_norm_err

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _built():
    from paper_1711_06127_b300 import build

    build.build()
    supra.load()
    yield
    assert supra.device_status() == 0


def gpu_rf(p, ch):
    plan = supra.Plan(**p)
    rf = plan.beamform(torch.as_tensor(np.asarray(ch)).cuda())
    torch.cuda.synchronize()
    return rf.cpu().numpy().astype(np.float64)


def setups():
    out = {
        "linear16_ragged": small_linear(16, 12, 300),
        "linear_phantom": small_linear(32, 24, 700),
        "sector": phantom.sector_setup(24, 0.3e-3, 17, 35.0, 350, fc=3.5e6, fs=20e6),
        "pyramid": phantom.pyramid_setup(8, 8, 0.3e-3, 5, 4, 25.0, 260, fc=3.5e6, fs=20e6),
        "multiline": phantom.linear_setup(16, 0.3e-3, 31, 400, fc=5e6, fs=40e6, lines_per_tx=2),
        "single_element": phantom.linear_setup(1, 0.3e-3, 1, 200, fc=5e6, fs=40e6),
        "unaligned_ns": small_linear(12, 8, 301),
    }
    return out


@pytest.mark.parametrize("name", list(setups().keys()))
def test_beamform_matches_oracle(name):
    s = setups()[name]
    p = s.params()
    if name == "linear_phantom":
        ch = phantom.synth_channels(s, phantom.default_phantom(s, 11), 11).numpy()
    else:
        ch = phantom.random_channels(s, 3).numpy()
    ref = oracle.das(p, ch)
    got = gpu_rf(p, ch)
    assert max_norm_err(got, ref) <= RF_TOL


def test_beamform_config1_full_size():
    s = phantom.config1()
    p = s.params()
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 1), 1).numpy()
    assert max_norm_err(gpu_rf(p, ch), oracle.das(p, ch)) <= RF_TOL


def test_beamform_record_start_and_coarse_depth():
    s = small_linear(16, 10, 400)
    p = s.params()
    p.update(t0=37.3 / s.fs, depth0=0.7e-3, depth_step=1.5 * s.c / (2 * s.fs), n_depth=250)
    ch = phantom.random_channels(s, 5).numpy()
    assert max_norm_err(gpu_rf(p, ch), oracle.das(p, ch)) <= RF_TOL


def test_beamform_unaligned_record_pointer():
    s = small_linear(16, 10, 256)
    p = s.params()
    ch = phantom.random_channels(s, 6)
    buf = torch.zeros(ch.numel() + 1, dtype=torch.int16, device="cuda")
    view = buf[1:].view(ch.shape)
    view.copy_(ch.cuda())
    plan = supra.Plan(**p)
    rf = plan.beamform(view).cpu().numpy()
    assert max_norm_err(rf, oracle.das(p, ch.numpy())) <= RF_TOL


@pytest.mark.parametrize("window", ["rect", "hamming"])
def test_beamform_hard_edge_windows(window):
    # A hard aperture edge makes the sum jump when an element crosses it; samples
    # whose aperture has an element within 1e-9 m of the edge are decided by
    # rounding and are left out (fp32 and fp64 may place it on either side).
    s = small_linear(16, 9, 260, window=window)
    p = s.params()
    ch = phantom.random_channels(s, 8).numpy()
    ref = oracle.das(p, ch)
    got = gpu_rf(p, ch)
    keep = np.ones_like(ref, bool)
    for l in range(s.n_lines):
        for i in range(s.n_depth):
            _, _, margin = oracle.aperture(p, l, i)
            keep[l, i] = np.min(np.abs(margin)) > 1e-9
    assert keep.mean() > 0.9
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)[keep]) / scale <= RF_TOL


def test_envelope_matches_oracle():
    s = small_linear(16, 12, 700)
    p = s.params()
    rf = np.random.default_rng(0).normal(size=(s.n_lines, s.n_depth)).astype(np.float32)
    ref = oracle.envelope(p, rf.astype(np.float64))
    plan = supra.Plan(**p)
    got = plan.envelope(torch.as_tensor(rf).cuda()).cpu().numpy()
    assert max_norm_err(got, ref) <= ENV_TOL


def test_logcompress_matches_oracle():
    s = small_linear(16, 12, 700)
    p = s.params()
    env = np.exp(np.random.default_rng(1).uniform(-2, 11, (s.n_lines, s.n_depth))).astype(np.float32)
    env[0, :5] = 0.0
    ref = oracle.logcompress(env.astype(np.float64), p["log_ref"], p["dyn_range_db"])
    plan = supra.Plan(**p)
    got = plan.logcompress(torch.as_tensor(env).cuda()).cpu().numpy()
    d = np.abs(got.astype(int) - ref.astype(int))
    assert d.max() <= 1 and np.mean(d == 0) >= 0.999


@pytest.mark.parametrize("kind", ["linear", "sector", "pyramid"])
def test_scanconvert_matches_oracle(kind):
    if kind == "linear":
        s = phantom.linear_setup(32, 0.3e-3, 64, 500, grid_n=(123, 201))
    elif kind == "sector":
        s = phantom.sector_setup(32, 0.3e-3, 48, 40.0, 400, grid_n=(150, 130))
    else:
        s = phantom.pyramid_setup(8, 8, 0.3e-3, 12, 10, 30.0, 300, grid_n=(41, 37, 53))
    p = s.params()
    bm = np.random.default_rng(2).integers(0, 256, (s.n_lines, s.n_depth)).astype(np.uint8)
    ref = oracle.scanconvert(p, bm)
    ref = ref[:, 0, :] if p["grid"]["n"][1] == 1 else ref
    plan = supra.Plan(**p)
    got = plan.scanconvert(torch.as_tensor(bm).cuda()).cpu().numpy()
    assert got.shape == ref.shape
    assert_gray(got, ref, what=kind)
    assert np.abs(got.astype(int) - ref.astype(int)).max() <= 1


def test_scanconvert_identity_grid_is_exact():
    s = phantom.linear_setup(16, 0.3e-3, 16, 300)
    p = s.params()
    xs = s.line_origin[:, 0]
    p["grid"] = {"n": (16, 1, 300), "origin": (xs[0], 0.0, 0.0), "spacing": (xs[1] - xs[0], 1.0, s.depth_step)}
    bm = np.random.default_rng(4).integers(0, 256, (16, 300)).astype(np.uint8)
    plan = supra.Plan(**p)
    got = plan.scanconvert(torch.as_tensor(bm).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, bm.T)


def _chain_case(name):
    if name == "linear_lines":
        s = small_linear(32, 24, 700)
    elif name == "linear_image":
        s = phantom.linear_setup(48, 0.3e-3, 64, 900, fc=7e6, fs=40e6, grid_n=(140, 190))
    elif name == "sector_image":
        s = phantom.sector_setup(32, 0.3e-3, 40, 35.0, 600, fc=3.5e6, fs=20e6, grid_n=(160, 150))
    else:
        s = phantom.pyramid_setup(8, 8, 0.3e-3, 10, 9, 30.0, 400, fc=3.5e6, fs=20e6, grid_n=(40, 36, 50))
    p = s.params()
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 21, 1500, n_points=3), 21).numpy()
    ref = oracle.bmode(p, ch)
    return s, p, ch, ref


@pytest.mark.parametrize("name", ["linear_lines", "linear_image", "sector_image", "pyramid_volume"])
def test_fused_bmode_matches_oracle(name):
    s, p, ch, ref = _chain_case(name)
    plan = supra.Plan(**p)
    got = plan.bmode(torch.as_tensor(ch).cuda()).cpu().numpy()
    assert got.shape == ref.shape
    assert_gray(got, ref, what=name)


def test_fused_equals_unfused_chain():
    s = phantom.linear_setup(48, 0.3e-3, 64, 900, fc=7e6, fs=40e6, grid_n=(140, 190))
    p = s.params()
    ch = torch.as_tensor(phantom.synth_channels(s, phantom.default_phantom(s, 5), 5)).cuda()
    plan = supra.Plan(**p)
    img_unfused = plan.scanconvert(plan.logcompress(plan.envelope(plan.beamform(ch))))
    img_fused = plan.bmode(ch)
    assert_gray(img_fused.cpu().numpy(), img_unfused.cpu().numpy(), frac=0.9999, what="fused vs unfused")


def test_batched_uneven_frames_equal_single_frames():
    a = phantom.linear_setup(32, 0.3e-3, 40, 600, fc=7e6, fs=40e6, grid_n=(100, 120))
    b = phantom.sector_setup(24, 0.3e-3, 30, 35.0, 500, fc=3.5e6, fs=20e6)   # no grid: lines out
    pa, pb = supra.Plan(**a.params()), supra.Plan(**b.params())
    plans = [pa, pa, pa, pb, pa, pb, pb, pa, pa, pa, pa, pa, pa, pa, pa, pa]
    chs = []
    for k, pl in enumerate(plans):
        s = a if pl is pa else b
        chs.append(torch.as_tensor(phantom.random_channels(s, 100 + k)).cuda())
    outs = supra.bmode_batched(plans, chs)
    for pl, c, o in zip(plans, chs, outs):
        single = pl.bmode(c)
        d = (single.int() - o.int()).abs().max().item()
        assert d <= 1
        assert (single == o).float().mean().item() >= 0.9999


def test_config2_batch_of_64_matches_oracle_on_first_and_last_frame():
    s = phantom.config2()
    p = s.params()
    plan = supra.Plan(**p)
    seeds = list(range(1000, 1064))
    chs = []
    for sd in seeds:
        chs.append(phantom.synth_channels(s, phantom.default_phantom(s, sd), sd, device="cuda"))
    outs = supra.bmode_batched([plan] * 64, chs)
    torch.cuda.synchronize()
    for k in (0, 63):
        ch = chs[k].cpu().numpy()
        ref = oracle.bmode(p, ch)
        assert_gray(outs[k].cpu().numpy(), ref, what=f"frame {k}")
    # and the RF of one frame at full size
    rf = plan.beamform(chs[7]).cpu().numpy()
    assert max_norm_err(rf, oracle.das(p, chs[7].cpu().numpy())) <= RF_TOL


@pytest.mark.parametrize("kind", ["one_tile", "whole_tile", "pyramid", "plane_waves"])
def test_sixteen_frame_groups_match_single_frames(kind):
    # groups of 9-16 frames run the demodulating FIR on the tensor cores (split FP16 operands,
    # FP32 accumulation); single frames run it on the FP32 cores.  Records of one depth tile (the
    # FIR's halo and lag tile), of exactly one tile, a matrix-array pyramid (square 3D aperture)
    # and compounded plane-wave lines (the extended transmit model) must agree with the
    # single-frame path and with the oracle.
    if kind == "one_tile":
        s = phantom.linear_setup(24, 0.3e-3, 20, 200, fc=5e6, fs=40e6, grid_n=(40, 60))
    elif kind == "whole_tile":
        s = phantom.linear_setup(24, 0.3e-3, 20, 256, fc=5e6, fs=40e6, grid_n=(40, 60))
    elif kind == "pyramid":
        s = phantom.pyramid_setup(8, 8, 0.3e-3, 10, 9, 30.0, 400, fc=3.5e6, fs=20e6, grid_n=(40, 36, 50))
    else:
        s = phantom.planewave_setup(32, 0.3e-3, 24, 700, angles_deg=(-8, 0, 8), fc=5e6, fs=40e6,
                                    grid_n=(96, 160))
    p = s.params()
    plan = supra.Plan(**p)
    n = 13
    chs = [phantom.random_channels(s, 500 + k).cuda() for k in range(n)]
    outs = supra.bmode_batched([plan] * n, chs)
    # images of 2400-72000 pixels: identical codes on >= 99.9 % (a handful of pixels may sit on a
    # code boundary, where the two FIR forms' summation orders differ), never more than one level
    for k in (0, 6, n - 1):
        single = plan.bmode(chs[k])
        assert (single.int() - outs[k].int()).abs().max().item() <= 1
        assert (single == outs[k]).float().mean().item() >= 0.999
    assert_gray(outs[n - 1].cpu().numpy(), oracle.bmode(p, chs[n - 1].cpu().numpy()), what=kind)
    assert supra.device_status() == 0


def test_contiguous_batch_uses_tensor_copies_and_matches():
    # frames at a uniform stride are staged with one tensor copy per element for all
    # frames of a group; results equal the per-frame path and the oracle
    s = phantom.linear_setup(48, 0.3e-3, 40, 700, fc=7e6, fs=40e6, grid_n=(96, 128))
    p = s.params()
    plan = supra.Plan(**p)
    n = 21                                              # groups of 16 + 5 (a partial group)
    batch = torch.empty((n, *plan.ch_shape), dtype=torch.int16, device="cuda")
    for k in range(n):
        batch[k].copy_(phantom.random_channels(s, 300 + k))
    outs = supra.bmode_batched([plan] * n, list(batch))
    for k in (0, 7, 15, 16, 20):
        single = plan.bmode(batch[k].clone())
        assert (single.int() - outs[k].int()).abs().max().item() <= 1
        assert (single == outs[k]).float().mean().item() >= 0.9999
    ref = oracle.bmode(p, batch[20].cpu().numpy())
    assert_gray(outs[20].cpu().numpy(), ref, what="frame 20")
    # lines without a grid, contiguous 8-frame group
    plan_l = supra.Plan(**dict(p, grid=None))
    outs_l = supra.bmode_batched([plan_l] * 8, list(batch[:8]))
    ref_l = oracle.bmode(dict(p, grid=None), batch[3].cpu().numpy())
    assert_gray(outs_l[3].cpu().numpy(), ref_l, what="lines frame 3")


def test_config1_bmode_lines_full_size():
    s = phantom.config1()
    p = s.params()
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 1), 1)
    plan = supra.Plan(**p)
    got = plan.bmode(ch.cuda()).cpu().numpy()
    assert_gray(got, oracle.bmode(p, ch.numpy()), what="64-element frame")


def test_config3_volume_full_size_sampled():
    # 32x32 matrix array, 64x64 lines on a +-30 deg pyramid, 1536 samples: 12 GiB of records per
    # volume.  Sampled lines (RF, log-compressed lines) and sampled voxels of the 256^3 volume are
    # checked against the oracle, which reads only the transmit records it needs.
    s = phantom.config3()
    p = s.params()
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 3000), 3000, device="cuda")
    plan = supra.Plan(**p)
    plan_l = supra.Plan(**dict(p, grid=None))
    vol = plan.bmode(ch).cpu().numpy()
    rf = plan.beamform(ch).cpu().numpy()
    bm = plan_l.bmode(ch).cpu().numpy()
    torch.cuda.synchronize()
    nd = s.n_depth
    rng = np.random.default_rng(7)

    def oracle_lines(lines):
        out = {}
        for l in lines:
            block = ch[int(s.line_tx[l])].cpu().numpy()
            out[l] = oracle.das_points(p, [l] * nd, np.arange(nd), [block] * nd)
        return out

    lines = sorted(set(rng.integers(0, s.n_lines, 10).tolist()) | {32 * 64 + 32})
    rf_o = oracle_lines(lines)
    ref = np.stack([rf_o[l] for l in lines])
    assert max_norm_err(rf[lines], ref) <= RF_TOL
    bm_o = oracle.logcompress(oracle.envelope(p, ref), p["log_ref"], p["dyn_range_db"])
    assert_gray(bm[lines], bm_o, what="pyramid lines")
    # voxels: every voxel of 24 randomly chosen line cells (the voxels between 2 x 2 neighbouring
    # lines, at all depths: ~25 000 voxels), through the oracle's own chain on the lines they need,
    # at the B-mode bar (>= 99.9 % within one gray level)
    pts_all = oracle.grid_points(p["grid"]).reshape(-1, 3)
    ux, uy, v, ok = oracle.scan_coordinates(p, pts_all)
    cx = np.minimum(np.floor(np.maximum(ux, 0)).astype(np.int64), s.lines_x - 2)
    cy = np.minimum(np.floor(np.maximum(uy, 0)).astype(np.int64), s.lines_y - 2)
    cells = {(int(a), int(b)) for a, b in rng.integers(0, s.lines_x - 1, (24, 2))}
    pick = np.nonzero(ok & np.isin(cy * s.lines_x + cx, [b * s.lines_x + a for a, b in cells]))[0]
    assert len(pick) > 20000
    need = sorted({(b + dy) * s.lines_x + a + dx for a, b in cells for dy in (0, 1) for dx in (0, 1)})
    rf_n = oracle_lines(need)
    bm_full = np.zeros((s.n_lines, nd), np.uint8)
    for l, r in rf_n.items():
        bm_full[l] = oracle.logcompress(oracle.envelope(p, r[None]), p["log_ref"], p["dyn_range_db"])[0]
    assert_gray(bm[need], bm_full[need], what="lines of the chosen cells")
    want = oracle.scanconvert(p, bm_full, pts_all[pick])
    got = vol.reshape(-1)[pick]
    # scan conversion alone: the oracle's interpolation of the GPU's own lines
    bm_gpu = np.zeros_like(bm_full)
    bm_gpu[need] = bm[need]
    same_lines = oracle.scanconvert(p, bm_gpu, pts_all[pick])
    assert_gray(got, same_lines, frac=1.0, what="pyramid scan conversion of the GPU lines")
    assert_gray(got, want, what=f"{len(pick)} voxels of {len(cells)} line cells")


def test_table1_multiline_frame_matches_oracle():
    # Table 1's "128/2": 64 channels, 128 transmits with two receive lines each (255 lines),
    # 45 mm, 0.0225 mm isotropic output grid -- the whole frame through the oracle's chain
    s = phantom.table1_setup(128, 2)
    p = s.params()
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 77, 3000, n_points=5), 77, device="cuda")
    plan = supra.Plan(**p)
    rf = plan.beamform(ch).cpu().numpy()
    img = plan.bmode(ch).cpu().numpy()
    ref_rf = oracle.das(p, ch.cpu().numpy())
    assert max_norm_err(rf, ref_rf) <= RF_TOL
    bm = oracle.logcompress(oracle.envelope(p, ref_rf), p["log_ref"], p["dyn_range_db"])
    ref = oracle.scanconvert(p, bm)[:, 0, :]
    assert img.shape == ref.shape
    assert_gray(img, ref, what="table-1 128/2 frame")


def test_batched_mixed_plans_records_equal_halo_tiles():
    # An uneven batch (two plans, one with a grid, one with lines out) whose one-frame launches are
    # split along depth: with the recommended workspace (boundary records) and with the lines'
    # workspace only (each segment beamforms its halo), the same bytes.
    a = phantom.linear_setup(32, 0.3e-3, 40, 600, fc=7e6, fs=40e6, grid_n=(100, 120))
    b = phantom.sector_setup(24, 0.3e-3, 30, 35.0, 500, fc=3.5e6, fs=20e6)
    pa, pb = supra.Plan(**a.params()), supra.Plan(**b.params())
    plans = [pa, pb, pa, pa, pb, pa]
    chs = [torch.as_tensor(phantom.random_channels(a if pl is pa else b, 150 + k)).cuda() for k, pl in enumerate(plans)]
    need = supra.workspace_size(plans)
    lines = sum(-(-pl.line_shape[0] * pl.line_shape[1] // 256) * 256 for pl in plans if pl is pa)
    assert need > lines   # room for the records
    rec = [o.cpu().numpy() for o in supra.bmode_batched(plans, chs)]
    halo = [o.cpu().numpy() for o in
            supra.bmode_batched(plans, chs, workspace=torch.empty(lines, dtype=torch.uint8, device="cuda"))]
    for k, (x, y) in enumerate(zip(rec, halo)):
        np.testing.assert_array_equal(x, y, err_msg=f"frame {k}")
    assert supra.device_status() == 0


@pytest.mark.parametrize("segments", [0, 3, 5])
def test_segment_boundary_records_equal_halo_tiles(segments):
    # One frame split along depth: with the workspace supra_bmode_workspace_size reports, the
    # segments leave the outputs around their boundaries to the boundary kernel; with only the
    # lines' workspace each segment beamforms the halo it needs.  Same codes byte for byte,
    # whole-line codes too, and both the oracle's chain within the B-mode tolerance.
    s = phantom.table1_setup(64, 1)
    p = dict(s.params(), grid=None)
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 78, 3000, n_points=5), 78, device="cuda")
    plan = supra.Plan(**p)
    plan.tile_shape = dict(plan.tile_shape, frames_per_group=1, depth_segments=segments)
    need = supra.workspace_size([plan])
    assert need > 0   # lines out: only the boundary records
    rec = plan.bmode(ch).cpu().numpy()
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    halo = plan.bmode(ch, workspace=small).cpu().numpy()
    np.testing.assert_array_equal(rec, halo)
    whole = supra.Plan(**p)
    whole.tile_shape = dict(whole.tile_shape, frames_per_group=1, depth_segments=1)
    np.testing.assert_array_equal(rec, whole.bmode(ch).cpu().numpy())
    ref = oracle.logcompress(oracle.envelope(p, oracle.das(p, ch.cpu().numpy())), p["log_ref"], p["dyn_range_db"])
    assert_gray(rec, ref, what=f"{segments} segments")
    assert supra.device_status() == 0


def _compounding(s):
    s.n_bands, s.band_step = 3, s.fc / 4
    return s


def test_compounded_envelope_node_matches_oracle():
    # the band bank of Sec. 2 item 3 on identical fp32 RF input
    s = _compounding(small_linear(24, 6, 700))
    p = s.params()
    plan = supra.Plan(**p)
    rf = torch.as_tensor(np.random.default_rng(5).normal(0, 1000, plan.line_shape).astype(np.float32)).cuda()
    env = plan.envelope(rf).cpu().numpy()
    ref = oracle.envelope(p, rf.cpu().numpy().astype(np.float64))
    assert max_norm_err(env, ref) <= ENV_TOL


def test_compounded_chain_and_mixed_batch_match():
    s = _compounding(phantom.linear_setup(48, 0.3e-3, 24, 900, fc=5e6, fs=40e6, grid_n=(96, 160)))
    p = s.params()
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 91, 800, n_points=3), 91)
    plan = supra.Plan(**p)
    img = plan.bmode(ch.cuda()).cpu().numpy()
    assert_gray(img, oracle.bmode(p, ch.numpy()), what="compounded chain")
    # a batch mixing the compounding plan with a one-band plan: each frame as alone
    s1 = phantom.linear_setup(32, 0.3e-3, 16, 600, fc=5e6, fs=40e6, grid_n=(64, 96))
    plan1 = supra.Plan(**s1.params())
    ch1 = phantom.synth_channels(s1, phantom.make_phantom(s1, 92, 500), 92).cuda()
    outs = supra.bmode_batched([plan, plan1, plan], [ch.cuda(), ch1, ch.cuda()])
    np.testing.assert_array_equal(outs[0].cpu().numpy(), img)
    np.testing.assert_array_equal(outs[2].cpu().numpy(), img)
    np.testing.assert_array_equal(outs[1].cpu().numpy(), plan1.bmode(ch1).cpu().numpy())
    assert supra.device_status() == 0


def test_plane_wave_compounding_matches_oracle():
    # five plane waves at -8..8 degrees, every line averages all of them (coherent compounding)
    s = phantom.planewave_setup(32, 0.3e-3, 24, 700, angles_deg=(-8, -4, 0, 4, 8), fc=5e6, fs=40e6,
                                grid_n=(96, 160))
    p = s.params()
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 31, 1500, n_points=3), 31)
    plan = supra.Plan(**p)
    rf = plan.beamform(ch.cuda()).cpu().numpy()
    ref = oracle.das(p, ch.numpy())
    assert max_norm_err(rf, ref) <= RF_TOL
    img = plan.bmode(ch.cuda()).cpu().numpy()
    assert_gray(img, oracle.bmode(p, ch.numpy()), what="plane-wave compounding")
    # in a batch with a plan that does not compound: each frame as alone
    s1 = small_linear(24, 10, 500, grid_n=(64, 96))
    plan1 = supra.Plan(**s1.params())
    ch1 = phantom.random_channels(s1, 32).cuda()
    outs = supra.bmode_batched([plan1, plan, plan, plan1], [ch1, ch.cuda(), ch.cuda(), ch1])
    np.testing.assert_array_equal(outs[1].cpu().numpy(), img)
    np.testing.assert_array_equal(outs[2].cpu().numpy(), img)
    np.testing.assert_array_equal(outs[0].cpu().numpy(), plan1.bmode(ch1).cpu().numpy())
    with pytest.raises(supra.SupraError):   # MV is defined per transmit, not on compounded lines
        plan.mv(ch.cuda(), 8)
    assert supra.device_status() == 0


def test_single_steered_plane_wave_lines_match_oracle():
    # one 6-degree plane wave, every line formed from it (no compounding): DAS and MV
    s = phantom.planewave_setup(32, 0.3e-3, 16, 600, angles_deg=(6,), fc=5e6, fs=40e6)
    s.compound = 0
    p = s.params()
    ch = phantom.random_channels(s, 33)
    plan = supra.Plan(**p)
    rf = plan.beamform(ch.cuda()).cpu().numpy()
    assert max_norm_err(rf, oracle.das(p, ch.numpy())) <= RF_TOL
    mv = plan.mv(ch.cuda(), 8).cpu().numpy()
    lines, depths = list(range(16)), list(range(0, 600, 13))
    ref = oracle.mv(p, ch.numpy(), 8, lines=lines, depths=depths)
    keep = np.array([[np.min(np.abs(oracle.aperture(p, l, i)[2])) > 1e-9 for i in depths] for l in lines])
    assert np.max(np.abs(mv[np.ix_(lines, depths)] - ref)[keep]) <= 1e-3 * np.max(np.abs(ref))
