"""GPU tests of the real-time request loop (supra_server_*) and the autotuner.

The loop must not change results: each request's image equals the one the
direct entry points give for that request alone (the same kernels on the same
inputs; the tolerance is the B-mode bar, >= 99.9 % of pixels within one gray
level, and in practice the images are identical)."""
import numpy as np
import pytest
import torch

import paper_1711_06127_b300 as supra
from paper_1711_06127_b300.serving import Server
import phantom
from gpu_util import assert_gray

pytestmark = pytest.mark.gpu


def _setups():
    a = phantom.linear_setup(64, 0.3e-3, 64, 1024, fc=5e6, fs=40e6, grid_n=(128, 160), name="a")
    b = phantom.linear_setup(96, 0.3e-3, 96, 1536, fc=6e6, fs=40e6, grid_n=(160, 192), name="b")
    c = phantom.sector_setup(64, 0.3e-3, 48, 30.0, 1024, grid_n=(128, 128), name="c")
    return a, b, c


def _alone(kind, plan, ch, params=None, L=16):
    """The image of one request by the direct entry points."""
    if kind == "das":
        return plan.bmode(ch)
    rf = plan.mv(ch, L) if kind == "mv" else plan.apod(ch, params)
    bm = plan.logcompress(plan.envelope(rf))
    return plan.scanconvert(bm) if plan.image_shape is not None else bm


def _mix(n, seed):
    a, b, c = _setups()
    plans = [supra.Plan(**s.params()) for s in (a, b, c)]
    frames = [[phantom.synth_channels(s, phantom.make_phantom(s, 10 * k + j, 600, n_points=2), 10 * k + j,
                                      device="cuda") for j in range(2)] for k, s in enumerate((a, b, c))]
    params = torch.as_tensor(phantom.apod_init(3, out_scale=1.0, bias_scale=0.05)).cuda()
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        k = int(rng.integers(0, 3))
        kind = ["das", "mv", "apod"][int(rng.integers(0, 3))]
        reqs.append((kind, k, int(rng.integers(0, 2))))
    return plans, frames, params, reqs


def _kw(kind, params):
    if kind == "mv":
        return dict(mv_subaperture=16, mv_loading=0.01)
    if kind == "apod":
        return dict(apod_params=params)
    return {}


def test_each_result_is_the_same_alone_and_in_the_mix():
    plans, frames, params, reqs = _mix(40, 1)
    srv = Server(2 << 30, n_streams=3, max_batch=8, use_graphs=True)
    tickets = {}
    for i, (kind, k, j) in enumerate(reqs):
        t = srv.submit(kind, plans[k], ch=frames[k][j], tag=i, **_kw(kind, params))
        tickets[t] = i
    srv.wait(120)
    done = srv.poll()
    assert len(done) == len(reqs)
    for c in done:
        assert c["status"] == 0
        kind, k, j = reqs[c["tag"]]
        got = srv.result(c, plans[k].out_shape)
        srv.release(c["ticket"])
        ref = _alone(kind, plans[k], frames[k][j], params)
        assert_gray(got.cpu().numpy(), ref.cpu().numpy())
        assert c["t_submit"] <= c["t_admit"] <= c["t_done"]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["memory_used"] == 0
    assert 0 < st["batches"] and st["graph_launches"] <= st["batches"]
    assert max(c["batch_size"] for c in done) > 1    # requests were batched
    srv.close()
    assert supra.device_status() == 0


def test_memory_admission_keeps_the_footprint_inside_the_arena():
    a, _, _ = _setups()
    plan = supra.Plan(**a.params())
    ch = phantom.synth_channels(a, phantom.make_phantom(a, 5, 500), 5, device="cuda")
    info = plan.info
    per_req = info["channel_bytes"] + info["image_bytes"] + info["bmode_bytes"] + 3 * 256
    arena = int(2.5 * per_req)    # room for two ingested requests at a time
    ch_host = ch.cpu().pin_memory()
    outs = [torch.empty(plan.out_shape, dtype=torch.uint8).pin_memory() for _ in range(10)]
    srv = Server(arena, n_streams=2, max_batch=4, use_graphs=False)
    for i in range(10):
        srv.submit("das", plan, ch_host=ch_host, out_host=outs[i], tag=i)
    srv.wait(120)
    done = srv.poll()
    st = srv.stats()
    assert len(done) == 10 and all(c["status"] == 0 and c["out"] is None for c in done)
    assert st["memory_peak"] <= arena and st["memory_used"] == 0
    assert st["batches"] >= 5                        # at most two requests fit at once
    ref = plan.bmode(ch).cpu().numpy()
    for o in outs:
        assert_gray(o.numpy(), ref)
    srv.close()


def test_open_loop_trace_reports_latencies_and_reuses_graphs():
    a, _, _ = _setups()
    plan = supra.Plan(**a.params())
    ch = phantom.synth_channels(a, phantom.make_phantom(a, 6, 500), 6, device="cuda")
    srv = Server(1 << 30, n_streams=2, max_batch=4, use_graphs=True)
    n = 60
    t_arr = np.cumsum(np.random.default_rng(2).exponential(1.0 / 2000.0, n))
    srv.submit_trace([("das", plan, dict(ch=ch, tag=i)) for i in range(n)], t_arr)
    srv.wait(120)
    done = srv.poll()
    assert len(done) == n
    lat = np.array([c["t_done"] - c["t_submit"] for c in done])
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    # arrivals are the scheduled times (relative to the trace start, in order)
    subs = np.sort(np.array([c["t_submit"] for c in done]))
    np.testing.assert_allclose(np.diff(subs), np.diff(t_arr), atol=1e-9)
    st = srv.stats()
    assert st["graph_launches"] > 0 and st["graph_updates"] > 0   # recurring buckets replay their graph
    ref = plan.bmode(ch).cpu().numpy()
    for c in done:
        assert_gray(srv.result(c, plan.out_shape).cpu().numpy(), ref)
        srv.release(c["ticket"])
    srv.close()


def test_autotuner_picks_a_frames_per_tile_class_and_keeps_results():
    a, _, _ = _setups()
    plan = supra.Plan(**a.params())
    chs = [phantom.synth_channels(a, phantom.make_phantom(a, 20 + i, 400), 20 + i, device="cuda") for i in range(8)]
    ref = [plan.bmode(c).cpu().numpy() for c in chs]
    g, ms = plan.autotune(chs, reps=2)
    assert g in (1, 2, 4, 8) and plan.max_group == g and ms > 0
    outs = supra.bmode_batched([plan] * 8, chs)
    for o, r in zip(outs, ref):
        assert_gray(o.cpu().numpy(), r)
    plan.max_group = 16


def test_tile_shapes_give_the_same_images_and_the_tuner_keeps_its_pick():
    # A 16-frame group and a 3-frame tail of contiguous frames under every kind of tile shape
    # the tuner can pick.  Shapes that keep 16-frame groups give the untuned plan's images byte
    # for byte; smaller groups run the demodulating filter on the FP32 cores instead of the
    # tensor cores, and all of them (any group size, depth segments, CTAs per SM) give one
    # another's images byte for byte and the untuned ones within the B-mode tolerance.
    a, _, _ = _setups()
    p = a.params()
    plan = supra.Plan(**p)
    batch = torch.stack([phantom.synth_channels(a, phantom.make_phantom(a, 40 + i, 400), 40 + i) for i in range(19)])
    chs = list(batch.cuda())
    ref = [o.cpu().numpy() for o in supra.bmode_batched([plan] * 19, chs)]
    default = plan.tile_shape
    assert default == {"frames_per_group": 16, "elements_per_stage": 3, "stages": 3, "depth_segments": 0,
                       "ctas_per_sm": 0}

    def images(shape):
        tuned = supra.Plan(**p)
        tuned.tile_shape = shape
        assert tuned.tile_shape == shape
        return [o.cpu().numpy() for o in supra.bmode_batched([tuned] * 19, chs)]

    for k, (o, r) in enumerate(zip(images(dict(default, elements_per_stage=2, stages=4)), ref)):
        np.testing.assert_array_equal(o, r, err_msg=f"2 x 4 stages, frame {k}")
    ref_fp32 = images(dict(default, frames_per_group=8))
    for o, r in zip(ref_fp32, ref):
        assert_gray(o, r)
    shapes = [dict(default, frames_per_group=g, depth_segments=s) for g in (8, 2) for s in (1, 3)]
    shapes += [dict(default, frames_per_group=1, depth_segments=s, ctas_per_sm=c) for s in (0, 2) for c in (2, 3)]
    for sh in shapes:
        for k, (o, r) in enumerate(zip(images(sh), ref_fp32)):
            np.testing.assert_array_equal(o, r, err_msg=f"{sh} frame {k}")
    best, ms, ms0 = plan.autotune_shape(chs, reps=2)
    assert plan.tile_shape == best and ms > 0 and ms0 > 0 and ms <= ms0
    want = ref if best["frames_per_group"] == 16 else ref_fp32
    for o, r in zip(supra.bmode_batched([plan] * 19, chs), want):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    with pytest.raises(supra.SupraError):
        plan.tile_shape = dict(default, elements_per_stage=4, stages=2)
    with pytest.raises(supra.SupraError):
        plan.tile_shape = dict(default, ctas_per_sm=1)
    assert supra.device_status() == 0


def test_rejects_requests_that_cannot_run():
    a, _, _ = _setups()
    plan = supra.Plan(**a.params())
    ch = torch.zeros(plan.ch_shape, dtype=torch.int16, device="cuda")
    srv = Server(1 << 20, n_streams=1, max_batch=2)
    with pytest.raises(supra.SupraError):   # input + output do not fit 1 MiB
        srv.submit("das", plan, ch_host=ch.cpu().pin_memory())
    with pytest.raises(supra.SupraError):   # learned apodization without parameters
        srv.submit("apod", plan, ch=ch)
    with pytest.raises(supra.SupraError):   # neither or both channel sources
        srv.submit("das", plan)
    big = supra.Plan(**phantom.config3(lines=8).params())
    with pytest.raises(supra.SupraError):   # 1024 elements: more than the network's inputs
        srv.submit("apod", big, ch=ch, apod_params=torch.zeros(supra.APOD_PARAMS, device="cuda"))
    srv.close()
