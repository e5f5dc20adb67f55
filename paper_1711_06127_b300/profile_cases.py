"""Small, self-contained cases of each kernel for profiling (one warm-up call,
then the call to capture).  Sized so that a capture of one launch ends in a
minute or two: inputs larger than L2 where the kernel streams memory, a few GB
on the device at most.

    python -m paper_1711_06127_b300.profile_cases CASE

CASE: apod_train   gradient of 151552 feature rows (tcgen05 forward + backward), random rows
      apod_train_frames the same on the feature rows of a phantom frame (every third row of the
                   128-element / 256-line / 2048-sample frame: tiles of nearby depths of one line,
                   whose apertures leave whole output blocks empty, as in training on frames)
      apod_step    eight training steps as training runs them (supra_apod_step: the gradient, then
                   the reduction fused with Adam) of eight 128-pixel tile rounds each
      apod_minibatch eight training steps (gradient, reduction, Adam) of 65536-pixel
                   minibatches of 1.57 M feature rows
      apod_infer   fused gather + network beamformer, 128 el x 256 lines x 2048 samples
      apod_features feature rows of the same frame
      mv           exact minimum variance (L = 32) of the same frame
      das3d        fused B-mode of one 32x32-line pyramid volume (3 GiB of records)
      das3d_batch16 fused B-mode of 16 volumes of an 8x8-line pyramid in one batched call
                   (the 16-frame kernel; 3 GiB of records)
"""
from __future__ import annotations

import sys

import numpy as np


def main(case: str) -> int:
    import torch

    import paper_1711_06127_b300 as supra
    from paper_1711_06127_b300 import apod
    import phantom

    dev = torch.device("cuda", 0)
    if case == "apod_train":
        n = 148 * 128 * 8
        X, mask, norm, t = phantom.apod_random_batch(1, n)
        xh = np.divide(X, norm[:, None], out=np.zeros_like(X), where=norm[:, None] > 0)
        words = np.stack([(mask[:, 32 * w:32 * (w + 1)].astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
                          for w in range(4)], 1).astype(np.uint32)
        data = apod.Dataset(torch.as_tensor(xh).to(torch.bfloat16).to(dev),
                            torch.as_tensor(words.view(np.int32)).to(dev),
                            torch.as_tensor(norm.astype(np.float32)).to(dev),
                            torch.as_tensor((t * norm).astype(np.float32)).to(dev))
        tr = apod.Trainer(phantom.apod_init(2, out_scale=1.0, bias_scale=0.05))
        for _ in range(2):
            tr.compute_grad(data)
    elif case == "apod_train_frames":
        s = phantom.config2()
        plan = supra.Plan(**dict(s.params(), grid=None))
        P = plan.n_lines * plan.n_depth
        feat = torch.empty((P, supra.APOD_INPUTS), dtype=torch.bfloat16, device=dev)
        mask = torch.empty((P, 4), dtype=torch.int32, device=dev)
        norm = torch.empty((P,), dtype=torch.float32, device=dev)
        label = torch.empty((P,), dtype=torch.float32, device=dev)
        ch, _ = phantom.apod_frame(s, 4000, device=dev)
        plan.apod_features(ch, feat, mask, norm)
        plan.beamform(ch, label.view(plan.line_shape))
        data = apod.Dataset(feat, mask, norm, label)
        tr = apod.Trainer(phantom.apod_init(2, out_scale=1.0, bias_scale=0.05))
        for _ in range(2):
            tr.compute_grad(data, 0, 3, 148 * 128 * 8)
    elif case == "apod_step":
        n = 148 * 128 * 8
        X, mask, norm, t = phantom.apod_random_batch(1, 4 * n)
        xh = np.divide(X, norm[:, None], out=np.zeros_like(X), where=norm[:, None] > 0)
        words = np.stack([(mask[:, 32 * w:32 * (w + 1)].astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
                          for w in range(4)], 1).astype(np.uint32)
        data = apod.Dataset(torch.as_tensor(xh).to(torch.bfloat16).to(dev),
                            torch.as_tensor(words.view(np.int32)).to(dev),
                            torch.as_tensor(norm.astype(np.float32)).to(dev),
                            torch.as_tensor((t * norm).astype(np.float32)).to(dev))
        tr = apod.Trainer(phantom.apod_init(2, out_scale=1.0, bias_scale=0.05))
        for k in range(8):
            tr.step(data, k % 4, 4, n=n)
    elif case == "apod_minibatch":
        n = 65536 * 24
        X, mask, norm, t = phantom.apod_random_batch(1, n)
        xh = np.divide(X, norm[:, None], out=np.zeros_like(X), where=norm[:, None] > 0)
        words = np.stack([(mask[:, 32 * w:32 * (w + 1)].astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
                          for w in range(4)], 1).astype(np.uint32)
        data = apod.Dataset(torch.as_tensor(xh).to(torch.bfloat16).to(dev),
                            torch.as_tensor(words.view(np.int32)).to(dev),
                            torch.as_tensor(norm.astype(np.float32)).to(dev),
                            torch.as_tensor((t * norm).astype(np.float32)).to(dev))
        tr = apod.Trainer(phantom.apod_init(2, out_scale=1.0, bias_scale=0.05))
        for k in range(8):   # interleaved minibatches, as Trainer.epoch takes them
            tr.compute_grad(data, k, 24)
            tr.apply()
    elif case in ("apod_infer", "apod_features", "mv"):
        s = phantom.config2()
        plan = supra.Plan(**dict(s.params(), grid=None))
        ch, _ = phantom.apod_frame(s, 5000, device=dev)
        params = torch.as_tensor(phantom.apod_init(2, out_scale=1.0, bias_scale=0.05)).to(dev)
        for _ in range(2):
            if case == "apod_infer":
                plan.apod(ch, params)
            elif case == "apod_features":
                plan.apod_features(ch)
            else:
                plan.mv(ch, 32)
    elif case == "das3d":
        s = phantom.config3(32)
        plan = supra.Plan(**s.params())
        ch = phantom.synth_channels(s, phantom.default_phantom(s, 3000), 3000, device=dev)
        for _ in range(2):
            plan.bmode(ch)
    elif case == "das3d_batch16":
        s = phantom.config3(8)
        plan = supra.Plan(**s.params())
        batch = torch.empty((16, *plan.ch_shape), dtype=torch.int16, device=dev)
        for k in range(16):
            batch[k].copy_(phantom.synth_channels(s, phantom.default_phantom(s, 3000 + k), 3000 + k, device=dev))
        outs = [torch.empty(plan.out_shape, dtype=torch.uint8, device=dev) for _ in range(16)]
        for _ in range(2):
            supra.bmode_batched([plan] * 16, list(batch), outs)
    else:
        raise SystemExit(f"unknown case {case!r}")
    torch.cuda.synchronize()
    assert supra.device_status() == 0
    print(f"{case} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1] if len(sys.argv) > 1 else ""))
