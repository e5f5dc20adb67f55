"""Learned apodization: training and evaluation driver over the C ABI
(supra_apod_forward / supra_apod_grad / supra_apod_adam / supra_apod_step).  Argument
marshalling, minibatch bookkeeping and checkpoints only; the network's
forward and backward passes and the optimiser step run in libsupra's
kernels.

Data layout: one row per pixel (feature row bfloat16 [128], aperture mask
int32 [4], norm float32, label float32), frames concatenated.  Minibatch k of
K takes rows k, k + K, k + 2K, ... so every minibatch spans all frames,
lines and depths; the order of minibatches is reshuffled every epoch.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import APOD_INPUTS, APOD_PARAMS, _check, _stream_ptr, load


def _ptr(t, offset_rows=0):
    return t.data_ptr() + offset_rows * t.stride(0) * t.element_size()


def _check_rows(feat, mask, norm, label=None):
    import torch

    n = feat.shape[0]
    ok = (feat.is_cuda and feat.dtype == torch.bfloat16 and tuple(feat.shape) == (n, APOD_INPUTS)
          and feat.is_contiguous() and mask.dtype == torch.int32 and tuple(mask.shape) == (n, 4)
          and mask.is_contiguous() and norm.dtype == torch.float32 and tuple(norm.shape) == (n,)
          and (label is None or (label.dtype == torch.float32 and tuple(label.shape) == (n,))))
    if not ok:
        raise ValueError("feature rows must be bfloat16 [n,128], int32 [n,4], float32 [n] (+ float32 [n]) on CUDA")
    return n


@dataclass
class Dataset:
    """Feature rows of several frames plus their labels (device tensors)."""
    feat: object
    mask: object
    norm: object
    label: object

    @property
    def n(self) -> int:
        return int(self.feat.shape[0])


def make_dataset(plan, frames, label_fn, stream=None) -> Dataset:
    """Rows of every pixel of every frame (device int16 channel tensors);
    label_fn(plan, ch) -> float32 [n_lines, n_depth] device tensor (e.g. the
    MV beamformer)."""
    import torch

    frames = list(frames)
    P = plan.n_lines * plan.n_depth
    dev = frames[0].device
    feat = torch.empty((len(frames) * P, APOD_INPUTS), dtype=torch.bfloat16, device=dev)
    mask = torch.empty((len(frames) * P, 4), dtype=torch.int32, device=dev)
    norm = torch.empty((len(frames) * P,), dtype=torch.float32, device=dev)
    label = torch.empty((len(frames) * P,), dtype=torch.float32, device=dev)
    for f, ch in enumerate(frames):
        sl = slice(f * P, (f + 1) * P)
        plan.apod_features(ch, feat[sl], mask[sl], norm[sl], stream)
        label[sl] = label_fn(plan, ch).reshape(-1)
    return Dataset(feat, mask, norm, label)


def forward(params, feat, mask, norm, y=None, stream=None):
    """y = ||x|| * sum_e w_e xh_e for every row."""
    import torch

    n = _check_rows(feat, mask, norm)
    y = torch.empty((n,), dtype=torch.float32, device=feat.device) if y is None else y
    _check(load().supra_apod_forward(params.data_ptr(), n, 1, feat.data_ptr(), mask.data_ptr(), norm.data_ptr(),
                                     y.data_ptr(), _stream_ptr(stream)), "supra_apod_forward")
    return y


def workspace_size() -> int:
    return int(load().supra_apod_workspace_size())


class Trainer:
    """Adam on the flat parameter vector, FP32 master weights on the device."""

    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, device="cuda"):
        import torch

        self.params = torch.as_tensor(np.asarray(params, np.float32)).to(device).contiguous()
        assert self.params.shape == (APOD_PARAMS,)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.ws = torch.empty(workspace_size(), dtype=torch.uint8, device=device)
        self.lr, self.betas, self.eps = float(lr), tuple(float(b) for b in betas), float(eps)
        self.step_count = 0

    def compute_grad(self, data: Dataset, base=0, stride=1, n=None, stream=None):
        """Loss and gradient over rows base, base + stride, ... (n rows); fills
        self.grad and self.loss."""
        total = _check_rows(data.feat, data.mask, data.norm, data.label)
        if n is None:
            n = (total - base + stride - 1) // stride
        if n <= 0 or base + (n - 1) * stride >= total:
            raise ValueError("row range outside the dataset")
        _check(load().supra_apod_grad(self.params.data_ptr(), int(n), int(stride), _ptr(data.feat, base),
                                      _ptr(data.mask, base), _ptr(data.norm, base), _ptr(data.label, base),
                                      self.grad.data_ptr(), self.loss.data_ptr(), self.ws.data_ptr(),
                                      self.ws.numel(), _stream_ptr(stream)), "supra_apod_grad")
        return self.grad, self.loss

    def apply(self, stream=None):
        """One Adam step with the current self.grad."""
        self.step_count += 1
        _check(load().supra_apod_adam(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                      self.grad.data_ptr(), self.step_count, self.lr, self.betas[0], self.betas[1],
                                      self.eps, _stream_ptr(stream)), "supra_apod_adam")

    def step(self, data: Dataset, base=0, stride=1, n=None, loss_out=None, stream=None):
        """One training step: the gradient over rows base, base + stride, ...
        (n rows) and the Adam update, in two launches (supra_apod_step).  The
        minibatch loss goes to loss_out (a one-element device tensor) or to
        self.loss; self.grad holds the gradient."""
        total = _check_rows(data.feat, data.mask, data.norm, data.label)
        if n is None:
            n = (total - base + stride - 1) // stride
        if n <= 0 or base + (n - 1) * stride >= total:
            raise ValueError("row range outside the dataset")
        out = self.loss if loss_out is None else loss_out
        if out.numel() < 1 or not out.is_contiguous():
            raise ValueError("loss_out must be a contiguous device tensor of at least one element")
        self.step_count += 1
        _check(load().supra_apod_step(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.step_count,
                                      self.lr, self.betas[0], self.betas[1], self.eps, int(n), int(stride),
                                      _ptr(data.feat, base), _ptr(data.mask, base), _ptr(data.norm, base),
                                      _ptr(data.label, base), self.grad.data_ptr(), out.data_ptr(), self.ws.data_ptr(),
                                      self.ws.numel(), _stream_ptr(stream)), "supra_apod_step")

    def epoch(self, data: Dataset, n_batches: int, seed: int, stream=None, chunk: int = 1) -> float:
        """One pass over the data in n_batches interleaved minibatches (order
        shuffled with `seed`), the steps issued by the library in one call
        (supra_apod_epoch); returns the mean minibatch loss.  chunk: rows
        interleaved one at a time (1) or in blocks of 128 consecutive rows
        (128: each gradient tile reads one contiguous block)."""
        import torch

        total = _check_rows(data.feat, data.mask, data.norm, data.label)
        n_batches = int(n_batches)
        if chunk not in (1, 128) or n_batches < 1 or n_batches > -(-total // chunk):
            raise ValueError("chunk must be 1 or 128 and n_batches in 1 .. number of chunks")
        order = np.ascontiguousarray(np.random.default_rng(int(seed)).permutation(n_batches), dtype=np.int32)
        losses = torch.zeros(n_batches, dtype=torch.float32, device=self.params.device)
        _check(load().supra_apod_epoch(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.step_count,
                                       self.lr, self.betas[0], self.betas[1], self.eps, int(total), n_batches,
                                       int(chunk), order.ctypes.data, data.feat.data_ptr(), data.mask.data_ptr(),
                                       data.norm.data_ptr(), data.label.data_ptr(), self.grad.data_ptr(),
                                       losses.data_ptr(), self.ws.data_ptr(), self.ws.numel(), _stream_ptr(stream)),
               "supra_apod_epoch")
        self.step_count += n_batches
        return float(losses.mean())

    # ---- checkpoints -----------------------------------------------------
    def state_dict(self) -> dict:
        return {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "step": self.step_count, "lr": self.lr, "betas": self.betas, "eps": self.eps}

    def load_state_dict(self, st: dict):
        import torch

        for name in ("params", "m", "v"):
            getattr(self, name).copy_(torch.as_tensor(np.asarray(st[name], np.float32)))
        self.step_count = int(st["step"])
        self.lr, self.betas, self.eps = float(st["lr"]), tuple(st["betas"]), float(st["eps"])

    def save(self, path: str):
        st = self.state_dict()
        np.savez(path, params=st["params"], m=st["m"], v=st["v"],
                 meta=np.array([st["step"], st["lr"], st["betas"][0], st["betas"][1], st["eps"]], np.float64))

    def load(self, path: str):
        z = np.load(path)
        meta = z["meta"]
        self.load_state_dict({"params": z["params"], "m": z["m"], "v": z["v"], "step": int(meta[0]),
                              "lr": float(meta[1]), "betas": (float(meta[2]), float(meta[3])), "eps": float(meta[4])})
