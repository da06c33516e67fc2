"""Training and use of the learned per-pixel confidence weight.

Everything numeric runs in the library's kernels (itm_conf_features,
itm_mlp_loss_grad, itm_mlp_adam, itm_mlp_pack, itm_conf_weights); this module
owns the device buffers (torch tensors) and the loop.
"""

from __future__ import annotations

import numpy as np

from . import (ITM_MLP_FEATURES, ITM_MLP_HIDDEN, ITM_MLP_PACKED_BYTES, ITM_MLP_PARAMS,
               ITM_MLP_SCRATCH_PER_SAMPLE, itm_conf_features, itm_conf_weights, itm_mlp_adam,
               itm_mlp_loss_grad, itm_mlp_pack)


def init_params(seed=0) -> np.ndarray:
    """He-uniform weights, zero biases, a positive output bias (most
    measurements are good), fp32."""
    rng = np.random.default_rng(seed)
    nf, nh = ITM_MLP_FEATURES, ITM_MLP_HIDDEN
    parts = [rng.uniform(-1, 1, nh * nf) * np.sqrt(6.0 / nf), np.zeros(nh),
             rng.uniform(-1, 1, nh * nh) * np.sqrt(6.0 / nh), np.zeros(nh),
             rng.uniform(-1, 1, nh) * np.sqrt(6.0 / nh), np.array([2.0])]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ITM_MLP_PARAMS
    return p


class ConfidenceModel:
    """fp32 master parameters, Adam moments and the packed inference copy on
    one device."""

    def __init__(self, params=None, device="cuda", seed=0):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.from_numpy(p.copy()).to(self.dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.packed = torch.zeros(ITM_MLP_PACKED_BYTES, dtype=torch.uint8, device=self.dev)
        self.step = 0
        self._scratch = None

    def pack(self):
        itm_mlp_pack(self.params, self.packed)
        return self.packed

    def loss_grad(self, feat, labels):
        n = labels.numel()
        if self._scratch is None or self._scratch.numel() < n * ITM_MLP_SCRATCH_PER_SAMPLE:
            self._scratch = self.torch.empty(n * ITM_MLP_SCRATCH_PER_SAMPLE, dtype=self.torch.float32,
                                             device=self.dev)
        itm_mlp_loss_grad(self.params, feat, labels, n, self._scratch, self.grad, self.loss)
        return self.loss, self.grad

    def train(self, feat, labels, steps=300, batch=8192, lr=3e-3, seed=0):
        """Adam on mini-batches of (feat [N, 52], labels [N]) device tensors;
        returns the loss of every step (host floats, read at the end)."""
        torch = self.torch
        N = labels.numel()
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        perm = torch.randperm(N, generator=g).to(self.dev)
        pos = 0
        for it in range(steps):
            if pos + batch > N:
                perm = torch.randperm(N, generator=g).to(self.dev)
                pos = 0
            idx = perm[pos:pos + batch]
            pos += batch
            fb = feat.index_select(0, idx).contiguous()
            lb = labels.index_select(0, idx).contiguous()
            self.loss_grad(fb, lb)
            self.step += 1
            lr_t = lr * (0.5 * (1 + np.cos(np.pi * it / steps)) * 0.9 + 0.1)
            itm_mlp_adam(self.params, self.grad, self.m, self.v, self.step, lr_t)
            losses.append(self.loss.clone())
        self.pack()
        return [float(x.item()) for x in losses]

    def weights(self, depth, intr, mu, out):
        itm_conf_weights(depth, intr, mu, self.packed, out)
        return out


def build_training_set(frames, intr, mu, pixel_lists, label_maps, device="cuda"):
    """Features (computed by the library) and labels of the sampled pixels
    of several depth frames, concatenated on the device."""
    import torch
    feats, labs = [], []
    for depth, pix, lab in zip(frames, pixel_lists, label_maps):
        d = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.float32)).to(device)
        p = torch.from_numpy(np.ascontiguousarray(pix, dtype=np.int32)).to(device)
        f = torch.empty((p.numel(), ITM_MLP_FEATURES), dtype=torch.float32, device=device)
        itm_conf_features(d, intr, mu, p, p.numel(), f)
        feats.append(f)
        labs.append(torch.from_numpy(np.ascontiguousarray(lab.ravel()[pix], dtype=np.float32)).to(device))
    return torch.cat(feats), torch.cat(labs)
