"""Training and rendering with the learned thin-disk transfer function (marshalling only:
ray tracing, target construction, forward/backward passes, Adam and the surrogate render
all run in the library's kernels; this module slices device buffers and loops)."""
from __future__ import annotations

import math

import numpy as np

from . import binding as B
from . import workloads as W


def training_scene() -> dict:
    """Prototype for the training rays: thin disk from r_ISCO to 20 M, mixed precision."""
    return W.scene(precision="mixed")


class Surrogate:
    def __init__(self, tracer: B.Tracer, max_batch: int = 65536, seed: int = W.SEED + 3):
        import torch
        self.torch = torch
        self.tracer = tracer
        self.max_batch = max_batch
        self.mlp = B.odx_mlp_create(tracer.ctx, max_batch, seed)

    def close(self):
        if self.mlp is not None:
            B.odx_mlp_destroy(self.mlp)
            self.mlp = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def make_data(self, n_rays: int, seed: int = W.SEED + 1, r_max: float = 60.0):
        """Trace n_rays seeded rays (alpha, beta ~ U[-20, 20], a ~ U[0, 0.998],
        i ~ U[1, 89] deg) and build inputs x[n_pad][4] and targets t[n_pad][8] on the GPU."""
        t = self.torch
        dev = f"cuda:{self.tracer.device}"
        rays = t.from_numpy(W.training_rays(n_rays, seed)).to(dev)
        rec, _ = self.tracer.trace_rays(training_scene(), rays)
        n_pad = (n_rays + 127) // 128 * 128
        x = t.empty((n_pad, 4), dtype=t.float32, device=dev)
        tt = t.empty((n_pad, 8), dtype=t.float32, device=dev)
        st = t.cuda.current_stream(self.tracer.device).cuda_stream
        B.odx_mlp_targets(self.tracer.ctx, rec.data_ptr(), rays.data_ptr(), n_rays, r_max,
                          x.data_ptr(), tt.data_ptr(), st)
        return x, tt

    def train(self, x, tt, epochs: int, batch: int = 65536, lr: float = 2e-3,
              lr_final: float = 1e-4):
        """Adam over contiguous batches (the rays are drawn at random already); learning rate
        decays geometrically from lr to lr_final.  Returns the per-step losses."""
        t = self.torch
        n = x.shape[0] // batch * batch
        steps = epochs * (n // batch)
        loss = t.zeros(steps, dtype=t.float32, device=x.device)
        st = t.cuda.current_stream(self.tracer.device).cuda_stream
        k = 0
        for _ in range(epochs):
            for b0 in range(0, n, batch):
                rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
                B.odx_mlp_train_step(self.mlp, x[b0].data_ptr(), tt[b0].data_ptr(), batch, rate,
                                     loss[k].data_ptr(), st)
                k += 1
        return loss

    def forward(self, x):
        t = self.torch
        y = t.empty((x.shape[0], 4), dtype=t.float32, device=x.device)
        B.odx_mlp_forward(self.mlp, x.data_ptr(), x.shape[0], y.data_ptr(),
                          t.cuda.current_stream(self.tracer.device).cuda_stream)
        return y

    def render(self, scene: dict, band: float = 0.5, p_lo: float = 0.05, p_hi: float = 0.95,
               out=None):
        """Surrogate image of a thin-disk scene with integrator fallback.  Returns
        (image, fallback records, fallback pixel indices, number of fallback rays)."""
        t = self.torch
        n = scene["n_alpha"] * scene["n_beta"]
        dev = f"cuda:{self.tracer.device}"
        if out is None:
            img = t.empty(n, dtype=t.float64, device=dev)
            fb = t.empty((n, B.RECORD_BYTES // 8), dtype=t.float64, device=dev)
            pix = t.empty(n, dtype=t.int64, device=dev)
        else:
            img, fb, pix = out
        m = B.odx_surrogate_render(self.mlp, scene, band, p_lo, p_hi, fb.data_ptr(),
                                   pix.data_ptr(), img.data_ptr(),
                                   t.cuda.current_stream(self.tracer.device).cuda_stream)
        return img, fb, pix, m


def image_error(img, ref) -> float:
    """sum |I - I_ref| / sum |I_ref|."""
    return float((img - ref).abs().sum() / ref.abs().sum())
