"""Learned proposal: a small network that picks, per ray, the depth-8 BVH
subtree most likely to hold its closest hit (not in the paper).

Everything that computes runs in this package's CUDA kernels behind the
C-ABI (``sc_mlp_*``, ``sc_trace_waves``, ``sc_trace_seeded``); torch only
owns the device buffers, and numpy only draws the initial weights and the
per-epoch shuffle keys on the host.

Pipeline:
  1. ``collect``: jittered primary rays and their diffuse bounce waves are
     traced by the plain (exact) traversal; every ray that hits becomes a
     training pair (ray, frontier index of the hit triangle's subtree).
     Misses are left out.
  2. ``fit``: Adam on the mean cross-entropy over minibatches gathered on
     the device through a per-epoch permutation (FP32 master weights, BF16
     copy for the kernels).
  3. ``predict`` / ``trace``: top-1 subtree per ray, then the seeded
     traversal, whose hits are bit-identical to the plain traversal's.
"""
from __future__ import annotations

import math

import numpy as np

from . import scenegen as sg
from . import subcull as sc

IN, HID, OUT = 6, 64, 256


def _he_uniform(seed: int) -> np.ndarray:
    """Initial parameters: He-uniform weights, zero biases (layout of
    sc_mlp_num_params: W1[64][6] b1 W2[64][64] b2 W3[256][64] b3)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((HID, IN), (HID, HID), (OUT, HID)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == sc.sc_mlp_num_params()
    return w


class LearnedProposal:
    """Network, frontier and training state for one BVH."""

    def __init__(self, bvh: sc.Bvh, depth: int = 8, seed: int = 0, device="cuda"):
        import torch
        self.device = torch.device(device)
        ent, cls_of_tri = sc.sc_bvh_frontier(bvh, depth)
        if ent.shape[0] == 0:
            raise ValueError("empty BVH: no frontier")
        self.depth = depth
        self.n_frontier = ent.shape[0]
        self.frontier = torch.from_numpy(ent).to(self.device)
        self.class_of_tri = torch.from_numpy(cls_of_tri).to(self.device)
        box = np.array(bvh.info().root_box, np.float64)
        centre = 0.5 * (box[:3] + box[3:])
        half = np.maximum(0.5 * (box[3:] - box[:3]), 1e-6)
        self.box = torch.tensor(np.concatenate([centre, half]), dtype=torch.float32,
                                device=self.device)
        P = sc.sc_mlp_num_params()
        self.w = torch.from_numpy(_he_uniform(seed)).to(self.device)
        self.wb = torch.empty(P, dtype=torch.bfloat16, device=self.device)
        self.grad = torch.zeros(P, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self._status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.step = 0
        sc.sc_mlp_to_bf16(self.w, self.wb)

    # ------------------------------------------------------------ data --
    def collect(self, dbvh: sc.DeviceBVH, rays_list, bounces: int = 1, seed: int = 7,
                cap: int | None = None):
        """Training pairs from the plain traversal of each primary ray batch
        in rays_list (device float32[n, 8]) and its bounce waves.  Returns
        (rays float32[m, 8], labels int32[m]) on the device."""
        import torch
        total = sum(int(r.shape[0]) for r in rays_list) * (bounces + 1)
        cap = total if cap is None else min(cap, total)
        out_r = torch.empty((cap, 8), dtype=torch.float32, device=self.device)
        out_l = torch.empty(cap, dtype=torch.int32, device=self.device)
        count = torch.zeros(1, dtype=torch.int32, device=self.device)
        for i, rays in enumerate(rays_list):
            bufs = sc.WaveBuffers(rays.shape[0], bounces, with_counts=False, device=self.device,
                                  with_rays=True)
            _, sizes = sc.trace_waves(dbvh, rays, bounces, seed + i, 0, bufs)
            for w in range(bounces + 1):
                k = int(sizes[w])
                if k == 0:
                    continue
                sc.sc_mlp_labels(bufs.rays[w][:k], bufs.hits[w][:k], self.class_of_tri, out_r,
                                 out_l, count)
        torch.cuda.current_stream().synchronize()
        m = min(int(count.item()), cap)
        return out_r[:m], out_l[:m]

    # -------------------------------------------------------- training --
    def fit(self, rays, labels, steps: int, batch: int = 4096, lr: float = 2e-3,
            seed: int = 0, log_every: int = 0, tensor_cores: bool = True):
        """`steps` Adam steps over minibatches drawn on the device through a
        new pseudo-random permutation of the pairs every epoch
        (sc_mlp_gather); warm-up then cosine learning rate.  tensor_cores:
        the gradient's contractions as tcgen05 products (sc_mlp_grad_tc,
        BF16 operands), else FP32 CUDA cores (sc_mlp_grad).  Returns the
        mean loss of the last min(steps, 50) steps."""
        import torch
        n = int(rays.shape[0])
        if n == 0:
            raise ValueError("no training pairs")
        batch = min(batch, n)
        ws = torch.empty(sc.sc_mlp_train_workspace_bytes(batch), dtype=torch.uint8,
                         device=self.device)
        rng = np.random.default_rng(seed)
        rays = rays.contiguous()
        labels = labels.contiguous()
        br = torch.empty((batch, 8), dtype=torch.float32, device=self.device)
        bl = torch.empty(batch, dtype=torch.int32, device=self.device)
        losses = torch.zeros(steps, dtype=torch.float32, device=self.device)
        key = 0
        pos = n
        warm = max(1, steps // 20)
        self._status.zero_()
        for it in range(steps):
            if pos + batch > n:
                key = int(rng.integers(0, 2 ** 63))
                pos = 0
            sc.sc_mlp_gather(rays, labels, key, pos, batch, br, bl)
            pos += batch
            if tensor_cores:
                sc.sc_mlp_grad_tc(self.wb, br, bl, self.box, self.grad, self.loss, ws,
                                  self._status)
            else:
                sc.sc_mlp_grad(self.wb, br, bl, self.box, self.grad, self.loss, ws)
            losses[it:it + 1].copy_(self.loss)
            frac = it / max(1, steps - 1)
            cur = lr * min(1.0, (it + 1) / warm) * (0.1 + 0.45 * (1.0 + math.cos(math.pi * frac)))
            self.step += 1
            sc.sc_mlp_adam(self.w, self.wb, self.grad, self.m, self.v, self.step, cur)
            if log_every and (it + 1) % log_every == 0:
                print(f"step {it + 1}: loss {losses[it].item():.4f}")
        tail = losses[max(0, steps - 50):]
        out = float(tail.mean().item())
        if tensor_cores:
            self.check()
        return out

    # ------------------------------------------------------- inference --
    def predict(self, rays, cls=None, logits=None, min_prob: float = 0.0,
                tensor_cores: bool = True):
        """Top-1 frontier index per ray (device int32[n]); -1 (no seed) where
        the top-1 probability is below min_prob.  tensor_cores: layers 2 and
        3 as tcgen05 products (BF16 activations), else FP32 CUDA cores."""
        import torch
        if cls is None:
            cls = torch.empty(rays.shape[0], dtype=torch.int32, device=self.device)
        if tensor_cores:
            sc.sc_mlp_forward_tc(self.wb, rays, self.box, cls, self._status, logits, min_prob)
        else:
            sc.sc_mlp_forward(self.wb, rays, self.box, cls, logits, min_prob)
        return cls

    def state_dict(self) -> dict:
        """Weights, Adam moments and step (host tensors) for torch.save."""
        return {"w": self.w.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "step": self.step,
                "depth": self.depth, "n_frontier": self.n_frontier}

    def load_state_dict(self, st: dict):
        """Restores a state_dict made for a BVH with the same frontier."""
        if st["depth"] != self.depth or st["n_frontier"] != self.n_frontier:
            raise ValueError("the state belongs to another frontier")
        self.w.copy_(st["w"])
        self.m.copy_(st["m"])
        self.v.copy_(st["v"])
        self.step = int(st["step"])
        sc.sc_mlp_to_bf16(self.w, self.wb)

    def check(self):
        """Raises if a tensor-core wait ran out in a forward or training pass."""
        if int(self._status.item()) != 0:
            raise RuntimeError("tensor-core pass: a wait for the tensor cores ran out")

    def trace(self, dbvh: sc.DeviceBVH, rays, cls, hits=None, counts=None, cull: int = 1,
              work=None):
        """Seeded closest-hit traversal with the given classes."""
        import torch
        n = rays.shape[0]
        if hits is None:
            hits = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        if work is None:
            work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8,
                               device=self.device)
        sc.sc_trace_seeded(dbvh, rays, cls, self.frontier, hits, counts, cull, work)
        return hits


def primary_rays(W: int, H: int, jitter_seed: int, device="cuda"):
    """Jittered pinhole rays on the device."""
    import torch
    return torch.from_numpy(sg.pinhole(W, H, jitter_seed=jitter_seed)).to(device)
