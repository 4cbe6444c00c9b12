"""The learned initializer: a 3-layer BF16 MLP (2048 -> 128 -> 128 -> 32) that proposes the
log-scale, opacity logit and semantic feature of newly inserted Gaussians from 7x7 RGB-D-
semantic patches.  Training and inference run in the tcgen05 kernels behind the C ABI
(sg_mlp_forward / sg_mlp_backward / sg_adam_multi / sg_mlp_pack_weights); PyTorch only
holds the buffers.

The paper inserts Gaussians from keyframes (Sec. III-A) without saying how their initial
shape, opacity and semantics are chosen; the heuristic initializer (sg_init_gaussians)
is the plain form and this network is the learned form.
"""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import _lib
from ._lib import SgAdamGroup, SgMlp, SgMlpActs, SgMlpGrads, call

IN, HID, OUT = 2048, 128, 32
USED_OUT = 20  # log-scale 3, opacity logit 1, semantic feature 16


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class MLPInit:
    def __init__(self, seed=0, device="cuda", lr=1e-3):
        _lib.load()
        g = torch.Generator().manual_seed(seed)
        dev = torch.device(device)
        # He-style initialisation of the fp32 master weights ([out][in])
        self.W1 = (torch.randn(HID, IN, generator=g) * math.sqrt(2.0 / 2009)).to(dev)
        self.W1[:, 2009:] = 0
        self.W2 = (torch.randn(HID, HID, generator=g) * math.sqrt(2.0 / HID)).to(dev)
        self.W3 = (torch.randn(OUT, HID, generator=g) * math.sqrt(1.0 / HID)).to(dev)
        self.b1 = torch.zeros(HID, device=dev)
        self.b2 = torch.zeros(HID, device=dev)
        self.b3 = torch.zeros(OUT, device=dev)
        self.params = [self.W1, self.W2, self.W3, self.b1, self.b2, self.b3]
        self.grads = [torch.zeros_like(t) for t in self.params]
        self.m = [torch.zeros_like(t) for t in self.params]
        self.v = [torch.zeros_like(t) for t in self.params]
        bf = lambda *s: torch.zeros(*s, dtype=torch.bfloat16, device=dev)
        self.W1b, self.W2b, self.W3b = bf(HID, IN), bf(HID, HID), bf(OUT, HID)
        self.W2t, self.W3t = bf(HID, HID), bf(HID, 64)
        self.lr = lr
        self.step_count = 0
        self.y_mean = torch.zeros(OUT, device=dev)
        self.y_std = torch.ones(OUT, device=dev)
        self.out_w = torch.zeros(OUT, device=dev)
        self.out_w[:USED_OUT] = 1.0 / USED_OUT
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.device = dev
        self._acts = {}
        self.pack()

    def pack(self):
        call("sg_mlp_pack_weights", _p(self.W1), _p(self.W2), _p(self.W3), _p(self.W1b), _p(self.W2b),
             _p(self.W3b), _p(self.W2t), _p(self.W3t), _s())

    def net(self):
        return SgMlp(*[t.data_ptr() for t in (self.W1b, self.W2b, self.W3b, self.W2t, self.W3t, self.b1,
                                              self.b2, self.b3)])

    def acts(self, B):
        if B not in self._acts:
            bf = lambda *s: torch.zeros(*s, dtype=torch.bfloat16, device=self.device)
            a = dict(H1=bf(B, HID), H1t=bf(HID, B), H2=bf(B, HID), H2t=bf(HID, B),
                     Y=torch.zeros(B, OUT, device=self.device), dY=bf(B, 64), dYt=bf(OUT, B), dH2=bf(B, HID),
                     dH2t=bf(HID, B), dH1t=bf(HID, B))
            s = SgMlpActs(*[a[k].data_ptr() for k in ("H1", "H1t", "H2", "H2t", "Y", "dY", "dYt", "dH2", "dH2t",
                                                       "dH1t")])
            self._acts[B] = (a, s)
        return self._acts[B]

    def set_standardisation(self, T):
        """Per-output mean/std of the (un-standardised) training targets T [n][32]."""
        self.y_mean = T.mean(0)
        self.y_std = T.std(0).clamp_min(1e-3)
        self.y_mean[USED_OUT:] = 0
        self.y_std[USED_OUT:] = 1

    def forward(self, X, B):
        a, s = self.acts(B)
        net = self.net()
        call("sg_mlp_forward", C.byref(net), _p(X), B, C.byref(s), _p(self.status), _s())
        return a["Y"]

    def train_step(self, X, Xt, T_std, B, loss_acc):
        """One Adam step on a batch: X [B][2048], Xt [2048][B] bf16, standardised targets."""
        a, s = self.acts(B)
        net = self.net()
        G = SgMlpGrads(*[t.data_ptr() for t in self.grads])
        call("sg_mlp_forward", C.byref(net), _p(X), B, C.byref(s), _p(self.status), _s())
        call("sg_mlp_backward", C.byref(net), _p(Xt), _p(T_std), _p(self.out_w), B, C.byref(s), C.byref(G),
             _p(loss_acc), _p(self.status), _s())
        self.step_count += 1
        groups = (SgAdamGroup * 6)(*[SgAdamGroup(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(),
                                                  p.numel(), self.lr)
                                     for p, g, m, v in zip(self.params, self.grads, self.m, self.v)])
        call("sg_adam_multi", groups, 6, 0.9, 0.999, 1e-8, self.step_count, 1, None, _s())
        self.W1[:, 2009:] = 0  # padding features stay inert
        self.pack()

    def fit(self, X, T, epochs=3, batch=None, seed=0, log=None):
        """X: bf16 [n][2048]; T: fp32 [n][32] raw targets.  batch: rows per Adam step (a
        multiple of 128); default 16384 when that still gives 32 steps per epoch, else 4096
        (large batches keep the tensor cores and HBM busy: the layer-1 GEMM streams its
        operand at about 2.8 TB/s at 65536 rows and is latency-bound below 16384).  The
        learning rate grows with the square root of the batch from 1e-3 at 4096."""
        n = X.shape[0]
        if batch is None:
            batch = 16384 if n >= 32 * 16384 else 4096
        base_lr = self.lr
        self.lr = base_lr * math.sqrt(batch / 4096)
        self.set_standardisation(T)
        T_std = ((T - self.y_mean) / self.y_std).contiguous()
        loss = torch.zeros(1, device=self.device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        history = []
        n_batches = n // batch
        # every batch's transposed input [2048][batch] once, contiguous (the weight gradient of
        # layer 1 reads it K-major)
        Xb = X[:n_batches * batch].view(n_batches, batch, IN)
        Xtb = Xb.transpose(1, 2).contiguous()
        for ep in range(epochs):
            perm = torch.randperm(n_batches, generator=g)
            loss.zero_()
            for bi in perm.tolist():
                sl = slice(bi * batch, (bi + 1) * batch)
                self.train_step(Xb[bi], Xtb[bi], T_std[sl], batch, loss)
            history.append(float(loss.item()) / max(1, n_batches))
            if log:
                log(f"epoch {ep}: loss {history[-1]:.4f}")
        self.lr = base_lr
        return history

    def predict(self, X, B):
        """Raw (de-standardised) outputs [B][32] for bf16 rows X [B][2048]."""
        Y = self.forward(X, B)
        return Y * self.y_std + self.y_mean

    def state_dict(self):
        return {k: getattr(self, k).detach().cpu() for k in ("W1", "W2", "W3", "b1", "b2", "b3", "y_mean", "y_std")}

    def load_state_dict(self, sd):
        for k, v in sd.items():
            getattr(self, k).copy_(v.to(self.device))
        self.pack()
