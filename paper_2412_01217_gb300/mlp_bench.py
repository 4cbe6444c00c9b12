"""Timing of the learned initializer's network on the tcgen05 kernels: the forward (three
GEMMs with fused bias / ReLU / bf16 epilogues) and the backward of one batch, with CUDA
events after warm-up, and the layer-1 GEMM's achieved TFLOP/s and HBM bytes per second.

Run: python -m paper_2412_01217_gb300.mlp_bench [--batch 4096 16384 65536] [--reps 20]
Prints one JSON line per batch size.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json

import torch

from . import _lib
from ._lib import SgMlpGrads, call
from .learned_init import IN, MLPInit


def _events(fn, reps):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps / 1e3


def time_batch(B, reps=20, seed=0):
    _lib.load()
    mlp = MLPInit(seed=seed)
    g = torch.Generator(device="cuda").manual_seed(seed)
    X = (torch.randn(B, IN, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    Xt = X.T.contiguous()
    T = torch.randn(B, 32, device="cuda", generator=g)
    a, s = mlp.acts(B)
    net = mlp.net()
    st = lambda: C.c_void_p(torch.cuda.current_stream().cuda_stream)
    grads = SgMlpGrads(*[t.data_ptr() for t in mlp.grads])
    loss = torch.zeros(1, device="cuda")

    def fwd():
        call("sg_mlp_forward", C.byref(net), C.c_void_p(X.data_ptr()), B, C.byref(s), C.c_void_p(mlp.status.data_ptr()),
             st())

    def bwd():
        call("sg_mlp_backward", C.byref(net), C.c_void_p(Xt.data_ptr()), C.c_void_p(T.data_ptr()),
             C.c_void_p(mlp.out_w.data_ptr()), B, C.byref(s), C.byref(grads), C.c_void_p(loss.data_ptr()),
             C.c_void_p(mlp.status.data_ptr()), st())

    # layer 1's GEMM alone: X W1^T into fp32 (the forward adds the bias / ReLU / bf16 epilogue)
    def layer1():
        call("sg_gemm_bf16", C.c_void_p(X.data_ptr()), IN, C.c_void_p(mlp.W1b.data_ptr()), IN, B, 128, IN,
             C.c_void_p(l1_out.data_ptr()), 128, 0,
             C.c_void_p(mlp.status.data_ptr()), st())

    l1_out = torch.empty(B, 128, device="cuda")
    for f in (fwd, bwd, layer1):
        for _ in range(3):
            f()
    torch.cuda.synchronize()
    t_fwd, t_bwd, t_l1 = _events(fwd, reps), _events(bwd, reps), _events(layer1, reps)
    assert int(mlp.status.item()) == 0
    l1_flops = 2.0 * B * 128 * IN
    l1_bytes = B * IN * 2 + 128 * IN * 2 + B * 128 * 4
    return {"batch": B, "forward_us": t_fwd * 1e6, "backward_us": t_bwd * 1e6, "layer1_us": t_l1 * 1e6,
            "layer1_tflops": l1_flops / t_l1 / 1e12, "layer1_GBps": l1_bytes / t_l1 / 1e9,
            "layer1_bytes": l1_bytes, "layer1_flops": l1_flops}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, nargs="+", default=[4096, 16384, 65536])
    ap.add_argument("--reps", type=int, default=20)
    args = ap.parse_args()
    for B in args.batch:
        print(json.dumps(time_batch(B, args.reps)), flush=True)


if __name__ == "__main__":
    main()
