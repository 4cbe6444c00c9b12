"""GPU checks of the tcgen05 GEMM and the learned-initializer MLP (through the C ABI)
against torch matmul of the same bf16 operands and against the float64 MLP reference."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("M,N,K", [(256, 128, 2048), (128, 32, 512), (384, 256, 128), (200, 96, 192),
                                   (1024, 16, 64)])
def test_tcgen05_gemm_matches_fp32_reference(M, N, K):
    from paper_2412_01217_gb300._lib import call
    torch.manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    call("sg_gemm_bf16", _p(A), K, _p(B), K, M, N, K, _p(D), N, 0, _p(status), _s())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = (A.double() @ B.double().T)
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-4, err


def test_tcgen05_gemm_split_k_accumulate():
    from paper_2412_01217_gb300._lib import call
    torch.manual_seed(3)
    M, N, K = 128, 256, 8192
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    D = torch.ones((M, N), device="cuda")
    call("sg_gemm_bf16", _p(A), K, _p(B), K, M, N, K, _p(D), N, 1, None, _s())
    torch.cuda.synchronize()
    ref = 1.0 + (A.double() @ B.double().T)
    assert (D.double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() + 1e-3


def test_tcgen05_bounded_wait_times_out_reports_and_leaves_context_usable():
    """Failure detection without a fault: every CTA waits on an mbarrier nothing arrives on,
    gives up after 1000 polls, sets SG_STATUS_TIMEOUT, writes nothing, frees its tensor
    memory and returns; the next GEMM on the same stream is correct."""
    from paper_2412_01217_gb300._lib import STATUS_TIMEOUT, call
    torch.manual_seed(7)
    M, N, K = 256, 128, 256
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    D = torch.full((M, N), 7.0, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    call("sg_gemm_bf16_timeout_probe", _p(A), K, _p(B), K, M, N, K, _p(D), N, 1000, _p(status), _s())
    torch.cuda.synchronize()
    assert int(status.item()) & STATUS_TIMEOUT
    assert torch.all(D == 7.0)
    status.zero_()
    call("sg_gemm_bf16", _p(A), K, _p(B), K, M, N, K, _p(D), N, 0, _p(status), _s())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.double() @ B.double().T
    assert (D.double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() + 1e-4


class Net:
    def __init__(self, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.W1 = (torch.randn(128, 2048, generator=g) * 0.03).cuda()
        self.W2 = (torch.randn(128, 128, generator=g) * 0.1).cuda()
        self.W3 = (torch.randn(32, 128, generator=g) * 0.1).cuda()
        self.b1 = (torch.randn(128, generator=g) * 0.1).cuda()
        self.b2 = (torch.randn(128, generator=g) * 0.1).cuda()
        self.b3 = (torch.randn(32, generator=g) * 0.1).cuda()
        bf = lambda *s: torch.zeros(*s, dtype=torch.bfloat16, device="cuda")
        self.W1b, self.W2b, self.W3b = bf(128, 2048), bf(128, 128), bf(32, 128)
        self.W2t, self.W3t = bf(128, 128), bf(128, 64)

    def pack(self):
        from paper_2412_01217_gb300._lib import call
        call("sg_mlp_pack_weights", _p(self.W1), _p(self.W2), _p(self.W3), _p(self.W1b), _p(self.W2b),
             _p(self.W3b), _p(self.W2t), _p(self.W3t), _s())

    def struct(self):
        from paper_2412_01217_gb300._lib import SgMlp
        return SgMlp(*[t.data_ptr() for t in (self.W1b, self.W2b, self.W3b, self.W2t, self.W3t, self.b1,
                                              self.b2, self.b3)])


def _decided_batch(net, B, seed):
    """Seeded inputs and targets with every row's bf16 roundings decided (oracle.mlp
    undecided_rows): undecided rows are drawn again until none is left."""
    d = lambda t: t.double().cpu().numpy()
    W = [d(net.W1b), d(net.b1), d(net.W2b), d(net.b2), d(net.W3b), d(net.b3)]
    rng = np.random.default_rng(seed)
    w = np.zeros(32)
    w[:20] = 1.0

    def draw(n):
        X = rng.normal(size=(n, 2048)) * 0.5
        X[:, 2009:] = 0
        return mlp.bf16(X), rng.normal(size=(n, 32))

    X, T = draw(B)
    for _ in range(200):
        u = mlp.undecided_rows(X, T, w, *W)
        if not u.any():
            break
        X[u], T[u] = draw(int(u.sum()))
    assert not mlp.undecided_rows(X, T, w, *W).any()
    return X, T, w, W


def test_mlp_forward_backward_match_reference():
    """Element by element against the FP64 reference with bf16 storage points, on a batch whose
    every bf16 rounding is decided for FP32 accumulation: the bf16 activations H1, H2, dY, dH2,
    dH1 are bit-identical; Y, the loss and every weight and bias gradient agree within the
    FP32 accumulation bound 2^-18 sum |terms| of each entry (dot products of up to 2048 terms,
    some 64 times their usual error)."""
    from paper_2412_01217_gb300._lib import SgMlpActs, SgMlpGrads, call
    B = 512
    net = Net()
    net.pack()
    X, T, w, W = _decided_batch(net, B, seed=0)
    Xb = torch.tensor(X, dtype=torch.float32).cuda().to(torch.bfloat16).contiguous()
    Xt = Xb.T.contiguous()
    Tt = torch.tensor(T, dtype=torch.float32).cuda()
    wt = torch.tensor(w, dtype=torch.float32).cuda()
    bf = lambda *s: torch.zeros(*s, dtype=torch.bfloat16, device="cuda")
    acts = dict(H1=bf(B, 128), H1t=bf(128, B), H2=bf(B, 128), H2t=bf(128, B), Y=torch.zeros(B, 32, device="cuda"),
                dY=bf(B, 64), dYt=bf(32, B), dH2=bf(B, 128), dH2t=bf(128, B), dH1t=bf(128, B))
    A = SgMlpActs(*[acts[k].data_ptr() for k in ("H1", "H1t", "H2", "H2t", "Y", "dY", "dYt", "dH2", "dH2t", "dH1t")])
    grads = dict(W1=torch.zeros(128, 2048, device="cuda"), W2=torch.zeros(128, 128, device="cuda"),
                 W3=torch.zeros(32, 128, device="cuda"), b1=torch.zeros(128, device="cuda"),
                 b2=torch.zeros(128, device="cuda"), b3=torch.zeros(32, device="cuda"))
    G = SgMlpGrads(*[grads[k].data_ptr() for k in ("W1", "W2", "W3", "b1", "b2", "b3")])
    loss = torch.zeros(1, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = net.struct()
    call("sg_mlp_forward", C.byref(s), _p(Xb), B, C.byref(A), _p(status), _s())
    call("sg_mlp_backward", C.byref(s), _p(Xt), _p(Tt), _p(wt), B, C.byref(A), C.byref(G), _p(loss), _p(status), _s())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    d = lambda t: t.double().cpu().numpy()
    W1, b1, W2, b2, W3, b3 = W
    L, gref, aref = mlp.loss_and_grads(X, T, w, *W)
    # the bf16 activations: bit-identical (every rounding decided), in both layouts
    H1, H2 = aref["H1"], aref["H2"]
    dY = mlp.bf16(2.0 * w[None] * (aref["Y"] - T) / B)
    dH2 = mlp.bf16((dY @ W3) * (H2 > 0))
    dH1 = mlp.bf16((dH2 @ W2) * (H1 > 0))
    for name, got, ref in (("H1", d(acts["H1"]), H1), ("H1t", d(acts["H1t"]).T, H1), ("H2", d(acts["H2"]), H2),
                           ("H2t", d(acts["H2t"]).T, H2), ("dY", d(acts["dY"])[:, :32], dY),
                           ("dYt", d(acts["dYt"]).T, dY), ("dH2", d(acts["dH2"]), dH2), ("dH2t", d(acts["dH2t"]).T, dH2),
                           ("dH1t", d(acts["dH1t"]).T, dH1)):
        assert np.array_equal(got, ref), f"{name}: {int((got != ref).sum())} entries differ"
    assert not d(acts["dY"])[:, 32:].any()
    eps = 2.0 ** -18
    a = np.abs
    bound_Y = eps * (H2 @ a(W3).T + a(b3))
    assert np.all(a(d(acts["Y"]) - aref["Y"]) <= bound_Y), "Y"
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    bounds = dict(W1=a(dH1).T @ a(X), W2=a(dH2).T @ H1, W3=a(dY).T @ H2, b1=a(dH1).sum(0), b2=a(dH2).sum(0),
                  b3=a(dY).sum(0))
    for k, bnd in bounds.items():
        err = a(d(grads[k]) - gref[k])
        assert np.all(err <= eps * bnd + 1e-30), (k, float((err / (bnd + 1e-30)).max()))
        assert np.count_nonzero(gref[k]) > 0.5 * gref[k].size, k
