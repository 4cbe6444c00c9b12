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


def test_mlp_forward_backward_match_reference():
    from paper_2412_01217_gb300._lib import SgMlpActs, SgMlpGrads, call
    rng = np.random.default_rng(0)
    B = 512
    net = Net()
    net.pack()
    X = torch.tensor(rng.normal(size=(B, 2048)) * 0.5, dtype=torch.float32).cuda()
    X[:, 2009:] = 0
    Xb = X.to(torch.bfloat16).contiguous()
    Xt = Xb.T.contiguous()
    T = torch.tensor(rng.normal(size=(B, 32)), dtype=torch.float32).cuda()
    w = torch.zeros(32, device="cuda")
    w[:20] = 1.0
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
    call("sg_mlp_backward", C.byref(s), _p(Xt), _p(T), _p(w), B, C.byref(A), C.byref(G), _p(loss), _p(status), _s())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    d = lambda t: t.double().cpu().numpy()
    W = [d(net.W1b), d(net.b1), d(net.W2b), d(net.b2), d(net.W3b), d(net.b3)]
    L, gref, aref = mlp.loss_and_grads(d(Xb), d(T), d(w), *W)
    rel = lambda a, b: np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
    assert rel(d(acts["Y"]), aref["Y"]) < 2e-3
    assert np.mean(d(acts["H1"]) == aref["H1"]) > 0.99    # bf16 values agree except at rounding ties
    assert float(loss.item()) == pytest.approx(L, rel=2e-3)
    for k in ("W1", "W2", "W3", "b1", "b2", "b3"):
        assert rel(d(grads[k]), gref[k]) < 1e-2, k
