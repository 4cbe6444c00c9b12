"""The loss entry point for callers that cannot allocate device memory.

Some callers get their input and output buffers from a host framework that owns all of
the device's memory and offers this library no way to obtain scratch space; others run on
a latency-critical thread where a cudaMalloc could block on other device work.  For them
sg_pyramid_loss_noalloc uses scratch built into the library instead of a workspace.  This
test calls it through the C ABI twice in a row and checks that each call gives the same
loss terms and image gradients as sg_pyramid_loss with a caller-provided workspace.  The
file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(seed, W=160, H=96, levels=3, n_cams=2, Cs=16, K=32):
    import synthetic
    from paper_2412_01217_gb300.splat import make_views, views_to_device
    rng = np.random.default_rng(seed)
    intr = dict(W=W, H=H, fx=W / 2.0, fy=W / 2.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5)
    cams = synthetic.Room(seed=3).trajectory(n_cams, intr, seed=7)
    views, P, _ = make_views(cams, levels)
    dev = torch.device("cuda")
    t = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device=dev)
    depth = rng.uniform(1, 3, size=P)
    depth[rng.uniform(size=P) < 0.1] = 0.0
    return dict(views=views, dviews=views_to_device(views, dev), V=n_cams * levels, P=P, C=Cs, K=K,
                r_rgb=t(rng.uniform(size=3 * P)), r_depth=t(rng.uniform(1, 3, size=P)),
                r_sem=t(rng.normal(size=Cs * P)), g_rgb=t(rng.uniform(size=3 * P)), g_depth=t(depth),
                g_label=t(rng.integers(-1, K, size=P), torch.int32), dec=t(rng.normal(size=(K, Cs)) * 0.3))


def _call(x, noalloc):
    from paper_2412_01217_gb300._lib import SgImages, SgLossConfig, SgTargets, call, load
    lib = load()
    P, Cs, K = x["P"], x["C"], x["K"]
    rendered = SgImages(x["r_rgb"].data_ptr(), x["r_depth"].data_ptr(), x["r_sem"].data_ptr())
    gt = SgTargets(x["g_rgb"].data_ptr(), x["g_depth"].data_ptr(), x["g_label"].data_ptr(), None)
    dL = [torch.full((n * P,), float("nan"), device="cuda") for n in (3, 1, Cs)]
    dLi = SgImages(*[d.data_ptr() for d in dL])
    dec_grad = torch.zeros(K, Cs, device="cuda")
    lc = SgLossConfig(0.2, 0.2, 1.0, 1.0, 0, K, x["dec"].data_ptr(), dec_grad.data_ptr())
    terms = torch.full((4 * x["V"],), float("nan"), device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if noalloc:
        call("sg_pyramid_loss_noalloc", C.byref(rendered), C.byref(gt), C.c_void_p(x["dviews"].data_ptr()),
             x["views"], x["V"], Cs, C.byref(lc), C.c_void_p(terms.data_ptr()), C.byref(dLi), None, stream)
    else:
        ws = torch.zeros(lib.sg_loss_workspace_size(x["views"], x["V"], Cs, K), dtype=torch.uint8, device="cuda")
        call("sg_pyramid_loss", C.byref(rendered), C.byref(gt), C.c_void_p(x["dviews"].data_ptr()), x["views"],
             x["V"], Cs, C.byref(lc), C.c_void_p(terms.data_ptr()), C.byref(dLi), C.c_void_p(ws.data_ptr()),
             ws.numel(), None, stream)
    torch.cuda.synchronize()
    return [terms.cpu().numpy(), *[d.cpu().numpy() for d in dL], dec_grad.cpu().numpy()]


def test_noalloc_loss_matches_workspace_loss_on_two_calls():
    for call_no, seed in enumerate((0, 1)):
        x = _inputs(seed)
        ref = _call(x, noalloc=False)
        got = _call(x, noalloc=True)
        for name, g, r in zip(("terms", "dL_rgb", "dL_depth", "dL_sem", "dL_decoder"), got, ref):
            assert np.isfinite(g).all(), (call_no, name)
            scale = np.abs(r).max()
            assert np.allclose(g, r, rtol=1e-5, atol=1e-6 * scale), (call_no, name)


def test_noalloc_loss_rejects_images_beyond_its_scratch():
    from paper_2412_01217_gb300._lib import SgError
    # 2048 x 2048 pixels with a decoder gradient need more than the built-in 16 MiB
    import synthetic
    from paper_2412_01217_gb300.splat import make_views, views_to_device
    big = synthetic.make_camera(2048, 2048, 1000.0, 1000.0, 1023.5, 1023.5)
    views, P, _ = make_views([big], 1)
    x = dict(views=views, dviews=views_to_device(views, torch.device("cuda")), V=1, P=P, C=16, K=32)
    dev = torch.device("cuda")
    for k, n in (("r_rgb", 3), ("r_depth", 1), ("r_sem", 16), ("g_rgb", 3), ("g_depth", 1)):
        x[k] = torch.zeros(n * P, device=dev)
    x["g_label"] = torch.zeros(P, dtype=torch.int32, device=dev)
    x["dec"] = torch.zeros(32, 16, device=dev)
    with pytest.raises(SgError) as e:
        _call(x, noalloc=True)
    assert e.value.code == 2 and "scratch" in str(e.value)


def test_noalloc_loss_matches_workspace_loss_in_paper_mode():
    """The paper's semantic term (Eq. 12: L1 + D-SSIM on a semantic colour image, 8 planes)
    takes its own partial-sum block of the built-in scratch: same terms and image gradients
    as with a caller workspace, on two calls in a row."""
    from paper_2412_01217_gb300._lib import SgImages, SgLossConfig, SgTargets, call, load
    lib = load()
    for seed in (2, 3):
        x = _inputs(seed, Cs=8, K=8)
        rng = np.random.default_rng(seed + 10)
        g_sem = torch.tensor(rng.uniform(size=8 * x["P"]), dtype=torch.float32, device="cuda")
        r_sem = torch.tensor(rng.uniform(size=8 * x["P"]), dtype=torch.float32, device="cuda")
        outs = []
        for noalloc in (False, True):
            P, Cs = x["P"], 8
            rendered = SgImages(x["r_rgb"].data_ptr(), x["r_depth"].data_ptr(), r_sem.data_ptr())
            gt = SgTargets(x["g_rgb"].data_ptr(), x["g_depth"].data_ptr(), x["g_label"].data_ptr(), g_sem.data_ptr())
            dL = [torch.full((n * P,), float("nan"), device="cuda") for n in (3, 1, Cs)]
            dLi = SgImages(*[d.data_ptr() for d in dL])
            # a decoder gradient buffer given in paper mode is ignored (no decoder there) and
            # reserves no scratch: the same sizing rule as the workspace call
            dgrad = torch.zeros(Cs, Cs, device="cuda")
            lc = SgLossConfig(0.2, 0.2, 1.0, 1.0, 1, Cs, None, dgrad.data_ptr())
            terms = torch.full((4 * x["V"],), float("nan"), device="cuda")
            stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
            if noalloc:
                call("sg_pyramid_loss_noalloc", C.byref(rendered), C.byref(gt), C.c_void_p(x["dviews"].data_ptr()),
                     x["views"], x["V"], Cs, C.byref(lc), C.c_void_p(terms.data_ptr()), C.byref(dLi), None, stream)
            else:
                ws = torch.zeros(lib.sg_loss_workspace_size(x["views"], x["V"], Cs, Cs), dtype=torch.uint8,
                                 device="cuda")
                call("sg_pyramid_loss", C.byref(rendered), C.byref(gt), C.c_void_p(x["dviews"].data_ptr()),
                     x["views"], x["V"], Cs, C.byref(lc), C.c_void_p(terms.data_ptr()), C.byref(dLi),
                     C.c_void_p(ws.data_ptr()), ws.numel(), None, stream)
            torch.cuda.synchronize()
            outs.append([terms.cpu().numpy(), *[d.cpu().numpy() for d in dL]])
        for name, r, g in zip(("terms", "dL_rgb", "dL_depth", "dL_sem"), *outs):
            assert np.isfinite(g).all(), (seed, name)
            assert np.allclose(g, r, rtol=1e-5, atol=1e-6 * np.abs(r).max()), (seed, name)
        assert np.abs(outs[0][3]).max() > 0   # the semantic term has a gradient
        assert not dgrad.any()


def _sized_inputs(W, H, seed=5, Cs=16, K=32):
    """One W x H view-level with random rendered and target images."""
    import synthetic
    from paper_2412_01217_gb300.splat import make_views, views_to_device
    rng = np.random.default_rng(seed)
    views, P, _ = make_views([synthetic.make_camera(W, H, W / 2.0, W / 2.0, W / 2 - 0.5, H / 2 - 0.5)], 1)
    dev = torch.device("cuda")
    t = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device=dev)
    return dict(views=views, dviews=views_to_device(views, dev), V=1, P=P, C=Cs, K=K,
                r_rgb=t(rng.uniform(size=3 * P)), r_depth=t(rng.uniform(1, 3, size=P)),
                r_sem=t(rng.normal(size=Cs * P)), g_rgb=t(rng.uniform(size=3 * P)), g_depth=t(rng.uniform(1, 3, size=P)),
                g_label=t(rng.integers(-1, K, size=P), torch.int32), dec=t(rng.normal(size=(K, Cs)) * 0.3))


def test_noalloc_loss_at_the_edge_of_its_scratch():
    """An image whose scratch need (sg_loss_workspace_size, cross-entropy with a 32 x 16 decoder
    gradient) lies just under the built-in 16 MiB uses the last partial-sum blocks of the array
    and matches the workspace call on two calls in a row; one row more is rejected."""
    from paper_2412_01217_gb300._lib import SgError, load
    from paper_2412_01217_gb300.splat import make_views
    import synthetic
    lib = load()
    limit = 16 << 20
    W = 1920

    def need(H):
        v, _, _ = make_views([synthetic.make_camera(W, H, W / 2.0, W / 2.0, W / 2 - 0.5, H / 2 - 0.5)], 1)
        return lib.sg_loss_workspace_size(v, 1, 16, 32)

    lo, hi = 1, 4096
    while hi - lo > 1:  # largest H whose need fits
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if need(mid) <= limit else (lo, mid)
    H = lo
    assert need(H) > 0.99 * limit and need(H + 1) > limit
    for seed in (7, 8):
        x = _sized_inputs(W, H, seed=seed)
        ref = _call(x, noalloc=False)
        got = _call(x, noalloc=True)
        for name, g, r in zip(("terms", "dL_rgb", "dL_depth", "dL_sem", "dL_decoder"), got, ref):
            assert np.isfinite(g).all(), (seed, name)
            assert np.allclose(g, r, rtol=1e-5, atol=1e-6 * np.abs(r).max()), (seed, name)
    x = _sized_inputs(W, H + 1, seed=9)
    with pytest.raises(SgError) as e:
        _call(x, noalloc=True)
    assert e.value.code == 2 and "scratch" in str(e.value)


def test_noalloc_loss_checks_arguments_before_sizing():
    """Invalid arguments give SG_ERR_INVALID_ARG (the workspace call's checks), not a
    capacity error computed from them."""
    from paper_2412_01217_gb300._lib import SgError, SgImages, SgLossConfig, SgTargets, call
    x = _inputs(4)
    P = x["P"]
    rendered = SgImages(x["r_rgb"].data_ptr(), x["r_depth"].data_ptr(), x["r_sem"].data_ptr())
    gt = SgTargets(x["g_rgb"].data_ptr(), x["g_depth"].data_ptr(), x["g_label"].data_ptr(), None)
    dL = [torch.zeros(n * P, device="cuda") for n in (3, 1, 16)]
    dLi = SgImages(*[d.data_ptr() for d in dL])
    terms = torch.zeros(4 * x["V"], device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for lc in (SgLossConfig(0.2, 0.2, 1.0, 1.0, 0, -5, x["dec"].data_ptr(), None),   # negative classes
               SgLossConfig(0.2, 0.2, 1.0, 1.0, 0, 32, None, None)):                 # 32 classes, no decoder
        with pytest.raises(SgError) as e:
            call("sg_pyramid_loss_noalloc", C.byref(rendered), C.byref(gt), C.c_void_p(x["dviews"].data_ptr()),
                 x["views"], x["V"], 16, C.byref(lc), C.c_void_p(terms.data_ptr()), C.byref(dLi), None, stream)
        assert e.value.code == 1
