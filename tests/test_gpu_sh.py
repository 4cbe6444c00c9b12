"""GPU parity of the view-dependent (spherical-harmonic) colour and semantic feature of
Sec. III-B against the FP64 oracle: the projection's per-record colour / semantic feature
feeds the compositing kernels, and the adjoint chains the per-record gradients to the SH
coefficients, rgb / sem and the mean.  Same
tolerances as the other parity tests (forward 1e-4 rel + 1e-5 abs, gradients 2e-3 rel +
1e-5 of the group's largest entry)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import AMBIGUOUS_GRAD, FWD_ABS, FWD_REL, MAX_MASKED, check_close, check_grads, ref_render, unambiguous
from test_gpu_parity import f32_camera, oracle_cams, room_small, view_images

pytestmark = pytest.mark.gpu

BASE = ("mean", "log_scale", "quat", "opacity_logit", "rgb", "sem")
KEYS = BASE + ("sh",)


def make(g, cams, levels=1, **kw):
    from paper_2412_01217_gb300 import PyramidRasterizer, RenderConfig, to_device_params
    from paper_2412_01217_gb300.splat import sh_degree
    p = to_device_params(g)
    r = PyramidRasterizer(g["mean"].shape[0], g["sem"].shape[1], cams, levels, RenderConfig(**kw),
                          sh_degree=sh_degree(p), sem_sh="sem_sh" in p)
    return r, p


def sh_cloud(degree, n=2000, seed=1, colour=True, semantic=False):
    g = synthetic.cloud_scene(n, 8, seed=seed)
    if colour:
        g["sh"] = synthetic.sh_coefficients(n, degree, seed=seed + 10)
    if semantic:
        g["sem_sh"] = synthetic.sh_coefficients(n, degree, seed=seed + 20, channels=8, scale=0.5)
    # a camera away from the origin and turned a little, so that the centre -R^T t and the
    # rotation both enter the view directions
    cam = synthetic.cloud_camera()
    a = 0.15
    R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    cam = f32_camera(dict(cam, R_cw=R, t_cw=np.array([0.1, -0.05, 0.3])))
    return g, cam


def upstream(ref_f, H, W, C, seed):
    keep = unambiguous(ref_f["flags"], AMBIGUOUS_GRAD).astype(np.float64)
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(3, H, W)) * keep, rng.normal(size=(H, W)) * keep,
            rng.normal(size=(C, H, W)) * keep)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_sh_forward_matches_oracle(degree):
    g, cam = sh_cloud(degree)
    r, p = make(g, [cam])
    r.forward(p)
    got = view_images(r, 0, 8)
    ref = ref_render(g, cam)
    amb = ~unambiguous(ref["flags"], limit=max(MAX_MASKED, 1.0 / ref["flags"].size))
    for k in ("rgb", "depth", "sem", "T"):
        check_close(k, got[k], ref[k], FWD_REL, FWD_ABS, mask=~amb)
    # the SH term is not negligible in this scene: without it the image differs
    ref0 = ref_render({k: v for k, v in g.items() if k != "sh"}, cam)
    assert np.abs(ref0["rgb"] - ref["rgb"]).max() > 0.05


@pytest.mark.parametrize("degree, colour, semantic", [(2, False, True), (3, True, True)])
def test_semantic_sh_forward_matches_oracle(degree, colour, semantic):
    g, cam = sh_cloud(degree, seed=5, colour=colour, semantic=semantic)
    r, p = make(g, [cam])
    r.forward(p)
    got = view_images(r, 0, 8)
    ref = ref_render(g, cam)
    amb = ~unambiguous(ref["flags"])
    for k in ("rgb", "depth", "sem", "T"):
        check_close(k, got[k], ref[k], FWD_REL, FWD_ABS, mask=~amb)
    ref0 = ref_render({k: v for k, v in g.items() if k != "sem_sh"}, cam)
    assert np.abs(ref0["sem"] - ref["sem"]).max() > 0.05


@pytest.mark.parametrize("degree, ppt, colour, semantic", [(1, 1, True, False), (2, 2, True, False), (3, 1, True, False),
                                                           (3, 4, True, False), (2, 1, False, True),
                                                           (1, 2, True, True), (3, 1, True, True), (2, 0, True, True)])
def test_sh_backward_matches_oracle(degree, ppt, colour, semantic):
    """ppt 0: 8x8 tiles with half masks (the adjoint one warp per half tile, one pixel per
    thread)."""
    g, cam = sh_cloud(degree, seed=degree, colour=colour, semantic=semantic)
    kw = dict(tile_w=8, tile_h=8, pixels_per_thread_bwd=1, half_masks=True,
              half_tile_fwd=True) if ppt == 0 else \
        dict(pixels_per_thread_bwd=ppt)
    r, p = make(g, [cam], **kw)
    r.forward(p)
    ref_f = ref_render(g, cam)
    H, W = cam["H"], cam["W"]
    up = upstream(ref_f, H, W, 8, seed=20 + degree)
    dl = tuple(torch.tensor(u.reshape(-1), dtype=torch.float32, device="cuda") for u in up)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    r.backward(p, grads, dL=dl)
    got = {k: v.cpu().numpy() for k, v in grads.items()}
    up32 = [t.cpu().numpy().astype(np.float64).reshape(u.shape) for t, u in zip(dl, up)]
    ref = oracle.render_backward(g, cam, *up32)
    check_grads(got, ref, BASE + tuple(k for k in ("sh", "sem_sh") if k in g))
    # every workspace block (2D, record colour and record semantic gradients) is left zero
    assert not r.bwd_ws.any() and not r.work_counter.any()


def test_sh_multiview_pyramid_matches_oracle():
    """Two keyframes x three levels with degree-3 colour and semantic feature: every
    view-level's image and the summed gradients; the levels of one keyframe share its camera
    centre."""
    room, g, cams = room_small(n=6000, ncam=2, W=160, H=96)
    g["sh"] = synthetic.sh_coefficients(6000, 3, seed=7)
    g["sem_sh"] = synthetic.sh_coefficients(6000, 3, seed=8, channels=16)
    r, p = make(g, cams, levels=3)
    r.forward(p)
    ocams = oracle_cams(cams, 3)
    rng = np.random.default_rng(5)
    dl = [torch.zeros(3 * r.P, device="cuda"), torch.zeros(r.P, device="cuda"), torch.zeros(16 * r.P, device="cuda")]
    for v, oc in enumerate(ocams):
        got = view_images(r, v, 16)
        ref = ref_render(g, oc)
        amb = ~unambiguous(ref["flags"], limit=max(MAX_MASKED, 1.0 / ref["flags"].size))
        for k in ("rgb", "depth", "sem", "T"):
            check_close(f"v{v} {k}", got[k], ref[k], FWD_REL, FWD_ABS, mask=~amb)
        a, b, c = upstream(ref, oc["H"], oc["W"], 16, seed=v)
        r.view_slice(dl[0], v, 3).copy_(torch.tensor(a, dtype=torch.float32))
        r.view_slice(dl[1], v, 1).copy_(torch.tensor(b[None], dtype=torch.float32))
        r.view_slice(dl[2], v, 16).copy_(torch.tensor(c, dtype=torch.float32))
    grads = {k: torch.zeros_like(t) for k, t in p.items()}
    r.backward(p, grads, dL=tuple(dl))
    got = {k: t.cpu().numpy() for k, t in grads.items()}
    keys = KEYS + ("sem_sh",)
    ref = {k: 0.0 for k in keys}
    for v, oc in enumerate(ocams):
        a = r.view_slice(dl[0], v, 3).cpu().numpy().astype(np.float64)
        b = r.view_slice(dl[1], v, 1)[0].cpu().numpy().astype(np.float64)
        c = r.view_slice(dl[2], v, 16).cpu().numpy().astype(np.float64)
        rv = oracle.render_backward(g, oc, a, b, c)
        for k in keys:
            ref[k] = ref[k] + rv[k]
    check_grads(got, ref, keys)
    assert not r.bwd_ws.any()


def test_zero_sh_equals_plain_colour_path():
    """Zero SH coefficients route colour through the per-record buffers, yet give the plain
    path's images and gradients (up to the order of the float32 atomic sums)."""
    g, cam = sh_cloud(2, seed=4)
    g["sh"] = np.zeros_like(g["sh"])
    plain = {k: v for k, v in g.items() if k != "sh"}
    r1, p1 = make(g, [cam])
    r0, p0 = make(plain, [cam])
    r1.forward(p1)
    r0.forward(p0)
    for k in ("rgb", "depth", "sem", "T", "n_contrib"):
        assert np.array_equal(view_images(r1, 0, 8)[k], view_images(r0, 0, 8)[k]), k
    rng = np.random.default_rng(0)
    dl = (torch.tensor(rng.normal(size=3 * r0.P), dtype=torch.float32, device="cuda"),
          torch.tensor(rng.normal(size=r0.P), dtype=torch.float32, device="cuda"),
          torch.tensor(rng.normal(size=8 * r0.P), dtype=torch.float32, device="cuda"))
    g1 = {k: torch.zeros_like(v) for k, v in p1.items()}
    g0 = {k: torch.zeros_like(v) for k, v in p0.items()}
    r1.backward(p1, g1, dL=dl)
    r0.backward(p0, g0, dL=dl)
    for k in ("mean", "log_scale", "quat", "opacity_logit", "rgb", "sem"):
        a, b = g1[k].cpu().numpy(), g0[k].cpu().numpy()
        assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * (np.abs(b).max() + 1e-12)), k


def test_sh_autograd_and_mapping_step():
    """pyramid_splat returns the SH gradient through autograd, and a captured mapping step
    updates the SH coefficients with their own Adam group."""
    from paper_2412_01217_gb300 import MappingStep, build_pyramid, pyramid_splat
    g, cam = sh_cloud(3, n=3000, seed=6, semantic=True)
    r, p = make(g, [cam])
    leaf = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    rgb, depth, sem = pyramid_splat(r, leaf)
    (rgb.square().sum() + 0.1 * depth.sum() + sem.square().sum()).backward()
    direct = {k: torch.zeros_like(v) for k, v in p.items()}
    r.forward(p)
    r.backward(p, direct, dL=(2 * r.img_rgb, torch.full_like(r.img_depth, 0.1), 2 * r.img_sem))
    for k in ("sh", "sem_sh"):
        assert leaf[k].grad is not None and leaf[k].grad.abs().max() > 0
        assert torch.allclose(leaf[k].grad, direct[k], rtol=1e-4, atol=1e-6 * float(direct[k].abs().max()))

    tgt = synthetic.random_targets(cam["H"], cam["W"], 8, seed=3)
    gt = build_pyramid(r, [tgt["rgb"]], [tgt["depth"]], [tgt["label"]])
    step = MappingStep(r, {k: v.clone() for k, v in p.items()}, gt)
    sh0, ssh0 = step.p["sh"].clone(), step.p["sem_sh"].clone()
    step.step()
    loss1 = step.total_loss()
    step.capture()
    for _ in range(20):
        step.replay()
    torch.cuda.synchronize()
    assert np.isfinite(step.total_loss()) and step.total_loss() < loss1
    assert not torch.equal(step.p["sh"], sh0) and not torch.equal(step.p["sem_sh"], ssh0)


def test_sh_with_eq2_isotropic_projection():
    """Degree-2 colour and semantic SH together with the Eq. 2 isotropic projection (the
    projection kernels' SH template and their isotropic branch in one launch): every image
    channel and all gradient groups against the oracle; the rotation and the unused
    log-scales get exactly zero."""
    g, cam = sh_cloud(2, seed=9, colour=True, semantic=True)
    r, p = make(g, [cam], isotropic=True)
    r.forward(p)
    ocfg = dict(isotropic=1)
    ref_f = ref_render(g, cam, ocfg)
    amb = ~unambiguous(ref_f["flags"], limit=max(MAX_MASKED, 1.0 / ref_f["flags"].size))
    got = view_images(r, 0, 8)
    for k in ("rgb", "depth", "sem", "T"):
        check_close(k, got[k], ref_f[k], FWD_REL, FWD_ABS, mask=~amb)
    up = upstream(ref_f, cam["H"], cam["W"], 8, seed=31)
    dl = tuple(torch.tensor(u.reshape(-1), dtype=torch.float32, device="cuda") for u in up)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    r.backward(p, grads, dL=dl)
    got = {k: v.cpu().numpy() for k, v in grads.items()}
    up32 = [t.cpu().numpy().astype(np.float64).reshape(u.shape) for t, u in zip(dl, up)]
    ref = oracle.render_backward(g, cam, *up32, cfg=ocfg)
    check_grads(got, ref, BASE + ("sh", "sem_sh"))
    assert not got["quat"].any() and not got["log_scale"][:, 1:].any()
    assert not r.bwd_ws.any()
