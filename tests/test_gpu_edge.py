"""Edge cases of the GPU path against the FP64 oracle (same tolerances as the other parity
tests): ragged image sizes in every tile shape, the semantic widths not covered elsewhere,
the maximum number of view-levels (more than one 32-view visibility block in the projection
adjoint), exact depth ties, a Gaussian covering the whole image next to sub-pixel ones,
Gaussians on both sides of the near plane, and empty or fully culled inputs."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import AMBIGUOUS_GRAD, FWD_ABS, FWD_REL, MAX_MASKED, check_close, check_grads, ref_render, unambiguous
from test_gpu_parity import (KEYS, f32_camera, lists_match_definition, lists_match_kernel_rule, make, oracle_cams,
                             view_images)

pytestmark = pytest.mark.gpu


def parity_all_views(g, cams, levels, seed=0, **cfg):
    """Tile lists against the FP64 definition (and bit-exact against the kernels' own rule),
    every pixel of every view-level within the forward tolerance, and all parameter gradients
    for a random upstream gradient on every view-level."""
    C = g["sem"].shape[1]
    r, p = make(g, cams, levels=levels, **cfg)
    r.forward(p)
    ocams = oracle_cams(cams, levels)
    lists_match_definition(r, g, ocams)
    lists_match_kernel_rule(r)
    rng = np.random.default_rng(seed)
    dl = [torch.zeros(3 * r.P, device="cuda"), torch.zeros(r.P, device="cuda"), torch.zeros(C * r.P, device="cuda")]
    for v, oc in enumerate(ocams):
        got = view_images(r, v, C)
        ref = ref_render(g, oc)
        # at most 0.1 % of the pixels (one pixel of the smallest levels) may be ambiguous
        limit = max(MAX_MASKED, 1.0 / ref["flags"].size)
        ok = unambiguous(ref["flags"], limit=limit)
        for k in ("rgb", "depth", "sem", "T"):
            check_close(f"v{v} {k}", got[k], ref[k], FWD_REL, FWD_ABS, mask=ok)
        assert np.array_equal(got["n_contrib"][ok], ref["n_contrib"][ok])
        keep = unambiguous(ref["flags"], AMBIGUOUS_GRAD, limit=limit).astype(np.float64)
        H, W = oc["H"], oc["W"]
        r.view_slice(dl[0], v, 3).copy_(torch.tensor(rng.normal(size=(3, H, W)) * keep, dtype=torch.float32))
        r.view_slice(dl[1], v, 1).copy_(torch.tensor(rng.normal(size=(1, H, W)) * keep, dtype=torch.float32))
        r.view_slice(dl[2], v, C).copy_(torch.tensor(rng.normal(size=(C, H, W)) * keep, dtype=torch.float32))
    grads = {k: torch.zeros_like(t) for k, t in p.items()}
    r.backward(p, grads, dL=tuple(dl))
    got = {k: t.cpu().numpy() for k, t in grads.items()}
    ref = {k: 0.0 for k in KEYS}
    for v, oc in enumerate(ocams):
        a = r.view_slice(dl[0], v, 3).cpu().numpy().astype(np.float64)
        b = r.view_slice(dl[1], v, 1)[0].cpu().numpy().astype(np.float64)
        c = r.view_slice(dl[2], v, C).cpu().numpy().astype(np.float64)
        rv = oracle.render_backward(g, oc, a, b, c)
        for k in KEYS:
            ref[k] = ref[k] + rv[k]
    check_grads(got, ref, KEYS)
    assert not r.bwd_ws.any() and not r.work_counter.any()
    return r, got


@pytest.mark.parametrize("tile, batch, batch_bwd, ppt, ppt_bwd, half", [((16, 16), 128, 0, 1, 2, False),
                                                                        ((8, 8), 64, 16, 1, 1, False),
                                                                        ((8, 8), 64, 16, 1, 1, True),
                                                                        ((32, 8), 256, 32, 2, 1, False),
                                                                        ((16, 8), 32, 0, 2, 2, False)])
def test_ragged_image_sizes_every_tile_shape(tile, batch, batch_bwd, ppt, ppt_bwd, half):
    """157 x 91 with 3 levels (157x91, 78x45, 39x22): no dimension is a multiple of any tile
    side, so every view-level ends in partial tiles (with half masks: tiles whose bottom half
    lies below the image, too)."""
    g = synthetic.cloud_scene(2500, 8, seed=21)
    cam = f32_camera(synthetic.make_camera(157, 91, 140.0, 140.0, 77.7, 44.6))
    parity_all_views(g, [cam], 3, tile_w=tile[0], tile_h=tile[1], batch=batch, batch_bwd=batch_bwd,
                     pixels_per_thread=ppt, pixels_per_thread_bwd=ppt_bwd, half_masks=half, half_tile_fwd=half)


@pytest.mark.parametrize("C, half", [(4, False), (32, False), (4, True), (32, True)])
def test_semantic_widths_4_and_32(C, half):
    g = synthetic.cloud_scene(2000, C, seed=22)
    cam = f32_camera(synthetic.cloud_camera())
    kw = dict(tile_w=8, tile_h=8, pixels_per_thread_bwd=1, half_masks=True, half_tile_fwd=True) if half else {}
    parity_all_views(g, [cam], 2, **kw)


def test_maximum_view_levels():
    """16 keyframes x 4 levels = 64 view-levels (the maximum), so the projection adjoint runs
    two 32-view visibility blocks per Gaussian and one launch covers 64 pyramids' tiles."""
    room = synthetic.Room(n_classes=32, seed=3)
    intr = dict(W=64, H=48, fx=40.0, fy=40.0, cx=31.5, cy=23.5)
    cams = [f32_camera(c) for c in room.trajectory(16, intr, seed=9)]
    g = room.sample_gaussians(6000, 8, seed=5, sem_mode="random")
    r, got = parity_all_views(g, cams, 4)
    assert r.V == 64
    # many Gaussians are visible in both 32-view blocks: their gradients sum across them
    rect = r.rect.view(r.V, r.N, 2).cpu().numpy()
    vis = rect[:, :, 0] != rect[:, :, 1]
    assert (vis[:32].any(0) & vis[32:].any(0)).sum() > 100


def test_exact_depth_ties_order_by_index():
    """Gaussians at exactly the same camera depth overlap in every tile: the lists order them
    by Gaussian index, and compositing follows that order on both sides."""
    rng = np.random.default_rng(23)
    n = 400
    g = synthetic.cloud_scene(n, 8, seed=23)
    g["mean"][:, 2] = np.float32(2.0)                       # identity camera: depth key = z
    g["mean"][:, :2] = rng.uniform(-0.3, 0.3, (n, 2)).astype(np.float32)
    # anisotropic (an isotropic Gaussian's quaternion gradient is identically zero)
    g["log_scale"][:] = (np.log(0.05) + rng.uniform(-0.4, 0.4, (n, 3))).astype(np.float32)
    cam = f32_camera(synthetic.cloud_camera())
    r, _ = parity_all_views(g, [cam], 1)
    assert r.instance_count() > 4 * n


def test_whole_image_gaussian_and_subpixel_gaussians():
    g = synthetic.cloud_scene(1500, 8, seed=24)
    # one Gaussian far larger than the image, in front of everything but half transparent
    g["mean"][0] = [0.0, 0.0, 1.05]
    g["log_scale"][0] = np.log([3.0, 2.5, 0.5])
    g["quat"][0] = [1.0, 0.0, 0.0, 0.0]
    g["opacity_logit"][0] = -0.5
    # sub-pixel Gaussians (footprint far below one pixel: only the 0.3 px^2 dilation remains)
    g["log_scale"][1:300] = np.log(1e-4)
    g["opacity_logit"][1:300] = 3.0
    cam = f32_camera(synthetic.cloud_camera())
    r, _ = parity_all_views(g, [cam], 2)
    rect = r.rect.view(-1, 2).cpu().numpy().view(np.uint32)
    assert (rect[0, 1] & 0xFFFF) - (rect[0, 0] & 0xFFFF) == r.views_host[0].tiles_x   # spans every tile column


def test_near_plane_culling():
    """Means just in front of and just behind the near plane (0.2 m): the ones behind are
    culled on both sides and get zero gradient."""
    g = synthetic.cloud_scene(1500, 8, seed=25)
    g["mean"][:200, 2] = np.float32(0.19)
    g["mean"][200:400, 2] = np.float32(0.21)
    g["mean"][:400, :2] *= 0.1
    # anisotropic (an isotropic Gaussian's quaternion gradient is zero by cancellation only)
    g["log_scale"][:400] = np.log(np.float32(0.01)) + np.random.default_rng(25).uniform(-0.4, 0.4, (400, 3))
    cam = f32_camera(synthetic.cloud_camera())
    r, got = parity_all_views(g, [cam], 1)
    rect = r.rect.view(-1, 2).cpu().numpy()
    assert (rect[:200, 0] == rect[:200, 1]).all()            # culled
    assert (rect[200:400, 0] != rect[200:400, 1]).any()
    for k in KEYS:
        assert not got[k][:200].any(), k


@pytest.mark.parametrize("case", ["empty", "all_culled"])
def test_empty_and_fully_culled_inputs(case):
    """No Gaussian at all, or every Gaussian behind the camera: empty tile lists, every pixel
    shows the background with T = 1, the loss is finite and the backward adds nothing."""
    from paper_2412_01217_gb300 import build_pyramid
    n = 0 if case == "empty" else 500
    g = synthetic.cloud_scene(max(n, 1), 8, seed=26)
    g = {k: v[:n].copy() for k, v in g.items()}
    if n:
        g["mean"][:, 2] = -1.0
    cam = f32_camera(synthetic.cloud_camera())
    r, p = make(g, [cam], levels=2, bg=(0.25, 0.5, 0.75))
    r.forward(p)
    torch.cuda.synchronize()
    assert r.instance_count() == 0
    for v in range(r.V):
        im = view_images(r, v, 8)
        assert np.all(im["T"] == 1.0) and np.all(im["n_contrib"] == 0)
        assert np.allclose(im["rgb"], np.array([0.25, 0.5, 0.75], np.float32)[:, None, None])
        assert not im["depth"].any() and not im["sem"].any()
    tgt = synthetic.random_targets(cam["H"], cam["W"], 8, seed=3)
    gt = build_pyramid(r, [tgt["rgb"]], [tgt["depth"]], [tgt["label"]])
    r.loss(gt)
    assert np.isfinite(r.terms.cpu().numpy()).all()
    grads = {k: torch.zeros_like(t) for k, t in p.items()}
    r.backward(p, grads)
    torch.cuda.synchronize()
    for k in KEYS:
        assert not grads[k].any(), k
