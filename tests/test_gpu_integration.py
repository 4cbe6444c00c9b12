"""GPU integration: the autograd Function, CUDA-graph replay vs eager execution, and the
full-size Replica-like pyramid (1200x680, 3 levels, 300k Gaussians) against the oracle on
sampled pixels, in the launch configuration the benchmark times."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import AMBIGUOUS_GRAD, FWD_ABS, FWD_REL, MAX_MASKED, check_close, check_grads, ref_render, unambiguous
from test_gpu_parity import KEYS, f32_camera, make

pytestmark = pytest.mark.gpu


def test_autograd_function_matches_direct_backward():
    from paper_2412_01217_gb300 import pyramid_splat
    g = synthetic.cloud_scene(1500, 8, seed=3)
    cam = f32_camera(synthetic.cloud_camera())
    r, p = make(g, [cam], levels=2)
    leaves = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    rgb, depth, sem = pyramid_splat(r, leaves)
    w = [torch.randn_like(t) for t in (rgb, depth, sem)]
    loss = (rgb * w[0]).sum() + (depth * w[1]).sum() + (sem * w[2]).sum()
    loss.backward()
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    r.forward(p)
    r.backward(p, grads, dL=tuple(x.contiguous() for x in w))
    torch.cuda.synchronize()
    for k in KEYS:
        a, b = leaves[k].grad.cpu().numpy(), grads[k].cpu().numpy()
        # same kernels; only the order of the float atomic additions differs
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5 * (np.abs(b).max() + 1e-12)), k


def _room_problem(W=320, H=180, n=30000, ncam=2, levels=3, C=16, K=32):
    room = synthetic.Room(n_classes=K, seed=3)
    intr = dict(W=W, H=H, fx=W / 2.0, fy=W / 2.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5)
    cams = [f32_camera(c) for c in room.trajectory(ncam, intr, seed=7)]
    g = room.sample_gaussians(n, C, seed=4, sem_mode="random")
    frames = [room.raycast(c) for c in cams]
    return room, g, cams, frames


def test_cuda_graph_replay_equals_eager():
    from paper_2412_01217_gb300 import MappingStep, build_pyramid
    room, g, cams, frames = _room_problem()
    dec = torch.randn(32, 16, device="cuda") * 0.3
    results = []
    for use_graph in (False, True):
        r, p = make(g, cams, levels=3)
        r.loss_cfg.n_classes = 32
        gt = build_pyramid(r, [f["rgb"] for f in frames], [f["depth"] for f in frames],
                           [f["label"] for f in frames])
        ms = MappingStep(r, p, gt, decoder=dec.clone())
        ms.step()   # step 1 eager in both runs
        if use_graph:
            ms.capture(warmup=0)
            for _ in range(3):
                ms.replay()
        else:
            for _ in range(3):
                ms._step_kernels(1)   # the graph freezes Adam's step count at capture
        torch.cuda.synchronize()
        results.append({k: v.detach().cpu().numpy().copy() for k, v in p.items()})
        results[-1]["terms"] = r.terms.cpu().numpy().copy()
    # The gradients are sums of float atomics whose order is not fixed, so both runs agree
    # only to rounding; Adam's first steps (epsilon 1e-15) turn a gradient that is pure
    # rounding noise into a step of +-lr.  Hence: loss terms to rounding, nearly every
    # parameter to rounding, and none further apart than 4 Adam steps can move it (an Adam
    # step with beta1 = 0.9, beta2 = 0.999 is below 3.2 lr).
    assert np.allclose(results[0]["terms"], results[1]["terms"], rtol=1e-4, atol=1e-6)
    from paper_2412_01217_gb300.splat import DEFAULT_LR
    for k in KEYS:
        a, b = results[0][k], results[1][k]
        close = np.isclose(a, b, rtol=1e-5, atol=1e-6)
        assert close.mean() > 0.995, (k, close.mean())
        assert np.abs(a - b).max() <= 2 * 4 * 3.2 * DEFAULT_LR[k], (k, np.abs(a - b).max())


def test_mapping_loss_decreases():
    from paper_2412_01217_gb300 import MappingStep, build_pyramid
    room, g, cams, frames = _room_problem(n=20000)
    r, p = make(g, cams, levels=3)
    r.loss_cfg.n_classes = 32
    gt = build_pyramid(r, [f["rgb"] for f in frames], [f["depth"] for f in frames],
                       [f["label"] for f in frames])
    dec = torch.randn(32, 16, device="cuda") * 0.3
    ms = MappingStep(r, p, gt, decoder=dec)
    ms.step()
    first = ms.total_loss()
    for _ in range(60):
        ms.step()
    last = ms.total_loss()
    assert np.isfinite(last) and last < 0.8 * first, (first, last)


@pytest.fixture(scope="module")
def replica_like():
    """The benchmark's workload: one 1200x680 keyframe, 3 pyramid levels, 300k Gaussians
    on the room's surfaces, C = 16 semantic features."""
    room = synthetic.Room(n_classes=32, seed=3)
    cam = f32_camera(room.trajectory(4, synthetic.REPLICA_LIKE, seed=7)[1])
    g = room.sample_gaussians(300_000, 16, seed=4, sem_mode="random")
    return room, g, cam


# the launch configuration bench.py times on this workload (autotuned: 8x8 tiles, forward batch
# 64, backward batch 16, one pixel per thread in both kernels), and the library default
BENCH_CFG = dict(tile_w=8, tile_h=8, batch=64, batch_bwd=16, pixels_per_thread=1, pixels_per_thread_bwd=1)
LAUNCH_CFGS = [pytest.param(BENCH_CFG, id="bench-8x8"),
               pytest.param(dict(BENCH_CFG, half_masks=True, half_tile_fwd=True), id="8x8-half"),
               pytest.param(dict(tile_w=16, tile_h=16, batch=128), id="16x16")]


@pytest.mark.parametrize("cfg", LAUNCH_CFGS)
def test_full_size_forward_sampled_pixels(replica_like, cfg):
    room, g, cam = replica_like
    r, p = make(g, [cam], levels=3, **cfg)
    r.forward(p)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    rng = np.random.default_rng(0)
    for v, oc in enumerate(oracle.level_cameras(cam, 3)):
        pix = np.stack([rng.integers(0, oc["W"], 600), rng.integers(0, oc["H"], 600)], 1)
        ref = ref_render(g, oc, pixels=pix)
        got = {k: r.view_slice(getattr(r, a), v, n).cpu().numpy()[:, pix[:, 1], pix[:, 0]]
               for k, a, n in (("rgb", "img_rgb", 3), ("sem", "img_sem", 16))}
        got["depth"] = r.view_slice(r.img_depth, v, 1).cpu().numpy()[0, pix[:, 1], pix[:, 0]]
        got["T"] = r.view_slice(r.T_final, v, 1).cpu().numpy()[0, pix[:, 1], pix[:, 0]]
        ok = unambiguous(ref["flags"], limit=max(MAX_MASKED, 1.0 / len(pix)))
        assert (ref["n_contrib"] > 0).mean() > 0.5
        for k in ("rgb", "depth", "sem", "T"):
            check_close(f"level {v} {k}", got[k], ref[k], FWD_REL, FWD_ABS, mask=ok)


@pytest.mark.parametrize("cfg", LAUNCH_CFGS)
def test_full_size_backward_sparse_upstream(replica_like, cfg):
    """Upstream gradient non-zero only on sampled pixels, so the oracle computes exactly
    the same parameter gradients from those pixels alone."""
    room, g, cam = replica_like
    r, p = make(g, [cam], levels=3, **cfg)
    r.forward(p)
    rng = np.random.default_rng(1)
    ocams = oracle.level_cameras(cam, 3)
    dl = [torch.zeros(3 * r.P, device="cuda"), torch.zeros(r.P, device="cuda"), torch.zeros(16 * r.P, device="cuda")]
    ref = {k: 0.0 for k in KEYS}
    for v, oc in enumerate(ocams):
        pix = np.unique(np.stack([rng.integers(0, oc["W"], 400), rng.integers(0, oc["H"], 400)], 1), axis=0)
        fl = ref_render(g, oc, pixels=pix)["flags"]
        pix = pix[unambiguous(fl, AMBIGUOUS_GRAD, limit=max(MAX_MASKED, 1.0 / len(pix)))]
        ups = (rng.normal(size=(3, len(pix))).astype(np.float32), rng.normal(size=len(pix)).astype(np.float32),
               rng.normal(size=(16, len(pix))).astype(np.float32))
        for t, u, n in zip(dl, ups, (3, 1, 16)):
            img = r.view_slice(t, v, n)
            img[:, torch.as_tensor(pix[:, 1]), torch.as_tensor(pix[:, 0])] = torch.as_tensor(u.reshape(n, -1)).cuda()
        rv = oracle.render_backward(g, oc, ups[0].astype(np.float64), ups[1].astype(np.float64),
                                    ups[2].astype(np.float64), pixels=pix)
        for k in KEYS:
            ref[k] = ref[k] + rv[k]
    grads = {k: torch.zeros_like(t) for k, t in p.items()}
    r.backward(p, grads, dL=tuple(dl))
    got = {k: t.cpu().numpy() for k, t in grads.items()}
    check_grads(got, ref, KEYS)


def test_autotuner_picks_a_valid_configuration_with_identical_output():
    from paper_2412_01217_gb300 import LossConfig, build_pyramid
    from paper_2412_01217_gb300.autotune import autotune
    room, g, cams, frames = _room_problem(n=20000, ncam=1)
    r, p = make(g, cams, levels=3)
    gt = build_pyramid(r, [f["rgb"] for f in frames], [f["depth"] for f in frames], [f["label"] for f in frames])
    dec = torch.randn(32, 16, device="cuda") * 0.3
    cfg, table = autotune(p, cams, 3, gt, LossConfig(n_classes=32), decoder=dec, reps=1, use_cache=False)
    from paper_2412_01217_gb300.autotune import BATCHES
    assert (cfg.tile_w, cfg.tile_h) in ((16, 16), (8, 8), (32, 8), (16, 8))
    assert cfg.batch in BATCHES and cfg.batch_bwd in BATCHES
    assert len(table) >= 20 and all(t["ms"] > 0 for t in table)
    r.forward(p)
    base = r.img_rgb.clone()
    r2, _ = make(g, cams, levels=3, **{k: getattr(cfg, k) for k in ("tile_w", "tile_h", "batch", "pixels_per_thread",
                                                                        "pixels_per_thread_bwd", "batch_bwd")})
    r2.forward(p)
    torch.cuda.synchronize()
    assert torch.equal(r2.img_rgb, base)
