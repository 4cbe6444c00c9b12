"""Host logic of the launch-shape autotuner (no GPU): the rasterizer and the CUDA calls are
replaced by fakes, and the timer returns a cost chosen per (configuration, operation), so the
test fixes which candidate is fastest and checks that the tuner returns exactly it, with the
list-build time counted and the half-mask options (adjoint, and the forward one warp per half
tile) compared against the shared-batch ones."""
import torch

from paper_2412_01217_gb300 import autotune as at
from paper_2412_01217_gb300.splat import LossConfig, RenderConfig


class FakeRasterizer:
    """Records which operation the tuner last ran and with which launch configuration."""
    last = None

    def __init__(self, N, C, cams, levels, cfg, loss_cfg=None):
        self.cfg = cfg
        self._ccfg = None

    def _mark(self, op):
        FakeRasterizer.last = (op, self.cfg)

    def project(self, params):
        self._mark("project")

    def build_lists(self):
        self._mark("lists")

    def rasterize(self, params):
        self._mark("fwd")

    def loss(self, gt, decoder=None, decoder_grad=None):
        self._mark("loss")

    def backward(self, params, grads):
        self._mark("bwd")

    def check_status(self):
        pass


def run_tuner(monkeypatch, cost):
    """cost(op, cfg) -> ms for op in lists / fwd / bwd."""
    monkeypatch.setattr(at, "PyramidRasterizer", FakeRasterizer)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "fake")

    def fake_time(fn, reps):
        fn()
        op, cfg = FakeRasterizer.last
        return cost(op, cfg)

    monkeypatch.setattr(at, "_time", fake_time)
    params = {"mean": torch.zeros(10, 3), "sem": torch.zeros(10, 16), "rgb": torch.zeros(10, 3)}
    cam = dict(W=64, H=48)
    return at.autotune(params, [cam], 3, None, LossConfig(), base=RenderConfig(), use_cache=False)


def test_the_fastest_shared_batch_configuration_wins(monkeypatch):
    # 16x16 tiles are cheapest everywhere; half masks cost more; batch 128 and 2 pixels per
    # thread are the best forward, batch 64 and 1 pixel per thread the best adjoint
    def cost(op, c):
        tile = 1.0 if (c.tile_w, c.tile_h) == (16, 16) else 2.0
        if op == "lists":
            return tile * (3.0 if c.half_masks else 1.0)
        if op == "fwd":
            return tile * (1.0 + 0.01 * abs(c.batch - 128) + (0.0 if c.pixels_per_thread == 2 else 0.5)
                           + (0.7 if c.half_tile_fwd else 0.0))
        b = c.batch_bwd or c.batch
        return tile * (2.0 + 0.01 * abs(b - 64) + (0.0 if c.pixels_per_thread_bwd == 1 else 0.3)
                       + (0.1 if c.half_masks else 0.0))

    cfg, table = run_tuner(monkeypatch, cost)
    assert (cfg.tile_w, cfg.tile_h) == (16, 16)
    assert cfg.batch == 128 and cfg.pixels_per_thread == 2
    assert cfg.batch_bwd == 64 and cfg.pixels_per_thread_bwd == 1
    assert not cfg.half_masks and not cfg.half_tile_fwd
    # the list build of every tile shape was timed and counted
    assert sum(1 for t in table if t["kernel"] == "lists") == len(at.TILES)


def test_half_masks_win_when_the_adjoint_gain_outweighs_the_list_cost(monkeypatch):
    # 8x8 tiles; the half-tile adjoint saves 1 ms for 0.1 ms more list build; the forward is
    # faster with shared batches
    def cost(op, c):
        tile = 1.0 if (c.tile_w, c.tile_h) == (8, 8) else 3.0
        if op == "lists":
            return tile * (1.1 if c.half_masks else 1.0)
        if op == "fwd":
            return tile * (1.0 + (0.2 if c.half_tile_fwd else 0.0) + (0.0 if c.pixels_per_thread == 1 else 0.4))
        return tile * (3.0 - (1.0 if c.half_masks and c.pixels_per_thread_bwd == 1 else 0.0))

    cfg, table = run_tuner(monkeypatch, cost)
    assert (cfg.tile_w, cfg.tile_h) == (8, 8)
    assert cfg.half_masks and not cfg.half_tile_fwd and cfg.pixels_per_thread_bwd == 1
    kinds = {t["kernel"] for t in table}
    assert {"lists_half", "fwd_half", "fwd_half_tile", "bwd_half"} <= kinds


def test_the_half_tile_forward_is_chosen_when_faster(monkeypatch):
    # as above, but the forward one warp per half tile is faster; it runs one pixel per
    # thread, whatever the shared-batch forward preferred
    def cost(op, c):
        tile = 1.0 if (c.tile_w, c.tile_h) == (8, 8) else 3.0
        if op == "lists":
            return tile * (1.1 if c.half_masks else 1.0)
        if op == "fwd":
            if c.half_tile_fwd:
                return tile * 0.5
            return tile * (1.0 + (0.0 if c.pixels_per_thread == 2 else 0.1))
        return tile * (3.0 - (1.0 if c.half_masks and c.pixels_per_thread_bwd == 1 else 0.0))

    cfg, _ = run_tuner(monkeypatch, cost)
    assert (cfg.tile_w, cfg.tile_h) == (8, 8)
    assert cfg.half_masks and cfg.half_tile_fwd
    assert cfg.pixels_per_thread == 1 and cfg.pixels_per_thread_bwd == 1
