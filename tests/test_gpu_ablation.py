"""The ablation analogues on a reduced setup (320x180 x 3 levels, 40k Gaussians): the
experiments run end to end through the mapper, and the loss-term ablation shows what each
term of Eq. 13 contributes: without the semantic term the decoded labels are much worse
(mIoU), without the depth term the rendered depth is worse (L1)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_loss_term_ablation_directions():
    from paper_2412_01217_gb300.ablation import loss_ablation
    res = loss_ablation(quick=True, keyframes=4, iters_per_kf=60)
    runs = res["runs"]
    for r in runs.values():
        assert all(math.isfinite(v) for v in r.values()), runs
    assert runs["no_semantic"]["miou"] < runs["full"]["miou"] - 0.1, runs
    assert runs["no_depth"]["depth_l1"] > runs["full"]["depth_l1"], runs


def test_pyramid_ablation_runs():
    from paper_2412_01217_gb300.ablation import pyramid_ablation
    res = pyramid_ablation(quick=True, keyframes=3, iters_per_kf=30)
    assert math.isfinite(res["single_level_final_psnr"]) and math.isfinite(res["pyramid_final_psnr"])
    assert res["pyramid_final_psnr"] > 10.0 and res["single_level_final_psnr"] > 10.0
