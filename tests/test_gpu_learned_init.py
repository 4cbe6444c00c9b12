"""What the learned initializer gains over the plain (heuristic) one, on a reduced version of
the time-to-PSNR experiment: 320x180 x 3 levels, 40k Gaussians, 6 keyframes.  The MLP is
trained on pairs that the plain mapper produces on two seeded rooms, then both mappers run the
same schedule on a held-out room; the learned form must reach the plain form's final
held-out-view PSNR in fewer GPU-seconds (insertion, patch extraction and MLP inference
included; training excluded, as it is done once offline)."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_initializer_reaches_plain_final_psnr_in_fewer_gpu_seconds():
    from paper_2412_01217_gb300.experiments import run
    res = run(quick=True, train_rooms=2, iters_per_kf=90, keyframes=6, epochs=4, workers=1)
    assert res["train_pairs"] >= 20_000
    assert res["train_loss_per_epoch"][-1] < res["train_loss_per_epoch"][0]
    assert res["learned_gpu_seconds_to_plain_final_psnr"] is not None, res["learned_curve"]
    assert res["speedup_to_plain_final_psnr"] > 1.05, (res["speedup_to_plain_final_psnr"],
                                                       res["plain_curve"], res["learned_curve"])
