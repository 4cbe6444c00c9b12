"""Device-side detection of non-finite values (the status-word contract of include/sg.h):
with checks on, a NaN made on the host in one Gaussian's mean, in one rendered pixel or in one
gradient sets SG_STATUS_NUMERIC, and sg_read_status turns it into SG_ERR_NUMERIC; every
kernel exits normally and the context stays usable.  With checks off nothing changes."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic
from test_gpu_parity import f32_camera, make

pytestmark = pytest.mark.gpu


def _read(status):
    from paper_2412_01217_gb300._lib import load
    lib = load()
    bits = C.c_uint32(0)
    code = lib.sg_read_status(C.c_void_p(status.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                              C.byref(bits))
    return code, int(bits.value), lib.sg_last_error().decode()


def test_nan_mean_sets_the_numeric_bit_only_with_checks_on():
    from paper_2412_01217_gb300._lib import STATUS_NUMERIC
    g = synthetic.cloud_scene(2000, 8, seed=1)
    cam = f32_camera(synthetic.cloud_camera())
    base, p = make(g, [cam], check_numeric=False)
    base.forward(p)
    ref = base.img_rgb.clone()
    chk, _ = make(g, [cam], check_numeric=True)
    chk.forward(p)
    torch.cuda.synchronize()
    assert _read(chk.status)[:2] == (0, 0)
    assert torch.equal(chk.img_rgb, ref)            # the check changes no result
    g_bad = {k: v.copy() for k, v in g.items()}
    g_bad["mean"][123, 1] = np.nan
    from paper_2412_01217_gb300 import to_device_params
    pb = to_device_params(g_bad)
    off, _ = make(g, [cam], check_numeric=False)
    off.forward(pb)
    torch.cuda.synchronize()
    assert _read(off.status)[:2] == (0, 0)          # checks off: not reported
    chk.status.zero_()
    chk.forward(pb)
    code, bits, msg = _read(chk.status)
    assert bits & STATUS_NUMERIC and code == 4 and "non-finite" in msg
    from paper_2412_01217_gb300 import SgError
    with pytest.raises(SgError) as e:
        chk.check_status()
    assert e.value.code == 4
    # the context is still usable: a clean forward afterwards is exactly the reference
    chk.status.zero_()
    chk.forward(p)
    torch.cuda.synchronize()
    assert _read(chk.status)[:2] == (0, 0) and torch.equal(chk.img_rgb, ref)


def test_nan_in_a_rendered_pixel_sets_the_bit_through_the_loss():
    from paper_2412_01217_gb300 import LossConfig, build_pyramid
    from paper_2412_01217_gb300._lib import STATUS_NUMERIC
    g = synthetic.cloud_scene(2000, 8, seed=1)
    cam = f32_camera(synthetic.cloud_camera())
    tg = synthetic.random_targets(cam["H"], cam["W"], 8, seed=2)
    for check in (False, True):
        r, p = make(g, [cam], levels=2)
        r.forward(p)
        gt = build_pyramid(r, [tg["rgb"]], [tg["depth"]], [tg["label"]])
        r.img_rgb[1234] = float("nan")
        r.loss(gt, loss_cfg=LossConfig(n_classes=8, check_numeric=check))
        code, bits, _ = _read(r.status)
        assert bool(bits & STATUS_NUMERIC) == check and (code == 4) == check
        assert not np.isfinite(r.terms.view(-1, 4)[0, 3].item())


def test_nan_gradient_sets_the_bit_in_adam():
    from paper_2412_01217_gb300._lib import STATUS_NUMERIC, SgAdamGroup, call
    for n, check in ((4000, True), (4001, True), (4000, False)):  # 16-byte and scalar kernels
        t = [torch.randn(n, device="cuda") for _ in range(4)]
        t[3] = t[3].abs()
        t[1][n // 2] = float("inf")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        grp = (SgAdamGroup * 1)(SgAdamGroup(*[x.data_ptr() for x in t], n, 1e-3))
        call("sg_adam_multi", grp, 1, 0.9, 0.999, 1e-8, 1, 0, C.c_void_p(status.data_ptr()) if check else None,
             C.c_void_p(torch.cuda.current_stream().cuda_stream))
        code, bits, _ = _read(status)
        assert bool(bits & STATUS_NUMERIC) == check and (code == 4) == check
