"""CPU checks of the C ABI: the library loads, exports every entry point include/sg.h
declares, the ctypes layouts match, and host-side argument validation rejects bad input
before any launch (none of these calls touches a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2412_01217_gb300 import _lib
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"{n} has no ctypes signature"


def test_struct_sizes_match_header_layout():
    from paper_2412_01217_gb300 import _lib
    assert C.sizeof(_lib.SgCamera) == 72
    assert C.sizeof(_lib.SgView) == 96
    assert C.sizeof(_lib.SgGaussians) == 80
    assert C.sizeof(_lib.SgConfig) == 76
    assert C.sizeof(_lib.SgLossConfig) == 48


def test_defaults_and_version():
    from paper_2412_01217_gb300 import _lib
    lib = _lib.load()
    c = _lib.SgConfig()
    lib.sg_default_config(C.byref(c))
    assert c.alpha_max == pytest.approx(0.99) and c.alpha_min == pytest.approx(1 / 255)
    assert c.T_min == pytest.approx(1e-4) and c.tile_w == 16 and c.tile_h == 16
    lc = _lib.SgLossConfig()
    lib.sg_default_loss_config(C.byref(lc))
    assert lc.lambda_r == pytest.approx(0.2) and lc.lambda_s == pytest.approx(0.2)
    assert c.check_numeric == 0 and lc.check_numeric == 0  # numeric checks are off by default
    assert c.half_tile_fwd == 0  # the forward shares staged batches by default
    assert b"sm_103a" in lib.sg_version()


def test_make_views_pyramid_geometry():
    import numpy as np
    from paper_2412_01217_gb300 import make_views
    import synthetic
    cam = synthetic.make_camera(1200, 680, 600.0, 600.0, 599.5, 339.5)
    views, P, T = make_views([cam, cam], 3)
    assert [(v.W, v.H) for v in views][:3] == [(1200, 680), (600, 340), (300, 170)]
    assert views[1].cx == 299.5 and views[2].cx == 149.5 and views[2].fx == 150.0
    assert P == 2 * (1200 * 680 + 600 * 340 + 300 * 170)
    assert T == 2 * (75 * 43 + 38 * 22 + 19 * 11)
    assert [v.pixel_offset for v in views] == list(np.cumsum([0] + [v.W * v.H for v in views])[:-1])


def test_host_validation_rejects_bad_arguments():
    from paper_2412_01217_gb300 import _lib
    from paper_2412_01217_gb300.splat import make_views
    lib = _lib.load()
    import synthetic
    cam = synthetic.make_camera(4, 4, 4.0, 4.0, 2.0, 2.0)
    with pytest.raises(_lib.SgError) as e:
        make_views([cam], 4)          # level 3 would be 0 x 0
    assert e.value.code == 1
    cfg = _lib.SgConfig()
    lib.sg_default_config(C.byref(cfg))
    cfg.tile_w = 12
    g = _lib.SgGaussians()
    g.N, g.C = 10, 7                  # C not supported
    proj = _lib.SgProjected()
    assert lib.sg_project_gaussians(C.byref(g), None, 1, C.byref(cfg), C.byref(proj), None, None) == 1
    assert b"C=7" in lib.sg_last_error()
    g.C = 8
    assert lib.sg_project_gaussians(C.byref(g), None, 1, C.byref(cfg), C.byref(proj), None, None) == 1
    assert b"NULL" in lib.sg_last_error()
    g.sh_degree = 4                   # spherical-harmonic colour goes to degree 3
    assert lib.sg_project_gaussians(C.byref(g), None, 1, C.byref(cfg), C.byref(proj), None, None) == 1
    assert b"sh_degree = 4" in lib.sg_last_error()
    assert lib.sg_adam_step(None, None, None, None, 5, 1e-3, 0.9, 0.999, 1e-8, 0, None) == 1
    assert lib.sg_read_status(None, None, None) == 1
    assert lib.sg_adam_step(None, None, None, None, 0, 1e-3, 0.9, 0.999, 1e-8, 1, None) == 0


def test_half_tile_forward_flag_is_checked_on_the_host():
    """sg_config.half_tile_fwd takes 0 or 1; anything else is refused before any launch (the
    buffer pointers below are never dereferenced)."""
    from paper_2412_01217_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.SgConfig()
    lib.sg_default_config(C.byref(cfg))
    cfg.half_tile_fwd = 2
    proj = _lib.SgProjected(16, 16, 16, 0, 0)
    lists = _lib.SgTileLists()
    assert lib.sg_build_tile_lists(C.byref(proj), 10, 1, None, 1, C.byref(cfg), C.byref(lists), None, 0, None,
                                   None) == 1
    assert b"half_tile_fwd" in lib.sg_last_error()


def test_timeout_probe_validates_on_the_host():
    """The failure-detection self-test refuses bad arguments before any launch."""
    from paper_2412_01217_gb300 import _lib
    lib = _lib.load()
    assert lib.sg_gemm_bf16_timeout_probe(None, 64, None, 64, 128, 32, 64, None, 32, 1000, None, None) == 1
    # a poll bound of 0 would disable the probe's wait: rejected
    import ctypes as C
    buf = (C.c_uint16 * 64)()
    fbuf = (C.c_float * 64)()
    assert lib.sg_gemm_bf16_timeout_probe(buf, 64, buf, 64, 128, 32, 64, fbuf, 32, 0, None, None) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the compiled library the package raises; there is no CPU or eager fallback."""
    from paper_2412_01217_gb300 import _build, _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libsg.so"))
    with pytest.raises(RuntimeError, match="libsg.so not found"):
        _lib.load(build_if_missing=False)


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the product package imports it."""
    pkg = os.path.join(ROOT, "paper_2412_01217_gb300")
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b|from\s+\.\.\s*oracle|.*importlib.*oracle)", re.M)
    checked = 0
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pat.search(text), f
                assert "sg_oracle" not in text, f
                checked += 1
    assert checked > 10


def test_numeric_checks_need_a_status_word():
    """check_numeric on without a status word is refused on the host (nothing launched)."""
    import numpy as np
    from paper_2412_01217_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.SgConfig()
    lib.sg_default_config(C.byref(cfg))
    cfg.check_numeric = 1
    buf = (C.c_float * 64)()
    g = _lib.SgGaussians(C.addressof(buf), C.addressof(buf), C.addressof(buf), C.addressof(buf), C.addressof(buf),
                         C.addressof(buf), 1, 8)
    views = (C.c_uint8 * 96)()
    proj = _lib.SgProjected(C.addressof(buf), C.addressof(buf), C.addressof(buf), None, None)
    assert lib.sg_project_gaussians(C.byref(g), views, 1, C.byref(cfg), C.byref(proj), None, None) == 1
    assert b"status" in lib.sg_last_error()
    cfg.check_numeric = 2
    assert lib.sg_project_gaussians(C.byref(g), views, 1, C.byref(cfg), C.byref(proj), None, None) == 1


def test_loss_workspace_must_be_16_byte_aligned():
    """The loss reads its per-unit partial sums with 16-byte loads: a workspace that is not
    16-byte aligned is refused on the host, before any launch."""
    from paper_2412_01217_gb300 import _lib
    from paper_2412_01217_gb300.splat import make_views
    import synthetic
    lib = _lib.load()
    views, P, nt = make_views([synthetic.make_camera(64, 48, 60.0, 60.0, 31.5, 23.5)], 1)
    buf = (C.c_float * 64)()
    a = C.addressof(buf)
    imgs = _lib.SgImages(a, a, a)
    dl = _lib.SgImages(a, a, a)
    gt = _lib.SgTargets(a, a, a, a)
    lc = _lib.SgLossConfig()
    lib.sg_default_loss_config(C.byref(lc))
    lc.n_classes = 8
    ws = (C.c_uint8 * 256)()
    base = (C.addressof(ws) + 15) // 16 * 16
    assert lib.sg_pyramid_loss(C.byref(imgs), C.byref(gt), views, views, 1, 8, C.byref(lc), a, C.byref(dl),
                               base + 4, 128, None, None) == 1
    assert b"16-byte" in lib.sg_last_error()
