"""The C ABI on a machine without a GPU: the library loads, exports every
function the header declares, and rejects bad arguments on the host before
touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2006_01201_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        names += re.findall(r"^PANO_API\s+[\w\s\*]+?\b(pano_\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(declared_functions())
    assert {"pano_flow_create", "pano_flow_pair", "pano_blend_pair", "pano_flow_destroy"} <= names
    assert names == set(binding.SIGNATURES), "binding and header disagree"


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_default(lib):
    p = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(p))
    assert (p.levels, p.iters, p.radius) == (4, 5, 2)
    assert abs(p.lam - 1e-2) < 1e-9 and p.soft_sharpness == 10.0 and p.flow_mag_coef == 20.0
    assert p.pyr_dtype == binding.PANO_F32


def test_create_rejects_bad_arguments_before_any_device_call(lib):
    out = ctypes.c_void_p(123)
    p = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(p))
    assert lib.pano_flow_create(None, 10, 10, 1, ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG
    assert out.value is None
    assert b"params" in lib.pano_last_error(None)
    assert lib.pano_flow_create(ctypes.byref(p), 10, 10, 1, None) == binding.PANO_ERR_INVALID_ARG
    for field, value in (("levels", 0), ("levels", 13), ("iters", -1), ("iters", 17), ("radius", 0),
                         ("radius", 4), ("lam", -1.0), ("lam", float("nan"))):
        q = binding.PanoParams()
        lib.pano_flow_params_default(ctypes.byref(q))
        setattr(q, field, value)
        assert lib.pano_flow_create(ctypes.byref(q), 10, 10, 1, ctypes.byref(out)) == \
            binding.PANO_ERR_INVALID_ARG, (field, value)
    q = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(q))
    for bad in (binding.PANO_U8, 7):
        q.pyr_dtype = bad
        assert lib.pano_flow_create(ctypes.byref(q), 10, 10, 1, ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_flow_create(ctypes.byref(p), 0, 10, 1, ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_flow_create(ctypes.byref(p), 10, 10, 2, ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG


def test_calls_reject_null_and_bad_images(lib):
    assert lib.pano_flow_destroy(None) == binding.PANO_OK
    img = binding.PanoImage(0x1000, 8, 8, 1, 32, binding.PANO_F32)
    assert lib.pano_flow_pair(None, ctypes.byref(img), ctypes.byref(img), 0x2000, 0x3000, None) == \
        binding.PANO_ERR_INVALID_ARG
    assert lib.pano_blend_pair(None, ctypes.byref(img), ctypes.byref(img), 0x2000, 0x3000, None,
                               ctypes.byref(img), None) == binding.PANO_ERR_INVALID_ARG
    # stage calls validate on the host too
    bad = [
        binding.PanoImage(None, 8, 8, 1, 32, binding.PANO_F32),         # null data
        binding.PanoImage(0x1000, 0, 8, 1, 32, binding.PANO_F32),       # empty
        binding.PanoImage(0x1000, 8, 8, 1, 16, binding.PANO_F32),       # pitch < row
        binding.PanoImage(0x1002, 8, 8, 1, 32, binding.PANO_F32),       # misaligned
        binding.PanoImage(0x1000, 8, 8, 1, 34, binding.PANO_F32),       # pitch not a multiple
        binding.PanoImage(0x1000, 8, 8, 7, 64, binding.PANO_U8),        # channels
        binding.PanoImage(0x1000, 8, 8, 1, 32, 9),                      # dtype
    ]
    expect = [1, 1, 1, 1, 1, 2, 1]
    for im, st in zip(bad, expect):
        assert lib.pano_stage_luma(ctypes.byref(im), 0x2000, 8, None) == st
    half = binding.PanoImage(0x1000, 8, 8, 1, 16, binding.PANO_BF16)
    assert lib.pano_stage_luma(ctypes.byref(half), 0x2000, 8, None) == binding.PANO_ERR_UNSUPPORTED
    assert lib.pano_stage_pyr_down(None, 8, 8, 8, 0x2000, 4, None) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_stage_pyr_down(0x1000, 8, 8, 7, 0x2000, 4, None) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_stage_lk(0x1000, 0x2000, 8, 8, 8, None, 0, 0, 0, 0x3004, 5, 2, 0.01, None) == \
        binding.PANO_ERR_INVALID_ARG   # flow_out not 8-byte aligned
    assert lib.pano_stage_lk(0x1000, 0x2000, 8, 8, 8, None, 0, 0, 0, 0x3000, 5, 9, 0.01, None) == \
        binding.PANO_ERR_INVALID_ARG   # radius
    assert lib.pano_stage_lk(0x1000, 0x2000, 8, 8, 8, 0x3000, 8, 8, 0, 0x3100, 1, 2, 0.01, None) == \
        binding.PANO_ERR_INVALID_ARG   # flow_in overlaps flow_out
    assert b"overlap" in lib.pano_last_error(None)
    for kernel, st in ((3, binding.PANO_ERR_INVALID_ARG), (-1, binding.PANO_ERR_INVALID_ARG)):
        assert lib.pano_stage_lk_kernel(0x1000, 0x2000, 8, 8, 8, None, 0, 0, 0, 0x3000, 5, 2, 0.01, kernel,
                                        None) == st
    assert lib.pano_stage_lk_kernel(0x1000, 0x2000, 8, 8, 8, None, 0, 0, 0, 0x3000, 0, 2, 0.01,
                                    binding.PANO_LK_STREAM, None) == binding.PANO_ERR_UNSUPPORTED


def test_compose_pair_rejects_bad_arguments_before_any_launch():
    lib = binding.load_library()
    par = binding.Params().to_c()
    im = binding.PanoImage(0x10000, 8, 8, 3, 24, binding.PANO_U8)
    out = binding.PanoImage(0x90000, 8, 8, 3, 24, binding.PANO_U8)
    small = binding.PanoImage(0x20000, 8, 7, 3, 24, binding.PANO_U8)
    inv, ok_args = binding.PANO_ERR_INVALID_ARG, dict(label=0x30000, lp=8, blend=0x40000, bp=8,
                                                     lr=0x50000, rl=0x60000, y0=0, x0=2, fh=8, fw=4)

    def call(L=im, R=im, F=out, **kw):
        a = dict(ok_args, **kw)
        return lib.pano_compose_pair(ctypes.byref(par), ctypes.byref(L), ctypes.byref(R), a["label"], a["lp"],
                                     a["blend"], a["bp"], a["lr"], a["rl"], a["y0"], a["x0"], a["fh"], a["fw"],
                                     ctypes.byref(F), None)

    assert call(R=small) == inv                      # canvas sizes differ
    assert call(label=None) == inv
    assert call(lp=7) == inv                         # label pitch < w
    assert call(blend=0x40002) == inv                # misaligned Blend
    assert call(x0=5) == inv                         # crop leaves the canvas (5 + 4 > 8)
    assert call(fh=0) == inv                         # empty crop
    assert call(y0=-1) == inv
    assert call(lr=0x50004) == inv                   # flow not 8-byte aligned
    assert call(F=binding.PanoImage(0x10000, 8, 8, 3, 24, binding.PANO_U8)) == inv   # F is L
    assert b"overlaps" in lib.pano_last_error(None)
    assert lib.pano_compose_pair(None, ctypes.byref(im), ctypes.byref(im), 0x30000, 8, 0x40000, 8, 0x50000,
                                 0x60000, 0, 0, 8, 8, ctypes.byref(out), None) == inv


def test_release_build_has_no_index_checks():
    lib = binding.load_library()
    out = (ctypes.c_uint * 4)(7, 7, 7, 7)
    assert lib.pano_debug_bounds(out) == binding.PANO_ERR_UNSUPPORTED
    assert tuple(out) == (0, 0, 0, 0)
    assert lib.pano_debug_bounds(None) == binding.PANO_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(binding.PanoError):
        binding.load_library(str(tmp_path / "nope.so"))


def _rig_desc(**kw):
    d = binding.PanoRigDesc()
    d.n_pairs, d.h, d.c, d.dtype = 2, 64, 3, binding.PANO_U8
    d.canvas_h, d.canvas_w, d.canvas_y0 = 64, 200, 0
    d.w[0], d.w[1] = 40, 50
    d.canvas_x0[0], d.canvas_x0[1] = 0, 100
    for k, v in kw.items():
        if k in ("w", "canvas_x0"):
            for i, x in enumerate(v):
                getattr(d, k)[i] = x
        else:
            setattr(d, k, v)
    return d


_INV, _UNS = binding.PANO_ERR_INVALID_ARG, binding.PANO_ERR_UNSUPPORTED


@pytest.mark.parametrize("bad,status", [(dict(n_pairs=0), _INV), (dict(n_pairs=9), _INV), (dict(h=0), _INV),
                                        (dict(c=2), _UNS), (dict(dtype=7), _INV),
                                        (dict(dtype=binding.PANO_BF16), _UNS), (dict(canvas_w=0), _INV),
                                        (dict(canvas_y0=1), _INV), (dict(canvas_y0=-1), _INV),
                                        (dict(w=[0, 50]), _INV), (dict(w=[40, 201]), _INV),
                                        (dict(canvas_x0=[200, 0]), _INV), (dict(canvas_x0=[-1, 0]), _INV)])
def test_rig_create_rejects_bad_geometry_before_any_device_call(lib, bad, status):
    p = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(p))
    out = ctypes.c_void_p(5)
    d = _rig_desc(**bad)
    assert lib.pano_rig_create(ctypes.byref(p), ctypes.byref(d), ctypes.byref(out)) == status
    assert out.value is None
    assert lib.pano_last_error(None)


def test_rig_null_arguments(lib):
    p = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(p))
    d = _rig_desc()
    out = ctypes.c_void_p()
    assert lib.pano_rig_create(None, ctypes.byref(d), ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_create(ctypes.byref(p), None, ctypes.byref(out)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_create(ctypes.byref(p), ctypes.byref(d), None) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_run(None, None, None, None, None, None, 0, None) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_autotune(None, None, None, 1, None) == binding.PANO_ERR_INVALID_ARG
    t = binding.PanoRigTuning()
    assert lib.pano_rig_get_tuning(None, 0, ctypes.byref(t)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_set_tuning(None, 0, ctypes.byref(t)) == binding.PANO_ERR_INVALID_ARG
    assert lib.pano_rig_destroy(None) == binding.PANO_OK
    assert lib.pano_rig_launches(None) == 0 and lib.pano_rig_graph_captures(None) == 0


def test_static_flow_rejects_bad_arguments_before_any_device_call(lib):
    """pano_flow_pair_static runs the checks of pano_flow_pair (parameters,
    images, flows that must not overlap) before it touches the device."""
    inv = binding.PANO_ERR_INVALID_ARG
    p = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(p))
    img = binding.PanoImage(0x100000, 64, 64, 1, 256, binding.PANO_F32)
    n = 64 * 64 * 8

    def call(q=p, L=img, R=img, lr=0x200000, rl=0x200000 + n):
        return lib.pano_flow_pair_static(ctypes.byref(q) if q is not None else None, ctypes.byref(L),
                                         ctypes.byref(R), lr, rl, None)

    assert call(q=None) == inv
    assert call(rl=0x200000 + n - 8) == inv            # the two flows overlap by one pixel
    assert b"overlap" in lib.pano_last_error(None)
    assert call(lr=0x200004) == inv                    # not 8-byte aligned
    assert call(R=binding.PanoImage(0x100000, 64, 63, 1, 256, binding.PANO_F32)) == inv
    for field, value in (("soft_sharpness", float("nan")), ("flow_mag_coef", float("nan")), ("levels", 13),
                         ("radius", 4), ("lam", -1.0)):
        q = binding.PanoParams()
        lib.pano_flow_params_default(ctypes.byref(q))
        setattr(q, field, value)
        assert call(q=q) == inv, field
    q = binding.PanoParams()
    lib.pano_flow_params_default(ctypes.byref(q))
    q.pyr_dtype = binding.PANO_BF16
    assert call(q=q) == binding.PANO_ERR_UNSUPPORTED
    big = binding.PanoImage(0x100000, 2048, 2048, 1, 8192, binding.PANO_F32)
    assert call(L=big, R=big, rl=0x200000 + 2048 * 2048 * 8) == inv
    assert b"scratch" in lib.pano_last_error(None)
