"""NumPy front end of the FP64 CPU oracle (``pano_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and to time the GPU path. The
GPU library neither imports nor links it, and it imports nothing from the GPU
package.

Every function takes and returns NumPy arrays (float64 unless stated) and
mirrors one function of ``pano_oracle.c``; the C file states which passage of
the paper each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pano_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpano_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        sig = {
            "oracle_num_threads": ([], i),
            "oracle_set_num_threads": ([i], None),
            "oracle_to_unit_u8": ([_U8, l, _D], None),
            "oracle_luma": ([_D, i, i, i, _D], None),
            "oracle_pyr_down": ([_D, i, i, _D], None),
            "oracle_bilinear": ([_D, i, i, d, d], d),
            "oracle_bilinear_many": ([_D, i, i, _D, _D, l, _D], None),
            "oracle_warp": ([_D, i, i, i, _D, d, _D], None),
            "oracle_gradient": ([_D, i, i, _D, _D], None),
            "oracle_lk_step": ([_D, _D, i, i, _D, i, d], None),
            "oracle_upsample_flow": ([_D, i, i, _D, i, i], None),
            "oracle_pyramid": ([_D, i, i, i, _D], None),
            "oracle_pyramid_stored": ([_D, i, i, i, i, _D], None),
            "oracle_round_storage": ([_D, l, i], None),
            "oracle_flow_pair_stored": ([_D, _D, i, i, i, i, i, d, i, _D, _D], None),
            "oracle_flow_dir": ([_D, _D, i, i, i, i, i, d, _D], None),
            "oracle_flow_pair": ([_D, _D, i, i, i, i, i, d, _D, _D], None),
            "oracle_blend_coeff": ([_U8, i, i, _D], None),
            "oracle_blend_ramp": ([i, _D], None),
            "oracle_blend_coeff_at": ([_U8, i, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), l, _D],
                                      None),
            "oracle_blend": ([_D, _D, i, i, i, _D, _D, _D, d, d, _D], None),
            "oracle_blend_weights": ([i, i, _D, _D, _D, d, d, _D, _D], None),
            "oracle_compose": ([_D, _D, i, i, i, _U8, _D, _D, _D, i, i, i, i, d, d, _D], None),
            "oracle_quantize_u8": ([_D, l, _U8], None),
            "oracle_energy": ([_D, _D, i, i, _D, d], d),
            "oracle_energy_grad": ([_D, _D, i, i, _D, d, _D, _D, _D], None),
            "oracle_pyr_down_adjoint": ([_D, i, i, _D], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Method parameters. The paper publishes none of them; these defaults
    are this project's readings (window radius 2, 5 steps per level,
    damping 1e-2 in unit intensity squared, softmax sharpness 10,
    flow-magnitude coefficient 20)."""

    levels: int = 4
    iters: int = 5
    radius: int = 2
    lam: float = 1e-2
    soft_sharpness: float = 10.0
    flow_mag_coef: float = 20.0
    pyr_fmt: int = 0      # storage of the pyramid levels: FMT_EXACT, FMT_BF16 or FMT_F16


# storage formats of the pyramid levels (oracle_round_storage)
FMT_EXACT, FMT_BF16, FMT_F16 = 0, 1, 2


def round_storage(a, fmt: int) -> np.ndarray:
    """Every value rounded to the nearest value of the format (ties to even)."""
    out = _f64(a).copy()
    lib().oracle_round_storage(_d(out), out.size, int(fmt))
    return out


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def to_unit(img: np.ndarray) -> np.ndarray:
    """uint8 -> v / 255 in float64; float input -> float64 unchanged."""
    if img.dtype == np.uint8:
        a = np.ascontiguousarray(img)
        out = np.empty(a.shape, dtype=np.float64)
        lib().oracle_to_unit_u8(a.ctypes.data_as(_U8), a.size, _d(out))
        return out
    return _f64(img)


def luma(img_unit: np.ndarray) -> np.ndarray:
    a = _f64(img_unit)
    h, w = a.shape[:2]
    c = 1 if a.ndim == 2 else a.shape[2]
    out = np.empty((h, w), dtype=np.float64)
    lib().oracle_luma(_d(a), h, w, c, _d(out))
    return out


def pyr_down(src: np.ndarray) -> np.ndarray:
    a = _f64(src)
    h, w = a.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2), dtype=np.float64)
    lib().oracle_pyr_down(_d(a), h, w, _d(out))
    return out


def level_shapes(h: int, w: int, levels: int):
    shapes = [(h, w)]
    for _ in range(1, levels):
        ph, pw = shapes[-1]
        shapes.append(((ph + 1) // 2, (pw + 1) // 2))
    return shapes


def pyramid(Y: np.ndarray, levels: int, fmt: int = FMT_EXACT) -> list:
    a = _f64(Y)
    h, w = a.shape
    shapes = level_shapes(h, w, levels)
    flat = np.empty(sum(s[0] * s[1] for s in shapes), dtype=np.float64)
    if fmt == FMT_EXACT:
        lib().oracle_pyramid(_d(a), h, w, levels, _d(flat))
    else:
        lib().oracle_pyramid_stored(_d(a), h, w, levels, int(fmt), _d(flat))
    out, off = [], 0
    for sh, sw in shapes:
        out.append(flat[off:off + sh * sw].reshape(sh, sw).copy())
        off += sh * sw
    return out


def bilinear(I: np.ndarray, xs, ys) -> np.ndarray:
    a = _f64(I)
    h, w = a.shape
    xs = _f64(np.atleast_1d(xs))
    ys = _f64(np.atleast_1d(ys))
    out = np.empty(xs.shape, dtype=np.float64)
    lib().oracle_bilinear_many(_d(a), h, w, _d(xs), _d(ys), xs.size, _d(out))
    return out


def warp(src: np.ndarray, flow: np.ndarray, s: float = 1.0) -> np.ndarray:
    a = _f64(src)
    h, w = a.shape[:2]
    c = 1 if a.ndim == 2 else a.shape[2]
    f = _f64(flow)
    out = np.empty(a.shape, dtype=np.float64)
    lib().oracle_warp(_d(a), h, w, c, _d(f), float(s), _d(out))
    return out


def gradient(T: np.ndarray):
    a = _f64(T)
    h, w = a.shape
    ix = np.empty_like(a)
    iy = np.empty_like(a)
    lib().oracle_gradient(_d(a), h, w, _d(ix), _d(iy))
    return ix, iy


def lk_step(T: np.ndarray, J: np.ndarray, u: np.ndarray, radius: int, lam: float) -> np.ndarray:
    t, j = _f64(T), _f64(J)
    h, w = t.shape
    out = _f64(u).copy()
    lib().oracle_lk_step(_d(t), _d(j), h, w, _d(out), int(radius), float(lam))
    return out


def upsample_flow(uc: np.ndarray, h: int, w: int) -> np.ndarray:
    a = _f64(uc)
    hc, wc = a.shape[:2]
    out = np.empty((h, w, 2), dtype=np.float64)
    lib().oracle_upsample_flow(_d(a), hc, wc, _d(out), h, w)
    return out


def flow_dir(Tpyr: list, Jpyr: list, p: Params) -> np.ndarray:
    h, w = Tpyr[0].shape
    tf = np.concatenate([_f64(x).ravel() for x in Tpyr])
    jf = np.concatenate([_f64(x).ravel() for x in Jpyr])
    out = np.empty((h, w, 2), dtype=np.float64)
    lib().oracle_flow_dir(_d(tf), _d(jf), h, w, p.levels, p.iters, p.radius, p.lam, _d(out))
    return out


def flow_pair_luma(YL: np.ndarray, YR: np.ndarray, p: Params):
    """(FlowLtoR, FlowRtoL) from two unit-scaled luma planes."""
    yl, yr = _f64(YL), _f64(YR)
    h, w = yl.shape
    lr = np.empty((h, w, 2), dtype=np.float64)
    rl = np.empty((h, w, 2), dtype=np.float64)
    if p.pyr_fmt == FMT_EXACT:
        lib().oracle_flow_pair(_d(yl), _d(yr), h, w, p.levels, p.iters, p.radius, p.lam, _d(lr), _d(rl))
    else:
        lib().oracle_flow_pair_stored(_d(yl), _d(yr), h, w, p.levels, p.iters, p.radius, p.lam, int(p.pyr_fmt),
                                      _d(lr), _d(rl))
    return lr, rl


def flow_pair(L: np.ndarray, R: np.ndarray, p: Params):
    """(FlowLtoR, FlowRtoL) of a raw pair (uint8 or float, 1 or 3 channels)."""
    return flow_pair_luma(luma(to_unit(L)), luma(to_unit(R)), p)


def blend_coeff(label: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(label, dtype=np.uint8)
    h, w = a.shape
    out = np.empty((h, w), dtype=np.float64)
    lib().oracle_blend_coeff(a.ctypes.data_as(_U8), h, w, _d(out))
    return out


def blend_coeff_at(label: np.ndarray, ys, xs) -> np.ndarray:
    """Eq. (1) at the pixels (ys[i], xs[i]) only (brute force per pixel)."""
    a = np.ascontiguousarray(label, dtype=np.uint8)
    h, w = a.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.empty(ys.shape, dtype=np.float64)
    ip = ctypes.POINTER(ctypes.c_int)
    lib().oracle_blend_coeff_at(a.ctypes.data_as(_U8), h, w, ys.ctypes.data_as(ip), xs.ctypes.data_as(ip),
                                ys.size, _d(out))
    return out


def blend_ramp(w: int) -> np.ndarray:
    out = np.empty(w, dtype=np.float64)
    lib().oracle_blend_ramp(int(w), _d(out))
    return out


def blend(L: np.ndarray, R: np.ndarray, flowLR: np.ndarray, flowRL: np.ndarray,
          p: Params, blend_arr=None) -> np.ndarray:
    """Code 1 on unit-scaled inputs; returns F (float64, same shape as L)."""
    a, b = to_unit(L), to_unit(R)
    h, w = a.shape[:2]
    c = 1 if a.ndim == 2 else a.shape[2]
    lr, rl = _f64(flowLR), _f64(flowRL)
    bl = None if blend_arr is None else _f64(blend_arr)
    out = np.empty(a.shape, dtype=np.float64)
    lib().oracle_blend(_d(a), _d(b), h, w, c, _d(lr), _d(rl), None if bl is None else _d(bl),
                       p.soft_sharpness, p.flow_mag_coef, _d(out))
    return out


def compose(L: np.ndarray, R: np.ndarray, label: np.ndarray, blend_arr: np.ndarray, flowLR: np.ndarray,
            flowRL: np.ndarray, origin, p: Params) -> np.ndarray:
    """Code 1 on a canvas (every branch) on unit-scaled inputs; returns F
    (float64, same shape as L). origin = (row, column) of the flows' crop."""
    a, b = to_unit(L), to_unit(R)
    h, w = a.shape[:2]
    c = 1 if a.ndim == 2 else a.shape[2]
    lab = np.ascontiguousarray(label, dtype=np.uint8)
    assert lab.shape == (h, w)
    bl = _f64(blend_arr)
    lr, rl = _f64(flowLR), _f64(flowRL)
    fh, fw = lr.shape[:2]
    out = np.empty(a.shape, dtype=np.float64)
    lib().oracle_compose(_d(a), _d(b), h, w, c, lab.ctypes.data_as(_U8), _d(bl), _d(lr), _d(rl),
                         int(origin[0]), int(origin[1]), fh, fw, p.soft_sharpness, p.flow_mag_coef, _d(out))
    return out


def blend_weights(flowLR, flowRL, p: Params, blend_arr=None):
    lr, rl = _f64(flowLR), _f64(flowRL)
    h, w = lr.shape[:2]
    bl = None if blend_arr is None else _f64(blend_arr)
    sl = np.empty((h, w))
    sr = np.empty((h, w))
    lib().oracle_blend_weights(h, w, _d(lr), _d(rl), None if bl is None else _d(bl),
                               p.soft_sharpness, p.flow_mag_coef, _d(sl), _d(sr))
    return sl, sr


def quantize_u8(F: np.ndarray) -> np.ndarray:
    a = _f64(F)
    out = np.empty(a.shape, dtype=np.uint8)
    lib().oracle_quantize_u8(_d(a), a.size, out.ctypes.data_as(_U8))
    return out


def stitch_pair(L: np.ndarray, R: np.ndarray, p: Params, blend_arr=None):
    """Whole path: flows, then Code 1; uint8 inputs give uint8 F."""
    lr, rl = flow_pair(L, R, p)
    F = blend(L, R, lr, rl, p, blend_arr)
    if L.dtype == np.uint8:
        F = quantize_u8(F)
    return lr, rl, F


# ---------------------------------------------------------------------------
# differentiable refinement (energy, its gradients, REDUCE transpose)
# ---------------------------------------------------------------------------

def energy(T, J, u, alpha: float) -> float:
    t, j, uu = _f64(T), _f64(J), _f64(u)
    h, w = t.shape
    return float(lib().oracle_energy(_d(t), _d(j), h, w, _d(uu), float(alpha)))


def energy_grad(T, J, u, alpha: float):
    """(dE/du (h, w, 2), dE/dT (h, w), dE/dJ (h, w))."""
    t, j, uu = _f64(T), _f64(J), _f64(u)
    h, w = t.shape
    gu = np.empty((h, w, 2))
    gt = np.empty((h, w))
    gj = np.empty((h, w))
    lib().oracle_energy_grad(_d(t), _d(j), h, w, _d(uu), float(alpha), _d(gu), _d(gt), _d(gj))
    return gu, gt, gj


def pyr_down_adjoint(gdst: np.ndarray, h: int, w: int) -> np.ndarray:
    g = _f64(gdst)
    assert g.shape == ((h + 1) // 2, (w + 1) // 2)
    out = np.empty((h, w))
    lib().oracle_pyr_down_adjoint(_d(g), h, w, _d(out))
    return out
