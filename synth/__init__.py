"""Seeded synthetic overlap pairs.

The paper evaluates on 20 photo sets that are not public in any form usable
here, so every input is synthetic: a band-limited noise texture (the "left"
strip) and a copy of it displaced by a known dense field (the "right" strip).
The displacement plays the role of the residual misalignment that is left after
the coarse feature-based registration of Section III-B.

This module is shared by the tests, the oracle checks and the benchmark. It
holds none of the method's arithmetic: no pyramid, no flow estimation, no
blend. Resampling of the texture uses scipy's cubic-spline interpolation
(``order=3``), which is deliberately different from the bilinear sampler the
method uses, so a test never "recovers" a displacement with the same
interpolant that produced it.

Ground truth convention (Section III-C-1): ``flow_RtoL`` lives on the right
strip's grid and satisfies ``R(p) = L(p + flow_RtoL(p))``; ``flow_LtoR`` lives
on the left strip's grid and satisfies ``L(q) = R(q + flow_LtoR(q))``. The x
component is the column offset, y the row offset, both in pixels. Flow arrays
are ``(H, W, 2)`` float64 with ``[..., 0] = x``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
from scipy import ndimage

__all__ = [
    "Pair",
    "band_limited_texture",
    "make_pair",
    "pair_small_gray",
    "pair_fullres_rgb",
    "pair_translation",
    "rig_pairs",
    "inverse_field",
    "RIG_WIDTHS",
]

# Widths of the eight overlap strips of the 360-degree rig workload.
RIG_WIDTHS = (800, 950, 1100, 1250, 1400, 1600, 1800, 2000)

# Fixed colour mixing matrix: positive rows that sum to one, so three
# independent textures become a correlated RGB texture.
_COLOUR_MIX = np.array(
    [[0.60, 0.25, 0.15],
     [0.20, 0.60, 0.20],
     [0.15, 0.25, 0.60]], dtype=np.float64)


@dataclass
class Pair:
    """One synthetic overlap pair and its ground-truth flows."""

    name: str
    L: np.ndarray            # (H, W) or (H, W, 3); float32 in [0, 1] or uint8
    R: np.ndarray
    flow_RtoL: np.ndarray    # (H, W, 2) float64, R(p) = L(p + flow_RtoL(p))
    dfun: Callable           # d(ys, xs) -> (dx, dy), the field flow_RtoL samples
    levels: int
    meta: dict = field(default_factory=dict)
    _flow_LtoR: Optional[np.ndarray] = None

    @property
    def flow_LtoR(self) -> np.ndarray:
        """(H, W, 2) float64 with L(q) = R(q + flow_LtoR(q)); computed on first use."""
        if self._flow_LtoR is None:
            h, w = self.shape
            self._flow_LtoR = inverse_field(self.dfun, h, w)
        return self._flow_LtoR

    @property
    def shape(self):
        return self.L.shape[:2]

    @property
    def channels(self) -> int:
        return 1 if self.L.ndim == 2 else self.L.shape[2]


def band_limited_texture(rng: np.random.Generator, h: int, w: int,
                         sigmas=(1.0, 2.0, 4.0, 8.0)) -> np.ndarray:
    """Sum of Gaussian-filtered white-noise octaves, min-max scaled to [0, 1].

    Each octave is N(0,1) white noise filtered with a Gaussian of standard
    deviation ``sigma`` (truncated at 4 sigma, reflecting border) and rescaled
    to unit standard deviation before the octaves are summed.
    """
    acc = np.zeros((h, w), dtype=np.float64)
    for s in sigmas:
        n = rng.standard_normal((h, w))
        f = ndimage.gaussian_filter(n, s, truncate=4.0, mode="reflect")
        f /= f.std()
        acc += f
    acc -= acc.min()
    acc /= acc.max()
    return acc


def _sample(canvas: np.ndarray, pad: int, ys: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Cubic-spline sample of a padded canvas at strip coordinates (ys, xs)."""
    coords = np.stack([ys + pad, xs + pad])
    return ndimage.map_coordinates(canvas, coords, order=3, mode="reflect")


def inverse_field(dfun: Callable[[np.ndarray, np.ndarray], tuple],
                  h: int, w: int, iters: int = 30) -> np.ndarray:
    """Flow e on the left grid with e(q) = -d(q + e(q)) by fixed-point iteration.

    ``dfun(ys, xs) -> (dx, dy)`` evaluates the right-grid field d anywhere.
    """
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    ex = np.zeros((h, w))
    ey = np.zeros((h, w))
    for _ in range(iters):
        dx, dy = dfun(ys + ey, xs + ex)
        ex, ey = -dx, -dy
    return np.stack([ex, ey], axis=-1)


def make_pair(name: str, h: int, w: int, channels: int, dtype: str, seed: int,
              dfun: Callable[[np.ndarray, np.ndarray], tuple], levels: int,
              noise_std: float, gain_range: Optional[tuple] = None,
              pad: int = 64, meta: Optional[dict] = None) -> Pair:
    """Build a pair: L = texture crop, R(p) = texture(p + d(p)) (+ gain, noise).

    ``dtype`` is ``"f32"`` (values clipped to [0, 1]) or ``"u8"`` (scaled by
    255, rounded half to even and clipped).
    """
    rng = np.random.default_rng(seed)
    H, W = h + 2 * pad, w + 2 * pad
    if channels == 1:
        planes = [band_limited_texture(rng, H, W)]
    else:
        base = [band_limited_texture(rng, H, W) for _ in range(3)]
        planes = [sum(_COLOUR_MIX[c, k] * base[k] for k in range(3)) for c in range(3)]
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    dx, dy = dfun(ys, xs)
    L = np.stack([p[pad:pad + h, pad:pad + w] for p in planes], axis=-1)
    R = np.stack([_sample(p, pad, ys + dy, xs + dx) for p in planes], axis=-1)
    if gain_range is not None:
        gains = rng.uniform(gain_range[0], gain_range[1], size=channels)
        R = R * gains[None, None, :]
    if noise_std > 0:
        R = R + rng.normal(0.0, noise_std, size=R.shape)
    R = np.clip(R, 0.0, 1.0)
    L = np.clip(L, 0.0, 1.0)
    if dtype == "u8":
        L = np.clip(np.rint(L * 255.0), 0, 255).astype(np.uint8)
        R = np.clip(np.rint(R * 255.0), 0, 255).astype(np.uint8)
    elif dtype == "f32":
        L = L.astype(np.float32)
        R = R.astype(np.float32)
    else:
        raise ValueError(f"unsupported dtype {dtype!r}")
    if channels == 1:
        L = np.ascontiguousarray(L[..., 0])
        R = np.ascontiguousarray(R[..., 0])
    flow_RtoL = np.stack([dx, dy], axis=-1)
    return Pair(name=name, L=np.ascontiguousarray(L), R=np.ascontiguousarray(R),
                flow_RtoL=flow_RtoL, dfun=dfun, levels=levels,
                meta=dict(meta or {}, seed=seed, noise_std=noise_std))


def pair_small_gray(seed: int = 0, h: int = 256, w: int = 512, amp_x: float = 3.0,
                    amp_y: float = 1.5, levels: int = 4, noise_std: float = 0.01) -> Pair:
    """256x512 grayscale float32 pair with a smooth sinusoidal displacement.

    d = (amp_x sin(2 pi y / 128), amp_y cos(2 pi x / 256)), noise N(0, 0.01).
    """
    def dfun(ys, xs):
        return amp_x * np.sin(2 * np.pi * ys / 128.0), amp_y * np.cos(2 * np.pi * xs / 256.0)
    return make_pair(f"pair_{h}x{w}_gray_f32", h, w, 1, "f32", seed, dfun, levels, noise_std,
                     meta={"field": "sinusoid", "amp_x": amp_x, "amp_y": amp_y})


def _parallax_field(rng: np.random.Generator, h: int, w: int, dmax: float):
    """Piecewise-planar horizontal parallax with three slanted step edges.

    Four depth regions are separated by the lines y = h*k/4 + 0.1*x (k = 1..3).
    In region k, dx = a_k + b_k x/w + c_k y/h + 1.5 sin(2 pi y / 900), clipped
    to [0, dmax]; dy = 0.1 dx.
    """
    coef = []
    for _ in range(4):
        b = rng.uniform(-0.2, 0.2) * dmax
        c = rng.uniform(-0.2, 0.2) * dmax
        lo = max(0.0, -b, -c, -(b + c))
        hi = min(dmax, dmax - b, dmax - c, dmax - (b + c))
        a = rng.uniform(lo, max(lo, hi))
        coef.append((a, b, c))
    coef = np.array(coef)

    def dfun(ys, xs):
        k = np.zeros(np.shape(ys), dtype=np.int64)
        for j in range(1, 4):
            k += (ys > h * j / 4.0 + 0.1 * xs).astype(np.int64)
        a, b, c = np.take(coef[:, 0], k), np.take(coef[:, 1], k), np.take(coef[:, 2], k)
        dx = a + b * xs / w + c * ys / h + 1.5 * np.sin(2 * np.pi * ys / 900.0)
        dx = np.clip(dx, 0.0, dmax)
        return dx, 0.1 * dx
    return dfun


def pair_fullres_rgb(seed: int = 1, h: int = 4000, w: int = 1500, dmax: float = 20.0,
                     levels: int = 6, gain_range: Optional[tuple] = (0.9, 1.1)) -> Pair:
    """4000x1500 RGB uint8 pair: colour texture, 0-dmax px parallax with steps,
    per-channel gain U(gain_range) (None: no gain) and N(0, 2/255) noise."""
    rng = np.random.default_rng(10_000 + seed)
    dfun = _parallax_field(rng, h, w, dmax)
    return make_pair(f"pair_{h}x{w}_rgb_u8", h, w, 3, "u8", seed, dfun, levels,
                     noise_std=2.0 / 255.0, gain_range=gain_range,
                     meta={"field": "parallax", "dmax": dmax, "gain_range": gain_range})


def pair_translation(dx: float, dy: float, seed: int = 5, h: int = 96, w: int = 128,
                     levels: int = 3, noise_std: float = 0.0, dtype: str = "f32",
                     channels: int = 1) -> Pair:
    """Pair related by a constant translation: R(p) = L(p + (dx, dy))."""
    def dfun(ys, xs):
        return np.full(np.shape(ys), float(dx)), np.full(np.shape(ys), float(dy))
    return make_pair(f"pair_{h}x{w}_shift", h, w, channels, dtype, seed, dfun, levels, noise_std,
                     meta={"field": "translation", "dx": dx, "dy": dy})


def _rig_pair_arrays(args):
    """Worker of rig_pairs: the arrays of one pair (the field closure stays
    behind; the parent rebuilds it from the same seed)."""
    seed, h, w, dmax, levels = args
    p = pair_fullres_rgb(seed=seed, h=h, w=w, dmax=dmax, levels=levels)
    return p.name, p.L, p.R, p.flow_RtoL, p.meta


def rig_pairs(h: int = 4000, widths=RIG_WIDTHS, dmax: float = 24.0, levels: int = 6,
              seed0: int = 100, workers: int = 1) -> list:
    """Eight overlap pairs of a 360-degree rig with uneven widths.

    workers > 1 generates the pairs in that many processes (started with
    ``spawn``, so it is safe in a process that already uses a GPU); the pairs
    are the same as with one worker."""
    jobs = [(seed0 + k, h, wk, dmax, levels) for k, wk in enumerate(widths)]
    if workers <= 1:
        return [pair_fullres_rgb(seed=s, h=hh, w=ww, dmax=d, levels=lv) for s, hh, ww, d, lv in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=min(workers, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
        arrays = list(ex.map(_rig_pair_arrays, jobs))
    out = []
    for (seed, hh, ww, d, lv), (name, L, R, flow, meta) in zip(jobs, arrays):
        dfun = _parallax_field(np.random.default_rng(10_000 + seed), hh, ww, d)
        out.append(Pair(name=name, L=L, R=R, flow_RtoL=flow, dfun=dfun, levels=lv, meta=meta))
    return out
