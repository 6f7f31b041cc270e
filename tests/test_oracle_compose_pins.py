"""Pins of the oracle's whole-canvas Code 1 (Section III-C-3, every branch).

What fixes each branch independently of the oracle's own formula:
  * Area1 / Area2 / neither: exact copies of L, of R, and zeros (Code 1,
    lines 2-5 and 22-23);
  * Area3 with a constant integer translation and exact flows: whatever the
    softmax weights, F(p) = L(p + Blend(p) d), checked against scipy's
    bilinear sampler;
  * swapping the roles of L and R (labels 1 <-> 2, Blend -> 1 - Blend, the
    two flows exchanged) gives the same F bit for bit;
  * the crop's canvas origin: flows given for a crop equal the same flows
    placed in a canvas-sized field (with the flow-magnitude term off, which
    divides by the crop width);
  * a canvas holding one overlap strip between Area1 and Area2 reduces, in the
    strip, to the strip form of Code 1 (itself pinned in test_oracle_pins).
"""
import numpy as np
import pytest

import oracle


def _texture(h, w, c, seed):
    from scipy import ndimage
    g = np.random.default_rng(seed)
    planes = [ndimage.gaussian_filter(g.uniform(0, 1, size=(h, w)), 1.5, mode="reflect") for _ in range(c)]
    return np.stack(planes, -1) if c > 1 else planes[0]


def _canvas(h, w, seed=0):
    """Area1 on the left, Area2 on the right, Area3 between them with a wavy
    seam band, and a 'neither' border row on top."""
    g = np.random.default_rng(seed)
    xs = np.arange(w)[None, :]
    ys = np.arange(h)[:, None]
    a = (w // 3 + 2 * np.sin(ys / 3.0)).astype(int)
    b = (2 * w // 3 + 2 * np.cos(ys / 4.0)).astype(int)
    lab = np.where(xs < a, 1, np.where(xs >= b, 2, 3)).astype(np.uint8)
    lab[0, :] = 0
    lab[1, g.integers(0, w)] = 7                     # a label outside {1, 2, 3}: neither
    return lab


def test_area1_area2_and_neither_are_copies_and_zeros():
    h, w, c = 20, 30, 3
    L, R = _texture(h, w, c, 1), _texture(h, w, c, 2)
    lab = _canvas(h, w)
    B = oracle.blend_coeff(lab)
    g = np.random.default_rng(3)
    fl = g.normal(0, 2, size=(h, w, 2))
    F = oracle.compose(L, R, lab, B, fl, -fl, (0, 0), oracle.Params())
    assert np.array_equal(F[lab == 1], L[lab == 1])
    assert np.array_equal(F[lab == 2], R[lab == 2])
    neither = (lab != 1) & (lab != 2) & (lab != 3)
    assert neither.any() and np.all(F[neither] == 0.0)


@pytest.mark.parametrize("d", [(2, -1), (-3, 1)])
def test_area3_constant_translation_closed_form(d):
    from scipy import ndimage
    h, w = 40, 60
    T = _texture(h + 20, w + 20, 1, 4)
    L = T[10:10 + h, 10:10 + w]
    R = T[10 + d[1]:10 + d[1] + h, 10 + d[0]:10 + d[0] + w]     # R(p) = L(p + d)
    lab = _canvas(h, w)
    B = oracle.blend_coeff(lab)
    y0, x0, fh, fw = 2, 15, 36, 30
    rl = np.tile(np.array(d, float), (fh, fw, 1))             # FlowRtoL = d, FlowLtoR = -d
    F = oracle.compose(L, R, lab, B, -rl, rl, (y0, x0), oracle.Params())
    yy, xx = np.nonzero(lab == 3)
    inside = (yy >= y0 + 4) & (yy < y0 + fh - 4) & (xx >= x0) & (xx < x0 + fw)
    yy, xx = yy[inside], xx[inside]
    want = ndimage.map_coordinates(L, [yy + B[yy, xx] * d[1], xx + B[yy, xx] * d[0]], order=1, mode="nearest")
    assert len(yy) > 100
    np.testing.assert_allclose(F[yy, xx], want, rtol=0, atol=1e-12)


def test_swapping_the_roles_of_L_and_R_is_exact():
    h, w, c = 24, 36, 3
    L, R = _texture(h, w, c, 5), _texture(h, w, c, 6)
    lab = _canvas(h, w, 1)
    B = np.round(oracle.blend_coeff(lab) * 1024) / 1024   # dyadic: 1 - (1 - B) == B exactly
    g = np.random.default_rng(7)
    lr, rl = g.normal(0, 1.5, size=(20, 18, 2)), g.normal(0, 1.5, size=(20, 18, 2))
    p = oracle.Params()
    F = oracle.compose(L, R, lab, B, lr, rl, (2, 9), p)
    swapped = np.where(lab == 1, 2, np.where(lab == 2, 1, lab)).astype(np.uint8)
    G = oracle.compose(R, L, swapped, 1.0 - B, rl, lr, (2, 9), p)
    assert np.array_equal(F, G)


def test_crop_origin_places_the_flows_on_the_canvas():
    h, w = 30, 40
    L, R = _texture(h, w, 1, 8), _texture(h, w, 1, 9)
    lab = _canvas(h, w, 2)
    B = oracle.blend_coeff(lab)
    g = np.random.default_rng(10)
    y0, x0, fh, fw = 3, 11, 22, 17
    lr, rl = g.normal(0, 2, size=(fh, fw, 2)), g.normal(0, 2, size=(fh, fw, 2))
    full_lr, full_rl = np.zeros((h, w, 2)), np.zeros((h, w, 2))
    full_lr[y0:y0 + fh, x0:x0 + fw] = lr
    full_rl[y0:y0 + fh, x0:x0 + fw] = rl
    p = oracle.Params(flow_mag_coef=0.0)
    F = oracle.compose(L, R, lab, B, lr, rl, (y0, x0), p)
    G = oracle.compose(L, R, lab, B, full_lr, full_rl, (0, 0), p)
    assert np.array_equal(F, G)


def test_strip_canvas_reduces_to_the_strip_form():
    # Area1 | strip | Area2 with the strip ramp of Eq. (1) and flows that keep
    # every sample inside the strip: the canvas form and the strip form agree
    h, ws, c = 16, 24, 3
    w = ws + 8
    L, R = _texture(h, w, c, 11), _texture(h, w, c, 12)
    lab = np.full((h, w), 3, np.uint8)
    lab[:, :4] = 1
    lab[:, 4 + ws:] = 2
    B = oracle.blend_coeff(lab)
    g = np.random.default_rng(13)
    lr = g.uniform(-0.4, 0.4, size=(h, ws, 2))
    rl = g.uniform(-0.4, 0.4, size=(h, ws, 2))
    lr[:, :2], rl[:, :2], lr[:, -2:], rl[:, -2:] = 0, 0, 0, 0
    lr[:2], rl[:2], lr[-2:], rl[-2:] = 0, 0, 0, 0
    p = oracle.Params()
    F = oracle.compose(L, R, lab, B, lr, rl, (0, 4), p)
    strip = oracle.blend(L[:, 4:4 + ws], R[:, 4:4 + ws], lr, rl, p, blend_arr=B[:, 4:4 + ws])
    np.testing.assert_allclose(F[:, 4:4 + ws], strip, rtol=0, atol=1e-12)
    np.testing.assert_allclose(B[:, 4:4 + ws], np.tile(oracle.blend_ramp(ws), (h, 1)), rtol=0, atol=1e-12)
