"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks one oracle function against a library routine that computes
the same special case (scipy / numpy), a brute-force solve, a closed form, a
hand-derived value from the paper's equations, or an invariant that the
paper's definitions force. Together they are chosen so that a dropped term,
a flipped sign, a swapped x/y or a transposed operand anywhere in the oracle
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed=0):
    return np.random.default_rng(seed)


def interior(a, m):
    return a[m:-m, m:-m]


def epe(a, b, m):
    d = np.hypot(*(a - b).transpose(2, 0, 1))
    return interior(d, m)


# --------------------------------------------------------------------------
# unit scaling, luma
# --------------------------------------------------------------------------

def test_to_unit_u8_endpoints_and_scale():
    a = np.array([0, 1, 128, 254, 255], dtype=np.uint8)
    out = oracle.to_unit(a)
    assert out[0] == 0.0 and out[-1] == 1.0
    np.testing.assert_allclose(out * 255.0, a.astype(np.float64), rtol=0, atol=1e-12)


def test_luma_gray_is_identity_and_weights_are_bt601():
    # a neutral colour keeps its value (the weights sum to one) ...
    g = rng(1).uniform(0, 1, size=(5, 7))
    rgb = np.stack([g, g, g], axis=-1)
    np.testing.assert_allclose(oracle.luma(rgb), g, rtol=0, atol=1e-15)
    # ... and each primary alone returns its BT.601 weight (ITU-R BT.601)
    for ch, wt in enumerate((0.299, 0.587, 0.114)):
        img = np.zeros((2, 3, 3))
        img[..., ch] = 1.0
        np.testing.assert_allclose(oracle.luma(img), wt, rtol=0, atol=1e-15)
    # one channel passes through
    np.testing.assert_array_equal(oracle.luma(g), g)


# --------------------------------------------------------------------------
# pyramid
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(7, 9), (8, 8), (13, 6), (1, 5), (2, 2)])
def test_pyr_down_matches_scipy_binomial_reduce(shape):
    src = rng(2).uniform(0, 1, size=shape)
    k = np.array([1, 4, 6, 4, 1], dtype=np.float64) / 16.0
    ref = ndimage.correlate1d(src, k, axis=0, mode="nearest")
    ref = ndimage.correlate1d(ref, k, axis=1, mode="nearest")[::2, ::2]
    out = oracle.pyr_down(src)
    assert out.shape == ((shape[0] + 1) // 2, (shape[1] + 1) // 2)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14)


def test_pyr_down_constant_and_linear_ramp():
    c = np.full((11, 14), 0.3141)
    np.testing.assert_allclose(oracle.pyr_down(c), 0.3141, rtol=0, atol=1e-15)
    # a symmetric kernel reproduces affine functions, so a ramp a + b x + c y
    # sampled at the kept (even) pixels is the same ramp with doubled slopes
    ys, xs = np.mgrid[0:20, 0:24].astype(np.float64)
    ramp = 0.2 + 0.01 * xs - 0.003 * ys
    out = oracle.pyr_down(ramp)
    yd, xd = np.mgrid[0:10, 0:12].astype(np.float64)
    expect = 0.2 + 0.02 * xd - 0.006 * yd
    np.testing.assert_allclose(out[1:-1, 1:-1], expect[1:-1, 1:-1], rtol=0, atol=1e-14)


def test_pyramid_level_shapes_and_chain():
    Y = rng(3).uniform(0, 1, size=(37, 50))
    pyr = oracle.pyramid(Y, 4)
    assert [p.shape for p in pyr] == [(37, 50), (19, 25), (10, 13), (5, 7)]
    np.testing.assert_array_equal(pyr[0], Y)
    for l in range(1, 4):
        np.testing.assert_array_equal(pyr[l], oracle.pyr_down(pyr[l - 1]))


# --------------------------------------------------------------------------
# bilinear sampler, warp, gradient
# --------------------------------------------------------------------------

def test_bilinear_matches_scipy_order1_nearest():
    I = rng(4).uniform(0, 1, size=(9, 11))
    r = rng(5)
    xs = r.uniform(-3, 14, size=500)
    ys = r.uniform(-3, 12, size=500)
    ref = ndimage.map_coordinates(I, [ys, xs], order=1, mode="nearest")
    np.testing.assert_allclose(oracle.bilinear(I, xs, ys), ref, rtol=0, atol=1e-14)


def test_bilinear_exact_at_pixels_and_affine_inside():
    I = rng(6).uniform(0, 1, size=(6, 8))
    ys, xs = np.mgrid[0:6, 0:8].astype(np.float64)
    np.testing.assert_array_equal(oracle.bilinear(I, xs.ravel(), ys.ravel()), I.ravel())
    A = 0.5 + 0.25 * xs - 0.125 * ys
    r = rng(7)
    px, py = r.uniform(0, 7, 200), r.uniform(0, 5, 200)
    np.testing.assert_allclose(oracle.bilinear(A, px, py), 0.5 + 0.25 * px - 0.125 * py,
                               rtol=0, atol=1e-14)


def test_warp_integer_shift_and_identity():
    img = rng(8).uniform(0, 1, size=(10, 12, 3))
    zero = np.zeros((10, 12, 2))
    np.testing.assert_array_equal(oracle.warp(img, zero, 1.0), img)
    flow = np.zeros((10, 12, 2))
    flow[..., 0] = 2.0
    flow[..., 1] = -1.0
    out = oracle.warp(img, flow, 1.0)
    # out(y, x) = img(y - 1, x + 2) wherever that stays inside the image
    np.testing.assert_array_equal(out[1:, :-2], img[:-1, 2:])
    # the scale factor multiplies the flow
    np.testing.assert_array_equal(oracle.warp(img, 2 * flow, 0.5), out)


def test_gradient_is_central_difference_with_replicate_border():
    T = rng(9).uniform(0, 1, size=(7, 9))
    ix, iy = oracle.gradient(T)
    padded = np.pad(T, 1, mode="edge")
    gy, gx = np.gradient(padded)
    np.testing.assert_allclose(ix, gx[1:-1, 1:-1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(iy, gy[1:-1, 1:-1], rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# one Lucas-Kanade step
# --------------------------------------------------------------------------

def _lk_step_bruteforce(T, J, u, r, lam):
    """Per pixel, the stacked least-squares system solved by numpy.lstsq.

    Rows: one per in-image window sample q,
        [Ix(q) Iy(q)] v = Ix(q) ux(q) + Iy(q) uy(q) - It(q),
    with It(q) = J(q + u(q)) - T(q) (scipy bilinear, nearest border), plus two
    rows sqrt(lam) v = sqrt(lam) u(p).
    """
    h, w = T.shape
    padded = np.pad(T, 1, mode="edge")
    gy, gx = np.gradient(padded)
    gx, gy = gx[1:-1, 1:-1], gy[1:-1, 1:-1]
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    It = ndimage.map_coordinates(J, [ys + u[..., 1], xs + u[..., 0]], order=1, mode="nearest") - T
    out = np.empty_like(u)
    for y in range(h):
        for x in range(w):
            rows, rhs = [], []
            for qy in range(max(0, y - r), min(h, y + r + 1)):
                for qx in range(max(0, x - r), min(w, x + r + 1)):
                    rows.append([gx[qy, qx], gy[qy, qx]])
                    rhs.append(gx[qy, qx] * u[qy, qx, 0] + gy[qy, qx] * u[qy, qx, 1] - It[qy, qx])
            s = math.sqrt(lam)
            rows += [[s, 0.0], [0.0, s]]
            rhs += [s * u[y, x, 0], s * u[y, x, 1]]
            out[y, x] = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return out


@pytest.mark.parametrize("r,lam", [(1, 1e-3), (2, 1e-2), (2, 1e-4)])
def test_lk_step_matches_bruteforce_least_squares(r, lam):
    g = rng(10)
    T = ndimage.gaussian_filter(g.uniform(0, 1, size=(9, 11)), 1.0)
    J = ndimage.gaussian_filter(g.uniform(0, 1, size=(9, 11)), 1.0)
    u = g.normal(0, 0.8, size=(9, 11, 2))
    got = oracle.lk_step(T, J, u, r, lam)
    ref = _lk_step_bruteforce(T, J, u, r, lam)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)


def test_lk_step_identical_images_zero_flow_stays_zero():
    T = rng(11).uniform(0, 1, size=(16, 20))
    u = np.zeros((16, 20, 2))
    np.testing.assert_array_equal(oracle.lk_step(T, T, u, 2, 1e-2), u)


def test_lk_step_integer_translation_is_a_fixed_point_and_attracts():
    # T(y, x) = big(y + 10, x + 10) and J(y, x) = big(y + 8, x + 13), so
    # J(q + d) = T(q) with d = (-3, 2) wherever q + d stays inside J. Then
    # u = d must be left unchanged (It = 0 and the linearisation is exact),
    # and a perturbed start must move towards d.
    big = ndimage.gaussian_filter(rng(12).uniform(0, 1, size=(60, 70)), 1.5)
    T = big[10:50, 10:60]
    J = big[8:48, 13:63]
    d = np.array([-3.0, 2.0])
    u = np.broadcast_to(d, T.shape + (2,)).copy()
    m = 6
    out = oracle.lk_step(T, J, u, 2, 1e-2)
    np.testing.assert_allclose(interior(out, m), interior(u, m), rtol=0, atol=1e-12)
    start = u + rng(13).normal(0, 0.3, size=u.shape)
    cur = start
    for _ in range(6):
        cur = oracle.lk_step(T, J, cur, 2, 1e-2)
    assert interior(np.abs(cur - u), m).mean() < 0.1 * interior(np.abs(start - u), m).mean()


# --------------------------------------------------------------------------
# coarse-to-fine propagation
# --------------------------------------------------------------------------

def test_upsample_flow_matches_scipy_and_doubles():
    uc = rng(14).normal(0, 1, size=(5, 7, 2))
    h, w = 10, 13
    out = oracle.upsample_flow(uc, h, w)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    for c in range(2):
        ref = 2.0 * ndimage.map_coordinates(uc[..., c], [ys / 2, xs / 2], order=1, mode="nearest")
        np.testing.assert_allclose(out[..., c], ref, rtol=0, atol=1e-14)
    const = np.full((4, 6, 2), 0.75)
    np.testing.assert_allclose(oracle.upsample_flow(const, 8, 11), 1.5, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# pyramidal flow in both directions
# --------------------------------------------------------------------------

def test_flow_pair_identical_strips_give_zero_flow():
    L = synth.pair_translation(0.0, 0.0, h=48, w=64, levels=3).L
    lr, rl = oracle.flow_pair(L, L, oracle.Params(levels=3))
    assert np.all(lr == 0.0) and np.all(rl == 0.0)


def test_flow_pair_swap_symmetry_bit_exact():
    p = synth.pair_small_gray(h=64, w=96, levels=3)
    P = oracle.Params(levels=3)
    lr, rl = oracle.flow_pair(p.L, p.R, P)
    lr2, rl2 = oracle.flow_pair(p.R, p.L, P)
    np.testing.assert_array_equal(lr2, rl)
    np.testing.assert_array_equal(rl2, lr)


def test_flow_pair_recovers_subpixel_translation():
    # measured 0.0525 / 0.0561 px; the same at lambda = 1e-4 and 0, and with the
    # per-window form of LK: the floor comes from sampling the target bilinearly
    # on a texture with a 1 px octave, not from the damping
    p = synth.pair_translation(0.37, -0.21, levels=3)
    lr, rl = oracle.flow_pair(p.L, p.R, oracle.Params(levels=3))
    m = 4 * 3
    assert epe(rl, p.flow_RtoL, m).mean() < 0.065
    assert epe(lr, p.flow_LtoR, m).mean() < 0.065
    # direction and axis: the mean flow has the sign and axis of the shift
    np.testing.assert_allclose(interior(rl, m).mean(axis=(0, 1)), [0.37, -0.21], atol=0.03)
    np.testing.assert_allclose(interior(lr, m).mean(axis=(0, 1)), [-0.37, 0.21], atol=0.03)


def test_flow_pair_needs_the_pyramid_for_large_motion():
    # a 6.5 px shift is far outside one level's basin; three levels (scale 4)
    # bring it to ~1.6 px at the coarsest level. This pins the doubling in the
    # coarse-to-fine step: without it the level-0 start would be half of d.
    p = synth.pair_translation(6.5, 2.25, h=96, w=128, levels=3)
    m = 16
    one = oracle.flow_pair(p.L, p.R, oracle.Params(levels=1))[1]
    three = oracle.flow_pair(p.L, p.R, oracle.Params(levels=3))[1]
    assert epe(three, p.flow_RtoL, m).mean() < 0.1
    assert epe(one, p.flow_RtoL, m).mean() > 1.0


def test_flow_pair_recovers_smooth_field_small_config():
    # measured 0.1084 / 0.1092 px (0.1098 / 0.1106 at lambda = 1e-4)
    p = synth.pair_small_gray()
    lr, rl = oracle.flow_pair(p.L, p.R, oracle.Params(levels=4))
    m = 8 * 3
    assert epe(rl, p.flow_RtoL, m).mean() < 0.125
    assert epe(lr, p.flow_LtoR, m).mean() < 0.125


def test_damping_keeps_flow_small_where_the_template_is_flat():
    # The damping lambda pulls v towards u(p) where G(p) is small. On a patch
    # with noise and no texture, lambda = 1e-2 (unit intensities) keeps the
    # noise-driven flow near zero; 1e-4 lets it wander by pixels. The textured
    # part is the same under both.
    p = synth.pair_translation(0.37, -0.21, h=96, w=128, levels=3)
    g = np.random.default_rng(3)
    L, R = p.L.copy(), p.R.copy()
    L[:, :48] = 0.5 + g.normal(0, 0.01, (96, 48))
    R[:, :48] = 0.5 + g.normal(0, 0.01, (96, 48))
    out = {}
    for lam in (1e-2, 1e-4):
        lr, rl = oracle.flow_pair(L.astype(np.float32), R.astype(np.float32), oracle.Params(levels=3, lam=lam))
        flat = np.hypot(*rl[12:-12, 12:36].transpose(2, 0, 1)).mean()
        tex = epe(rl, p.flow_RtoL, 12)[:, 40:].mean()
        out[lam] = (flat, tex)
    assert out[1e-2][0] < 0.3 and out[1e-4][0] > 1.0      # measured 0.18 and 1.69 px
    assert abs(out[1e-2][1] - out[1e-4][1]) < 0.005 and out[1e-2][1] < 0.065


# --------------------------------------------------------------------------
# Eq. (1)
# --------------------------------------------------------------------------

def _read_golden_canvases():
    cases, cur, mode = [], None, None
    with open(os.path.join(GOLDEN, "eq1_blend_coefficient.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("canvas"):
                cur = {"name": line.split()[1], "label": [], "expect": []}
                cases.append(cur)
                mode = "label"
            elif line == "expect":
                mode = "expect"
            elif mode == "label":
                cur["label"].append([int(t) for t in line.split()])
            else:
                env = {"sqrt": math.sqrt, "__builtins__": {}}
                cur["expect"].append([float(eval(t, env)) for t in line.split()])
    return cases


@pytest.mark.parametrize("case", _read_golden_canvases(), ids=lambda c: c["name"])
def test_blend_coeff_golden_eq1(case):
    out = oracle.blend_coeff(np.array(case["label"], dtype=np.uint8))
    np.testing.assert_allclose(out, np.array(case["expect"]), rtol=0, atol=1e-15)


def test_blend_coeff_matches_scipy_edt_on_random_masks():
    g = rng(15)
    label = g.choice([0, 1, 2, 3], p=[0.1, 0.1, 0.1, 0.7], size=(12, 15)).astype(np.uint8)
    label[0, 0], label[-1, -1] = 1, 2
    lmin = ndimage.distance_transform_edt(label != 1)
    rmin = ndimage.distance_transform_edt(label != 2)
    expect = np.full(label.shape, 0.5)
    expect[label == 1] = 0.0
    expect[label == 2] = 1.0
    a3 = label == 3
    expect[a3] = lmin[a3] / (lmin[a3] + rmin[a3])
    np.testing.assert_allclose(oracle.blend_coeff(label), expect, rtol=0, atol=1e-14)


def test_blend_coeff_at_sampled_pixels_matches_scipy_edt():
    g = rng(16)
    label = g.choice([0, 1, 2, 3], p=[0.05, 0.02, 0.03, 0.9], size=(40, 70)).astype(np.uint8)
    dl = ndimage.distance_transform_edt(label != 1)
    dr = ndimage.distance_transform_edt(label != 2)
    expect = np.where(label == 1, 0.0, np.where(label == 2, 1.0, np.where(label == 3, dl / (dl + dr), 0.5)))
    ys, xs = np.nonzero(np.ones_like(label))
    got = oracle.blend_coeff_at(label, ys, xs).reshape(label.shape)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-14)
    lab = np.full((4, 6), 3, np.uint8)
    lab[0, 0] = 2
    assert (oracle.blend_coeff_at(lab, [1, 3], [2, 5]) == 1.0).all()


def test_blend_coeff_with_a_missing_area_is_the_limit_of_eq1():
    # no Area1 pixel: Lmin -> infinity, Lmin / (Lmin + Rmin) -> 1; no Area2: -> 0
    lab = np.full((3, 5), 3, np.uint8)
    lab[:, -1] = 2
    out = oracle.blend_coeff(lab)
    assert (out[:, :-1] == 1.0).all() and (out[:, -1] == 1.0).all()
    lab[:, -1] = 1
    out = oracle.blend_coeff(lab)
    assert (out[:, :-1] == 0.0).all() and (out[:, -1] == 0.0).all()
    lab[:, -1] = 0
    assert (oracle.blend_coeff(lab) == 0.5).all()


@pytest.mark.parametrize("w", [1, 4, 9, 31])
def test_blend_ramp_is_eq1_for_a_strip(w):
    # canvas: Area1 column, w overlap columns, Area2 column, 3 rows
    label = np.full((3, w + 2), 3, dtype=np.uint8)
    label[:, 0], label[:, -1] = 1, 2
    full = oracle.blend_coeff(label)
    np.testing.assert_allclose(oracle.blend_ramp(w), full[1, 1:-1], rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# Code 1 blend
# --------------------------------------------------------------------------

P_BLEND = oracle.Params()


def test_blend_identical_strips_zero_flow_returns_input():
    L = rng(16).uniform(0, 1, size=(8, 10, 3))
    z = np.zeros((8, 10, 2))
    np.testing.assert_allclose(oracle.blend(L, L, z, z, P_BLEND), L, rtol=0, atol=1e-15)
    L8 = (L * 255).astype(np.uint8)
    F8 = oracle.quantize_u8(oracle.blend(L8, L8, z, z, P_BLEND))
    np.testing.assert_array_equal(F8, L8)


@pytest.mark.parametrize("d", [(2.0, -1.0), (0.6, 0.3)])
def test_blend_closed_form_for_constant_translation(d):
    # R(p) = L(p + d) with exact flows FlowRtoL = d, FlowLtoR = -d. Code 1 then
    # samples ColorL = L(p + B d) and ColorR = R(p - (1 - B) d) = L(p + B d),
    # so F(p) = L(p + B(p) d) whatever the softmax weights are.
    big = ndimage.gaussian_filter(rng(17).uniform(0, 1, size=(40, 60)), 1.0)
    h, w = 24, 36
    oy, ox = 8, 10
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    L = big[oy:oy + h, ox:ox + w]
    R = ndimage.map_coordinates(big, [ys + oy + d[1], xs + ox + d[0]], order=1)
    flowRL = np.broadcast_to(np.array(d), (h, w, 2)).copy()
    flowLR = -flowRL
    F = oracle.blend(L, R, flowLR, flowRL, P_BLEND)
    B = (xs + 1) / (w + 1)
    expect = ndimage.map_coordinates(big, [ys + oy + B * d[1], xs + ox + B * d[0]], order=1)
    m = 4
    tol = 1e-12 if float(d[0]).is_integer() and float(d[1]).is_integer() else 2e-2
    # sub-pixel d: R itself is a bilinear resample, so ColorR is a resample of
    # a resample; the identity then holds to interpolation error only
    np.testing.assert_allclose(interior(F, m), interior(expect, m), rtol=0, atol=tol)


def test_blend_swap_symmetry_exact():
    g = rng(18)
    h, w = 10, 14
    L = g.uniform(0, 1, size=(h, w, 3))
    R = g.uniform(0, 1, size=(h, w, 3))
    lr = g.normal(0, 2, size=(h, w, 2))
    rl = g.normal(0, 2, size=(h, w, 2))
    B = g.uniform(0, 1, size=(h, w))
    F = oracle.blend(L, R, lr, rl, P_BLEND, B)
    Fs = oracle.blend(R, L, rl, lr, P_BLEND, 1.0 - B)
    np.testing.assert_allclose(Fs, F, rtol=0, atol=1e-14)


def test_blend_mirror_symmetry_with_strip_ramp():
    # mirroring columns turns the ramp B into 1 - B, so swapping the strips,
    # mirroring them and negating the flows' x component mirrors F.
    g = rng(19)
    h, w = 9, 13
    L = g.uniform(0, 1, size=(h, w))
    R = g.uniform(0, 1, size=(h, w))
    lr = g.normal(0, 1.5, size=(h, w, 2))
    rl = g.normal(0, 1.5, size=(h, w, 2))

    def mirror_flow(f):
        f = f[:, ::-1].copy()
        f[..., 0] *= -1
        return f
    F = oracle.blend(L, R, lr, rl, P_BLEND)
    Fm = oracle.blend(R[:, ::-1], L[:, ::-1], mirror_flow(rl), mirror_flow(lr), P_BLEND)
    np.testing.assert_allclose(Fm[:, ::-1], F, rtol=0, atol=1e-14)


def test_blend_weights_sum_to_one_and_follow_the_blend_coefficient():
    g = rng(20)
    h, w = 6, 40
    lr = g.normal(0, 3, size=(h, w, 2))
    rl = g.normal(0, 3, size=(h, w, 2))
    sl, sr = oracle.blend_weights(lr, rl, P_BLEND)
    np.testing.assert_allclose(sl + sr, 1.0, rtol=0, atol=1e-15)
    z = np.zeros((h, w, 2))
    sl0, sr0 = oracle.blend_weights(z, z, P_BLEND)
    # with no flow, the weight of R grows from near 0 at Area1 to near 1 at
    # Area2, passing 1/2 in the middle of the strip
    assert np.all(np.diff(sr0, axis=1) > 0)
    assert sr0[0, 0] < 1e-3 and sr0[0, -1] > 1 - 1e-3
    odd = oracle.blend_weights(np.zeros((1, 5, 2)), np.zeros((1, 5, 2)), P_BLEND)[1]
    assert abs(odd[0, 2] - 0.5) < 1e-15


def test_blend_larger_RtoL_flow_pulls_weight_towards_L():
    # Code 1: FlowL (which scales the exponent of L) grows with FlowMagRL, the
    # magnitude of FlowRtoL. With L = 0 and R = 1 and Blend = 1/2, F is the
    # weight of R, so a large FlowRtoL must push F below 1/2 and a large
    # FlowLtoR above it.
    h, w = 4, 8
    L = np.zeros((h, w))
    R = np.ones((h, w))
    B = np.full((h, w), 0.5)
    big = np.zeros((h, w, 2))
    big[..., 1] = 3.0          # vertical, so the samples stay on the constant images
    z = np.zeros((h, w, 2))
    assert np.all(oracle.blend(L, R, z, big, P_BLEND, B) < 0.5)
    assert np.all(oracle.blend(L, R, big, z, P_BLEND, B) > 0.5)
    np.testing.assert_allclose(oracle.blend(L, R, z, z, P_BLEND, B), 0.5, rtol=0, atol=1e-15)


def test_quantize_u8_rounds_half_to_even_and_clamps():
    F = np.array([0.5, 1.5, 2.5, 3.49, 254.5, 256.0, -3.0]) / 255.0
    np.testing.assert_array_equal(oracle.quantize_u8(F), [0, 2, 2, 3, 254, 255, 0])


def test_stitch_pair_u8_path_shapes():
    p = synth.pair_translation(1.0, 0.5, h=32, w=48, levels=2, dtype="u8", channels=3)
    lr, rl, F = oracle.stitch_pair(p.L, p.R, oracle.Params(levels=2))
    assert F.dtype == np.uint8 and F.shape == p.L.shape
    assert lr.shape == rl.shape == (32, 48, 2)
