"""Pins of the oracle's refinement energy, its gradients and the REDUCE
transpose: central finite differences, a closed form, a vanishing case and
the dot-product identity of an adjoint."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def _setup(seed=0, h=12, w=15):
    g = np.random.default_rng(seed)
    T = ndimage.gaussian_filter(g.uniform(0, 1, (h, w)), 1.0)
    J = ndimage.gaussian_filter(g.uniform(0, 1, (h, w)), 1.0)
    # flows whose sample positions keep at least 0.1 px from the grid lines,
    # where the bilinear interpolant has kinks
    whole = g.integers(-2, 3, size=(h, w, 2)).astype(np.float64)
    frac = g.uniform(0.1, 0.9, size=(h, w, 2))
    return T, J, whole + frac, g


@pytest.mark.parametrize("alpha", [0.0, 0.05, 0.7])
def test_energy_gradient_in_u_matches_central_differences(alpha):
    T, J, u, g = _setup()
    gu, _, _ = oracle.energy_grad(T, J, u, alpha)
    h = 1e-6
    for _ in range(40):
        y, x, c = g.integers(0, 12), g.integers(0, 15), g.integers(0, 2)
        e = np.zeros_like(u)
        e[y, x, c] = 1.0
        fd = (oracle.energy(T, J, u + h * e, alpha) - oracle.energy(T, J, u - h * e, alpha)) / (2 * h)
        assert abs(fd - gu[y, x, c]) <= 1e-6 * max(1.0, abs(fd))


def test_energy_gradients_in_T_and_J_match_central_differences():
    # E is quadratic in T and J, so central differences are exact up to rounding
    T, J, u, g = _setup(1)
    _, gt, gj = oracle.energy_grad(T, J, u, 0.1)
    h = 1e-4
    for _ in range(30):
        y, x = g.integers(0, 12), g.integers(0, 15)
        e = np.zeros_like(T)
        e[y, x] = 1.0
        fdT = (oracle.energy(T + h * e, J, u, 0.1) - oracle.energy(T - h * e, J, u, 0.1)) / (2 * h)
        fdJ = (oracle.energy(T, J + h * e, u, 0.1) - oracle.energy(T, J - h * e, u, 0.1)) / (2 * h)
        assert abs(fdT - gt[y, x]) <= 1e-8
        assert abs(fdJ - gj[y, x]) <= 1e-8


def test_smoothness_energy_closed_form():
    # constant images: the data term vanishes for any flow; a linear flow
    # u_x = a x + b y has (w-1) h horizontal and w (h-1) vertical differences
    h, w, a, b, alpha = 7, 9, 0.3, -0.2, 0.25
    T = np.full((h, w), 0.4)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    u = np.stack([a * xs + b * ys, np.zeros((h, w))], -1)
    expect = alpha * (a * a * (w - 1) * h + b * b * w * (h - 1))
    assert oracle.energy(T, T, u, alpha) == pytest.approx(expect, rel=1e-12)


def test_energy_and_gradients_vanish_on_identical_images_and_zero_flow():
    T, _, _, _ = _setup(2)
    z = np.zeros(T.shape + (2,))
    assert oracle.energy(T, T, z, 0.3) == 0.0
    gu, gt, gj = oracle.energy_grad(T, T, z, 0.3)
    assert not gu.any() and not gt.any() and not gj.any()


@pytest.mark.parametrize("shape", [(7, 9), (8, 8), (1, 5), (13, 2), (33, 40)])
def test_reduce_transpose_dot_product_identity(shape):
    g = np.random.default_rng(3)
    x = g.normal(size=shape)
    y = g.normal(size=((shape[0] + 1) // 2, (shape[1] + 1) // 2))
    lhs = float((oracle.pyr_down(x) * y).sum())
    rhs = float((x * oracle.pyr_down_adjoint(y, *shape)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)
