"""Differentiable refinement on the GPU against the FP64 oracle: energy and
gradients on a 64x64 crop of the 1024x1024 pair, central finite differences
of the GPU's FP64 energy, the REDUCE transpose, gradients through pyramid
levels, and refinement by gradient steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_01201_gb300 import binding  # noqa: E402
from paper_2006_01201_gb300 import build as gpu_build  # noqa: E402
from paper_2006_01201_gb300 import refine  # noqa: E402

DEV = torch.device("cuda:0")
ALPHA = 0.05


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


@pytest.fixture(scope="module")
def pair1024():
    return synth.pair_small_gray(seed=3, h=1024, w=1024, amp_x=6.0, amp_y=3.0, levels=5)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def crop(pair, y0=480, x0=480, n=64):
    T = pair.L[y0:y0 + n, x0:x0 + n].astype(np.float32)
    J = pair.R[y0:y0 + n, x0:x0 + n].astype(np.float32)
    u = pair.flow_LtoR[y0:y0 + n, x0:x0 + n].astype(np.float32)
    u = u + np.random.default_rng(4).normal(0, 0.3, u.shape).astype(np.float32)
    return T, J, u


def test_energy_and_gradients_match_oracle_on_crop(pair1024):
    T, J, u = crop(pair1024)
    E, gu, gt, gj = binding.energy_grad(cuda(T), cuda(J), cuda(u), ALPHA)
    torch.cuda.synchronize()
    Eo = oracle.energy(T, J, u, ALPHA)
    guo, gto, gjo = oracle.energy_grad(T, J, u, ALPHA)
    assert float(E) == pytest.approx(Eo, rel=1e-5)
    for got, ref in ((gu, guo), (gt, gto), (gj, gjo)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_gpu_gradient_matches_central_differences(pair1024):
    T, J, u = crop(pair1024)
    Tt, Jt, ut = cuda(T), cuda(J), cuda(u)
    _, gu, _, _ = binding.energy_grad(Tt, Jt, ut, ALPHA)
    g = np.random.default_rng(5)
    h = 1e-3
    for trial in range(6):
        # every coordinate moves by h (random signs): smaller per-pixel steps
        # would drown in the FP32 rounding of the residuals
        d = g.choice([-1.0, 1.0], size=u.shape).astype(np.float32)
        if trial >= 3:                      # single coordinates as well
            d = np.zeros_like(u)
            d[g.integers(0, 64), g.integers(0, 64), g.integers(0, 2)] = 1.0
        dt = cuda(d)
        Ep = float(binding.energy_grad(Tt, Jt, ut + h * dt, ALPHA, want_u=False, want_T=False, want_J=False)[0])
        Em = float(binding.energy_grad(Tt, Jt, ut - h * dt, ALPHA, want_u=False, want_T=False, want_J=False)[0])
        fd = (Ep - Em) / (2 * h)
        an = float((gu.double() * dt.double()).sum())
        assert abs(fd - an) <= 2e-3 * max(abs(an), 1e-2), (trial, fd, an)


@pytest.mark.parametrize("shape", [(37, 53), (64, 64), (5, 2), (1, 9)])
def test_reduce_transpose_on_gpu(shape):
    g = np.random.default_rng(6)
    x = g.normal(size=shape).astype(np.float32)
    y = g.normal(size=((shape[0] + 1) // 2, (shape[1] + 1) // 2)).astype(np.float32)
    Ax = binding.stage_pyr_down(cuda(x)).cpu().numpy().astype(np.float64)
    ATy = binding.stage_pyr_down_adjoint(cuda(y), *shape).cpu().numpy().astype(np.float64)
    lhs, rhs = float((Ax * y).sum()), float((x * ATy).sum())
    assert lhs == pytest.approx(rhs, rel=1e-5, abs=1e-5)
    np.testing.assert_allclose(ATy, oracle.pyr_down_adjoint(y, *shape), rtol=0, atol=1e-6)


def test_pyramid_energy_gradients_through_levels():
    p = synth.pair_small_gray(seed=7, h=96, w=128, amp_x=2.0, amp_y=1.0, levels=3)
    level = 2
    T0, J0 = cuda(p.L), cuda(p.R)
    pyrT = oracle.pyramid(p.L, level + 1)
    pyrJ = oracle.pyramid(p.R, level + 1)
    hl, wl = pyrT[level].shape
    u = np.random.default_rng(8).normal(0, 0.4, (hl, wl, 2)).astype(np.float32)
    T0.requires_grad_(True)
    J0.requires_grad_(True)
    ut = cuda(u).requires_grad_(True)
    E = refine.pyramid_energy(T0, J0, ut, level, ALPHA)
    E.backward()
    Eo = oracle.energy(pyrT[level], pyrJ[level], u, ALPHA)
    guo, gto, gjo = oracle.energy_grad(pyrT[level], pyrJ[level], u, ALPHA)
    shapes = [x.shape for x in pyrT]
    for l in range(level, 0, -1):
        gto = oracle.pyr_down_adjoint(gto, *shapes[l - 1])
        gjo = oracle.pyr_down_adjoint(gjo, *shapes[l - 1])
    assert float(E.detach()) == pytest.approx(Eo, rel=1e-5)
    for got, ref in ((ut.grad, guo), (T0.grad, gto), (J0.grad, gjo)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


def test_refinement_lowers_energy_and_recovers_flow():
    p = synth.pair_small_gray(seed=9, h=256, w=256, amp_x=3.0, amp_y=1.5, levels=3)
    u, trace = refine.refine_flow(cuda(p.L), cuda(p.R), levels=3, steps=40, lr=0.05, alpha=ALPHA)
    torch.cuda.synchronize()
    for level, first, last in trace:
        assert last < first, (level, first, last)
    m = 12
    err = np.hypot(*(u.cpu().numpy() - p.flow_LtoR).transpose(2, 0, 1))[m:-m, m:-m]
    zero = np.hypot(*p.flow_LtoR.transpose(2, 0, 1))[m:-m, m:-m]
    assert err.mean() < 0.35 * zero.mean(), (err.mean(), zero.mean())
