"""16-bit pyramid storage (pano_flow_params.pyr_dtype = PANO_BF16 / PANO_F16)
against the oracle with the same storage rounding, and against the exact
FP64 oracle and the float32 GPU path.

Parity bar: the GPU rounds levels it computed in FP32, the oracle levels it
computed in FP64, so a value within FP32 rounding of a tie between two
16-bit neighbours can land one storage ulp apart (rare); flows therefore
match the storage-matched oracle to a mean endpoint error of 1e-3 px, and
the blended u8 strips to 1 LSB. Against the exact oracle the storage itself
costs accuracy: binary16 keeps 11 significand bits (luma steps of 2^-12 near
1), bfloat16 8 (2^-9), which on these pairs moves flows by up to about
0.005 px (binary16) and 0.05 px (bfloat16) on average; the bounds below are
twice that."""
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

DEV = torch.device("cuda:0")
FORMATS = [(binding.PANO_BF16, oracle.FMT_BF16), (binding.PANO_F16, oracle.FMT_F16)]
EXACT_BOUND = {binding.PANO_BF16: 0.1, binding.PANO_F16: 0.01}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def epe(a, b):
    return np.hypot(*(a - b).transpose(2, 0, 1))


def gpu_stitch(pair, levels, pyr_dtype):
    h, w = pair.L.shape[:2]
    c = pair.L.shape[2] if pair.L.ndim == 3 else 1
    with binding.FlowContext(binding.Params(levels=levels, pyr_dtype=pyr_dtype), h, w, c) as ctx:
        lr, rl, F = ctx.stitch_pair(cuda(pair.L), cuda(pair.R))
        torch.cuda.synchronize()
        return lr.cpu().numpy(), rl.cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("dt,fmt", FORMATS)
@pytest.mark.parametrize("kind", ["gray_f32", "rgb_u8"])
def test_half_pyramids_match_storage_matched_oracle(dt, fmt, kind):
    if kind == "gray_f32":
        pair, levels = synth.pair_small_gray(), 4
    else:
        # without the colour gain: flows that follow the scene, so the
        # comparison measures storage error, not the divergence an
        # uncorrected gain can cause
        pair, levels = synth.pair_fullres_rgb(seed=3, h=480, w=360, dmax=8.0, levels=4, gain_range=None), 4
    lr, rl, F = gpu_stitch(pair, levels, dt)
    olr, orl = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=levels, pyr_fmt=fmt))
    for g, o in ((lr, olr), (rl, orl)):
        e = epe(g, o)
        assert e.mean() <= 1e-3, e.mean()
    Fo = oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=levels))
    if pair.L.dtype == np.uint8:
        d = np.abs(F.astype(int) - oracle.quantize_u8(Fo).astype(int))
        assert np.percentile(d, 99.9) <= 1
    else:
        d = np.abs(F - Fo)
        assert np.percentile(d, 99.9) <= 1.0 / 255
    # against the exact oracle: the cost of the storage format
    xlr, xrl = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=levels))
    assert epe(lr, xlr).mean() <= EXACT_BOUND[dt] and epe(rl, xrl).mean() <= EXACT_BOUND[dt]


@pytest.mark.parametrize("dt", [binding.PANO_BF16, binding.PANO_F16])
def test_half_identical_strips_give_zero_flow_and_swap_is_exact(dt):
    pair = synth.pair_fullres_rgb(seed=4, h=256, w=200, dmax=6.0, levels=3)
    with binding.FlowContext(binding.Params(levels=3, pyr_dtype=dt), 256, 200, 3) as ctx:
        L, R = cuda(pair.L), cuda(pair.R)
        z1, z2 = ctx.flow_pair(L, L)
        lr, rl = ctx.flow_pair(L, R)
        rl2, lr2 = ctx.flow_pair(R, L)
        torch.cuda.synchronize()
        assert torch.count_nonzero(z1) == 0 and torch.count_nonzero(z2) == 0
        assert torch.equal(lr, lr2) and torch.equal(rl, rl2)


def test_half_rig_equals_half_single_pair_path():
    widths = (240, 300)
    pairs = [synth.pair_fullres_rgb(seed=60 + k, h=400, w=w, dmax=6.0, levels=4) for k, w in enumerate(widths)]
    prm = binding.Params(levels=4, pyr_dtype=binding.PANO_BF16)
    with binding.FlowContext(prm, 400, 300, 3) as ctx:
        ref = [ctx.flow_pair(cuda(p.L), cuda(p.R)) for p in pairs]
        torch.cuda.synchronize()
    with binding.Rig(prm, 400, widths, canvas_hw=(400, 600), canvas_x0=(0, 300)) as rig:
        rig.run([cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs], use_graph=True)
        torch.cuda.synchronize()
        for k in range(2):
            a, b = rig.flows(k)
            assert torch.equal(a, ref[k][0]) and torch.equal(b, ref[k][1])


def test_half_differs_from_float_only_by_storage_rounding():
    pair = synth.pair_fullres_rgb(seed=5, h=600, w=400, dmax=8.0, levels=4, gain_range=None)
    f32 = gpu_stitch(pair, 4, binding.PANO_F32)
    for dt, bound in ((binding.PANO_F16, EXACT_BOUND[binding.PANO_F16]), (binding.PANO_BF16, EXACT_BOUND[binding.PANO_BF16])):
        half = gpu_stitch(pair, 4, dt)
        assert 0 < epe(half[0], f32[0]).mean() <= bound
        assert 0 < epe(half[1], f32[1]).mean() <= bound


@pytest.mark.slow
def test_half_rig_full_size_matches_storage_matched_oracle():
    """The 8-pair, 4000-row rig with 16-bit pyramids (the bench's half-precision
    rig) against the oracle with the same storage rounding, pair by pair. On
    the pairs whose flows follow the scene (the exact oracle's FlowRtoL within
    5 px of the generator's field) the mean EPE stays below 1e-3 px. On the
    pairs where the uncorrected colour gain sends the iteration off (10-23 px
    from the field), rare one-ulp differences between the GPU's and the
    oracle's stored levels are amplified; those stay below 1e-2 px."""
    widths = (800, 950, 1100, 1250, 1400, 1600, 1800, 2000)
    pairs = synth.rig_pairs(widths=widths, workers=8)
    levels = 6
    exact = [oracle.flow_pair(p.L, p.R, oracle.Params(levels=levels)) for p in pairs]
    follows = [epe(exact[k][1], p.flow_RtoL).mean() <= 5.0 for k, p in enumerate(pairs)]
    assert sum(follows) >= 4
    for dt, fmt in FORMATS:
        prm = binding.Params(levels=levels, pyr_dtype=dt)
        with binding.Rig(prm, 4000, widths, canvas_hw=(4000, 9000), canvas_x0=[1125 * k for k in range(8)]) as rig:
            rig.run([cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs], use_graph=True)
            torch.cuda.synchronize()
            got = [tuple(t.cpu().numpy() for t in rig.flows(k)) for k in range(len(pairs))]
        for k, p in enumerate(pairs):
            slr, srl = oracle.flow_pair(p.L, p.R, oracle.Params(levels=levels, pyr_fmt=fmt))
            worst = max(epe(got[k][0], slr).mean(), epe(got[k][1], srl).mean())
            assert worst <= (1e-3 if follows[k] else 1e-2), (dt, k, worst)
