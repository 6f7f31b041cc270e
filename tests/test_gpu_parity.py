"""GPU path against the FP64 oracle, through the C ABI.

Stage tests feed the GPU and the oracle the same inputs. Tolerances:
  * pyramid, luma, upsampling, warp: FP32 rounding of a handful of
    operations on values in [0, 1] -> max-abs 1e-5;
  * one LK step: max-abs 1e-4 px;
  * Code 1 blend on identical flows: f32 max-abs 1e-5, u8 within 1 LSB
    (a value within FP32 rounding of a .5 tie may round either way);
  * end to end: mean endpoint error <= 0.05 px per direction, and every
    pixel of F within 1/255 of the oracle's whole path (u8: one level).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_01201_gb300 import binding  # noqa: E402
from paper_2006_01201_gb300 import build as gpu_build  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rng(s):
    return np.random.default_rng(s)


def texture(h, w, seed):
    from scipy import ndimage
    return ndimage.gaussian_filter(rng(seed).uniform(0, 1, size=(h, w)), 1.2)


def epe(a, b):
    return np.hypot(*(a - b).transpose(2, 0, 1))


# ---------------------------------------------------------------- luma, pyramid

@pytest.mark.parametrize("shape,dtype", [((37, 53, 3), np.uint8), ((64, 96, 1), np.uint8),
                                         ((17, 33, 3), np.float32), ((5, 7), np.float32)])
def test_luma_matches_oracle(shape, dtype):
    g = rng(1)
    a = (g.integers(0, 256, size=shape).astype(np.uint8) if dtype == np.uint8
         else g.uniform(0, 1, size=shape).astype(np.float32))
    if len(shape) == 3 and shape[2] == 1:
        a = a[..., 0]
    Y = host(binding.stage_luma(cuda(a)))
    ref = oracle.luma(oracle.to_unit(a))
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-6)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (2, 2), (5, 7), (37, 53), (131, 67), (256, 512)])
def test_pyr_down_matches_oracle(shape):
    src = rng(2).uniform(0, 1, size=shape).astype(np.float32)
    out = host(binding.stage_pyr_down(cuda(src)))
    np.testing.assert_allclose(out, oracle.pyr_down(src), rtol=0, atol=1e-6)


@pytest.mark.parametrize("shape,dtype", [((37, 53, 3), np.uint8), ((64, 96, 1), np.uint8), ((130, 260, 3), np.uint8),
                                         ((35, 131, 3), np.float32), ((1, 1, 3), np.uint8), ((2, 300, 1), np.float32)])
def test_fused_luma_and_reduce_equal_the_separate_kernels_and_the_oracle(shape, dtype):
    g = rng(31)
    img = g.integers(0, 256, size=shape).astype(np.uint8) if dtype == np.uint8 else \
        g.uniform(0, 1, size=shape).astype(np.float32)
    t = cuda(img if shape[2] == 3 else img[..., 0])
    Y, Y1 = binding.stage_luma_pyr(t)
    Ys = binding.stage_luma(t)
    Y1s = binding.stage_pyr_down(Ys)
    torch.cuda.synchronize()
    assert torch.equal(Y, Ys) and torch.equal(Y1, Y1s)
    Yo = oracle.luma(oracle.to_unit(img if shape[2] == 3 else img[..., 0]))
    np.testing.assert_allclose(host(Y), Yo, rtol=0, atol=1e-6)
    np.testing.assert_allclose(host(Y1), oracle.pyr_down(Yo), rtol=0, atol=1e-6)


@pytest.mark.parametrize("shape,nlev", [((300, 200), 6), ((37, 53), 5), ((1, 1), 4), ((130, 17), 7), ((64, 64), 3),
                                        ((2000, 750), 6)])
def test_multi_level_reduce_equals_one_level_steps_and_the_oracle(shape, nlev):
    Y = cuda(rng(33).uniform(0, 1, size=shape).astype(np.float32))
    got = binding.stage_pyramid(Y, nlev)
    ref = [Y]
    for _ in range(nlev - 1):
        ref.append(binding.stage_pyr_down(ref[-1]))
    torch.cuda.synchronize()
    for l, (a, b) in enumerate(zip(got, ref[1:]), start=1):
        assert torch.equal(a, b), l
    if shape[0] * shape[1] <= 100000:
        for a, o in zip(got, oracle.pyramid(host(Y), nlev)[1:]):
            np.testing.assert_allclose(host(a), o, rtol=0, atol=1e-6)


def test_pyr_down_respects_row_pitch():
    big = rng(3).uniform(0, 1, size=(40, 64)).astype(np.float32)
    view = cuda(big)[:, :45]                      # rows of 64 elements, 45 used
    out = host(binding.stage_pyr_down(view))
    np.testing.assert_allclose(out, oracle.pyr_down(big[:, :45]), rtol=0, atol=1e-6)


# ---------------------------------------------------------------- LK stage

@pytest.mark.parametrize("h,w,radius", [(100, 150, 2), (37, 61, 1), (64, 64, 3), (9, 11, 2)])
def test_one_lk_step_matches_oracle(h, w, radius):
    T = texture(h, w, 4)
    J = texture(h, w, 5) * 0.3 + T * 0.7
    u = np.stack([1.5 * np.sin(np.arange(w) / 9.0)[None, :].repeat(h, 0),
                  0.7 * np.cos(np.arange(h) / 7.0)[:, None].repeat(w, 1)], -1)
    u = u + rng(6).normal(0, 0.2, size=u.shape)
    lam = 1e-2
    got = host(binding.stage_lk(cuda(T.astype(np.float32)), cuda(J.astype(np.float32)),
                                cuda(u.astype(np.float32)), upsample=False, iters=1, radius=radius, lam=lam))
    ref = oracle.lk_step(T.astype(np.float32), J.astype(np.float32), u.astype(np.float32), radius, lam)
    assert np.abs(got - ref).max() <= 1e-4


def test_lk_steps_at_one_level_match_oracle():
    h, w = 90, 140
    T = texture(h, w, 7).astype(np.float32)
    J = np.roll(T, (1, -2), axis=(0, 1)).astype(np.float32)
    u0 = np.zeros((h, w, 2), dtype=np.float32)
    got = host(binding.stage_lk(cuda(T), cuda(J), cuda(u0), iters=5, radius=2, lam=1e-2))
    ref = u0.astype(np.float64)
    for _ in range(5):
        ref = oracle.lk_step(T, J, ref, 2, 1e-2)
    assert np.abs(got - ref).max() <= 1e-3
    assert epe(got, ref).mean() <= 1e-5


@pytest.mark.parametrize("kernel", [binding.PANO_LK_AUTO, binding.PANO_LK_STREAM, binding.PANO_LK_TILE])
@pytest.mark.parametrize("h,w,iters,radius,start", [(230, 317, 5, 2, "coarse"), (121, 203, 3, 1, "given"),
                                                    (64, 96, 4, 3, "zero"), (3, 5, 5, 2, "coarse")])
def test_each_lk_kernel_matches_oracle(kernel, h, w, iters, radius, start):
    # several bands, segments and tiles with ragged edges; each kernel
    # selected through pano_stage_lk_kernel
    T = texture(h, w, 11).astype(np.float32)
    J = (0.8 * np.roll(T, (1, -2), axis=(0, 1)) + 0.2 * texture(h, w, 12)).astype(np.float32)
    g = rng(13)
    if start == "coarse":
        uin = g.normal(0, 1.0, size=((h + 1) // 2, (w + 1) // 2, 2)).astype(np.float32)
        ref = oracle.upsample_flow(uin, h, w)
    elif start == "given":
        uin = g.normal(0, 1.5, size=(h, w, 2)).astype(np.float32)
        ref = uin.astype(np.float64)
    else:
        uin, ref = None, np.zeros((h, w, 2))
    for _ in range(iters):
        ref = oracle.lk_step(T, J, ref, radius, 1e-2)
    got = host(binding.stage_lk(cuda(T), cuda(J), None if uin is None else cuda(uin), upsample=start == "coarse",
                                iters=iters, radius=radius, lam=1e-2, kernel=kernel))
    assert np.isfinite(got).all()
    assert epe(got, ref).mean() <= 1e-5
    assert np.abs(got - ref).max() <= 1e-3


@pytest.mark.parametrize("kernel", [binding.PANO_LK_AUTO, binding.PANO_LK_TILE])
@pytest.mark.parametrize("h,w,iters,radius,start", [(70, 90, 8, 2, "zero"), (40, 60, 16, 1, "given")])
def test_lk_kernels_beyond_five_steps_match_oracle(kernel, h, w, iters, radius, start):
    # more steps than the streamed kernel takes (up to the API's maximum of 16):
    # AUTO falls back to the tiled kernel
    T = texture(h, w, 21).astype(np.float32)
    J = np.roll(T, (0, 1), axis=(0, 1)).astype(np.float32)
    uin = rng(22).normal(0, 0.5, size=(h, w, 2)).astype(np.float32) if start == "given" else None
    ref = uin.astype(np.float64) if uin is not None else np.zeros((h, w, 2))
    for _ in range(iters):
        ref = oracle.lk_step(T, J, ref, radius, 1e-2)
    got = host(binding.stage_lk(cuda(T), cuda(J), None if uin is None else cuda(uin), iters=iters, radius=radius,
                                lam=1e-2, kernel=kernel))
    assert np.isfinite(got).all()
    assert epe(got, ref).mean() <= 1e-5
    assert np.abs(got - ref).max() <= 1e-3


def test_streamed_kernel_refuses_more_than_five_steps():
    T = texture(64, 64, 23).astype(np.float32)
    with pytest.raises(binding.PanoError) as ei:
        binding.stage_lk(cuda(T), cuda(T), None, iters=6, kernel=binding.PANO_LK_STREAM)
    assert ei.value.status == binding.PANO_ERR_UNSUPPORTED


def test_upsample_stage_matches_oracle():
    hc, wc, h, w = 23, 37, 45, 73
    uc = rng(8).normal(0, 2, size=(hc, wc, 2)).astype(np.float32)
    T = np.zeros((h, w), np.float32)
    got = host(binding.stage_lk(cuda(T), cuda(T), cuda(uc), upsample=True, iters=0))
    np.testing.assert_allclose(got, oracle.upsample_flow(uc, h, w), rtol=0, atol=1e-5)


def test_zero_start_identical_images_gives_zero():
    T = texture(50, 70, 9).astype(np.float32)
    got = host(binding.stage_lk(cuda(T), cuda(T), None, iters=5))
    assert np.all(got == 0.0)


# ---------------------------------------------------------------- warp, blend

@pytest.mark.parametrize("shape,dtype,scale", [((33, 65, 3), np.uint8, 0.3), ((40, 50), np.float32, 1.0),
                                               ((16, 24, 3), np.float32, -0.5)])
def test_warp_matches_oracle(shape, dtype, scale):
    g = rng(10)
    a = (g.integers(0, 256, size=shape).astype(np.uint8) if dtype == np.uint8
         else g.uniform(0, 1, size=shape).astype(np.float32))
    flow = g.normal(0, 4, size=shape[:2] + (2,)).astype(np.float32)
    got = host(binding.stage_warp(cuda(a), cuda(flow), scale))
    ref = oracle.warp(oracle.to_unit(a), flow, scale)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5)


def _ctx(levels, h, w, c):
    return binding.FlowContext(binding.Params(levels=levels), max_h=h, max_w=w, max_c=c)


@pytest.mark.parametrize("shape,dtype", [((31, 47, 3), np.uint8), ((64, 100), np.float32),
                                         ((20, 33, 3), np.float32)])
def test_blend_matches_oracle_on_same_flows(shape, dtype):
    g = rng(11)
    L = (g.integers(0, 256, size=shape).astype(np.uint8) if dtype == np.uint8
         else g.uniform(0, 1, size=shape).astype(np.float32))
    R = (g.integers(0, 256, size=shape).astype(np.uint8) if dtype == np.uint8
         else g.uniform(0, 1, size=shape).astype(np.float32))
    lr = g.normal(0, 3, size=shape[:2] + (2,)).astype(np.float32)
    rl = g.normal(0, 3, size=shape[:2] + (2,)).astype(np.float32)
    with _ctx(2, shape[0], shape[1], 3) as ctx:
        F = host(ctx.blend_pair(cuda(L), cuda(R), cuda(lr), cuda(rl)))
        B = g.uniform(0, 1, size=shape[:2]).astype(np.float32)
        FB = host(ctx.blend_pair(cuda(L), cuda(R), cuda(lr), cuda(rl), blend=cuda(B)))
    P = oracle.Params()
    ref = oracle.blend(L, R, lr, rl, P)
    refB = oracle.blend(L, R, lr, rl, P, B)
    if dtype == np.uint8:
        assert np.abs(F.astype(int) - oracle.quantize_u8(ref).astype(int)).max() <= 1
        assert np.abs(FB.astype(int) - oracle.quantize_u8(refB).astype(int)).max() <= 1
    else:
        np.testing.assert_allclose(F, ref, rtol=0, atol=1e-5)
        np.testing.assert_allclose(FB, refB, rtol=0, atol=1e-5)


def test_blend_identical_strips_zero_flow_is_identity_u8():
    L = rng(12).integers(0, 256, size=(40, 60, 3)).astype(np.uint8)
    z = np.zeros((40, 60, 2), np.float32)
    with _ctx(2, 40, 60, 3) as ctx:
        F = host(ctx.blend_pair(cuda(L), cuda(L), cuda(z), cuda(z)))
    np.testing.assert_array_equal(F, L)


# ---------------------------------------------------------------- whole path

def _e2e(pair, check_blend_u8=True):
    h, w = pair.shape
    c = pair.channels
    P = oracle.Params(levels=pair.levels)
    with _ctx(pair.levels, h, w, c) as ctx:
        lr, rl, F = ctx.stitch_pair(cuda(pair.L), cuda(pair.R))
        lr, rl, F = host(lr), host(rl), host(F)
    olr, orl = oracle.flow_pair(pair.L, pair.R, P)
    e_lr, e_rl = epe(lr, olr), epe(rl, orl)
    assert e_lr.mean() <= 0.05 and e_rl.mean() <= 0.05, (e_lr.mean(), e_rl.mean())
    # Code 1 on the GPU flows: the blend stage alone
    Fo = oracle.blend(pair.L, pair.R, lr, rl, P)
    if pair.L.dtype == np.uint8:
        assert np.abs(F.astype(int) - oracle.quantize_u8(Fo).astype(int)).max() <= 1
    else:
        assert np.abs(F - Fo).max() <= 1e-5
    # the whole path against the whole oracle path (its own flows, then Code 1):
    # every blended pixel within 1/255 (u8: one level)
    Fw = oracle.blend(pair.L, pair.R, olr, orl, P)
    if pair.L.dtype == np.uint8:
        assert np.abs(F.astype(int) - oracle.quantize_u8(Fw).astype(int)).max() <= 1
    else:
        assert np.abs(F - Fw).max() <= 1.0 / 255
    return e_lr, e_rl, F, olr, orl


def test_end_to_end_small_gray_pair():
    pair = synth.pair_small_gray()
    e_lr, e_rl, F, olr, orl = _e2e(pair)
    # whole path against the whole oracle path: flows and F
    Fo = oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=pair.levels))
    d = np.abs(F - Fo)
    assert d.mean() <= 1e-4 and d.max() <= 1.0 / 255


@pytest.mark.parametrize("h,w,c,levels", [(1, 1, 1, 1), (2, 3, 3, 3), (5, 7, 1, 4), (33, 65, 3, 3),
                                          (70, 45, 1, 5), (16, 300, 3, 2), (100, 150, 3, 12)])
def test_end_to_end_edge_sizes(h, w, c, levels):
    g = rng(13)
    base = texture(h + 8, w + 8, 14)
    L = base[4:4 + h, 4:4 + w]
    R = base[5:5 + h, 3:3 + w]
    if c == 3:
        L = np.stack([L, L * 0.9, L * 0.8], -1)
        R = np.stack([R, R * 0.9, R * 0.8], -1)
    L8 = np.clip(np.rint(L * 255), 0, 255).astype(np.uint8)
    R8 = np.clip(np.rint(R * 255), 0, 255).astype(np.uint8)

    class P:
        pass
    pair = P()
    pair.L, pair.R, pair.levels, pair.shape, pair.channels = L8, R8, levels, (h, w), c
    _e2e(pair)


def test_flow_pair_swap_is_bit_exact_and_repeatable():
    pair = synth.pair_small_gray(h=128, w=200, levels=3)
    with _ctx(3, 128, 200, 1) as ctx:
        lr, rl = ctx.flow_pair(cuda(pair.L), cuda(pair.R))
        rl2, lr2 = ctx.flow_pair(cuda(pair.R), cuda(pair.L))
        lr3, rl3 = ctx.flow_pair(cuda(pair.L), cuda(pair.R))
        torch.cuda.synchronize()
        assert torch.equal(lr, lr2) and torch.equal(rl, rl2)
        assert torch.equal(lr, lr3) and torch.equal(rl, rl3)


def test_identical_strips_zero_flow_and_identity_blend():
    pair = synth.pair_fullres_rgb(h=256, w=384, levels=4)
    with _ctx(4, 256, 384, 3) as ctx:
        L = cuda(pair.L)
        lr, rl, F = ctx.stitch_pair(L, L)
        torch.cuda.synchronize()
        assert torch.count_nonzero(lr) == 0 and torch.count_nonzero(rl) == 0
        assert torch.equal(F, L)


def test_strided_input_rows():
    pair = synth.pair_small_gray(h=96, w=128, levels=3)
    padL = np.zeros((96, 160), np.float32)
    padR = np.zeros((96, 160), np.float32)
    padL[:, :128], padR[:, :128] = pair.L, pair.R
    with _ctx(3, 96, 128, 1) as ctx:
        a = ctx.flow_pair(cuda(pair.L), cuda(pair.R))
        b = ctx.flow_pair(cuda(padL)[:, :128], cuda(padR)[:, :128])
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_bad_arguments_raise():
    with _ctx(3, 64, 64, 1) as ctx:
        big = torch.zeros((65, 64), dtype=torch.float32, device=DEV)
        with pytest.raises(binding.PanoError) as ei:
            ctx.flow_pair(big, big)
        assert ei.value.status == binding.PANO_ERR_INVALID_ARG
        a = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
        b = torch.zeros((32, 31), dtype=torch.float32, device=DEV)
        with pytest.raises(binding.PanoError):
            ctx.flow_pair(a, b)


@pytest.mark.slow
def test_full_size_rgb_pair_matches_oracle():
    """4000x1500 RGB u8, 6 levels: the benchmark's workload and launch
    configuration, compared in full (the oracle runs it in seconds)."""
    pair = synth.pair_fullres_rgb()
    e_lr, e_rl, F, olr, orl = _e2e(pair)
    Fo = oracle.quantize_u8(oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=6)))
    d = np.abs(F.astype(int) - Fo.astype(int))
    assert d.mean() <= 0.05 and d.max() <= 1


@pytest.mark.slow
def test_large_strip_properties():
    """An 8000 x 12000 RGB u8 pair (288 MB per strip, 32-bit offsets near a
    quarter of their range), too large for the oracle: properties that hold
    at any size. Identical strips give zero flow exactly and F = L; an
    integer translation is recovered in the interior; swapping the strips
    swaps the flows bit for bit."""
    h, w = 8000, 12000
    gen = torch.Generator(device=DEV).manual_seed(5)
    noise = torch.rand((3, 1, h + 16, w + 16), generator=gen, device=DEV)
    k = torch.ones((1, 1, 5, 5), device=DEV) / 25.0
    tex = torch.nn.functional.conv2d(noise, k)                    # (3, 1, h + 12, w + 12), smooth
    tex = (tex - tex.amin()) / (tex.amax() - tex.amin())
    img = (tex[:, 0] * 255).round().to(torch.uint8).permute(1, 2, 0).contiguous()   # (h + 12, w + 12, 3)
    L = img[6:6 + h, 6:6 + w].contiguous()
    R = img[4:4 + h, 9:9 + w].contiguous()                       # R(p) = L(p + (3, -2))
    with _ctx(6, h, w, 3) as ctx:
        z1, z2, F = ctx.stitch_pair(L, L)
        torch.cuda.synchronize()
        assert torch.count_nonzero(z1) == 0 and torch.count_nonzero(z2) == 0
        assert torch.equal(F, L)
        del z1, z2, F
        lr, rl = ctx.flow_pair(L, R)
        rl2, lr2 = ctx.flow_pair(R, L)
        torch.cuda.synchronize()
        assert torch.equal(lr, lr2) and torch.equal(rl, rl2)
        m = 64
        mean_rl = rl[m:-m, m:-m].reshape(-1, 2).mean(0).cpu().numpy()
        mean_lr = lr[m:-m, m:-m].reshape(-1, 2).mean(0).cpu().numpy()
        np.testing.assert_allclose(mean_rl, [3.0, -2.0], atol=0.1)     # FlowRtoL: R(p) = L(p + (3, -2))
        np.testing.assert_allclose(mean_lr, [-3.0, 2.0], atol=0.1)
