"""Code 1 on a whole canvas (pano_compose_pair) against the FP64 oracle,
through the C ABI.

Tolerances: Area1 / Area2 / neither pixels are copies and zeros, so they
must be exact; Area3 pixels carry the blend's tolerances (float32 output
max-abs 1e-5 on [0, 1] values, uint8 output within 1 LSB: a value within
FP32 rounding of a .5 tie may round either way).
"""
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _labels(h, w, seed):
    """Area1 left, Area2 right, a wavy Area3 band between them, a top row and
    one pixel that belong to neither."""
    g = np.random.default_rng(seed)
    ys = np.arange(h)[:, None]
    xs = np.arange(w)[None, :]
    a = (w // 4 + 3 * np.sin(ys / 7.0)).astype(int)
    b = (3 * w // 4 + 3 * np.cos(ys / 5.0)).astype(int)
    lab = np.where(xs < a, 1, np.where(xs >= b, 2, 3)).astype(np.uint8)
    lab[0] = 0
    lab[h // 2, g.integers(0, w)] = 9
    return lab


def _image(h, w, c, dtype, seed):
    from scipy import ndimage
    g = np.random.default_rng(seed)
    planes = [ndimage.gaussian_filter(g.uniform(0, 1, size=(h, w)), 1.3) for _ in range(c)]
    img = np.stack(planes, -1) if c > 1 else planes[0]
    img = (img - img.min()) / (img.max() - img.min())
    return np.round(img * 255).astype(np.uint8) if dtype == np.uint8 else img.astype(np.float32)


def _check(got, F, lab, dtype):
    a1, a2, a3 = lab == 1, lab == 2, lab == 3
    neither = ~(a1 | a2 | a3)
    if dtype == np.uint8:
        want = oracle.quantize_u8(F)
        assert np.array_equal(got[a1 | a2 | neither], want[a1 | a2 | neither])
        assert np.abs(got[a3].astype(int) - want[a3].astype(int)).max() <= 1
    else:
        assert np.array_equal(got[neither], np.zeros_like(got[neither]))
        assert np.abs(got[a1 | a2] - F[a1 | a2]).max() == 0.0
        assert np.abs(got[a3] - F[a3]).max() <= 1e-5


@pytest.mark.parametrize("c,dtype", [(3, np.uint8), (1, np.float32), (3, np.float32)])
def test_compose_matches_oracle(c, dtype):
    h, w = 96, 160
    L, R = _image(h, w, c, dtype, 1), _image(h, w, c, dtype, 2)
    lab = _labels(h, w, 3)
    B = oracle.blend_coeff(lab).astype(np.float32)
    cols = np.nonzero((lab == 3).any(0))[0]
    x0, fw = int(cols.min()), int(cols.max() - cols.min() + 1)
    y0, fh = 1, h - 1
    yy, xx = np.mgrid[0:fh, 0:fw]
    g = np.random.default_rng(4)
    lr = np.stack([2.5 * np.sin(yy / 9.0 + 1), 1.0 * np.cos(xx / 7.0)], -1) + g.normal(0, 0.2, (fh, fw, 2))
    rl = -lr + g.normal(0, 0.3, (fh, fw, 2))
    lr, rl = lr.astype(np.float32), rl.astype(np.float32)
    p = binding.Params()
    got = host(binding.compose_pair(cuda(L), cuda(R), cuda(lab), cuda(B), cuda(lr), cuda(rl), origin=(y0, x0),
                                    params=p))
    F = oracle.compose(L, R, lab, B.astype(np.float64), lr, rl, (y0, x0), oracle.Params())
    _check(got, F, lab, dtype)


def test_area3_outside_the_crop_uses_zero_flow():
    h, w = 40, 64
    L, R = _image(h, w, 3, np.uint8, 5), _image(h, w, 3, np.uint8, 6)
    lab = np.full((h, w), 3, np.uint8)
    B = np.tile(((np.arange(w) + 1) / (w + 1)).astype(np.float32), (h, 1))
    g = np.random.default_rng(7)
    lr, rl = (g.normal(0, 2, (10, 12, 2)).astype(np.float32) for _ in range(2))
    got = host(binding.compose_pair(cuda(L), cuda(R), cuda(lab), cuda(B), cuda(lr), cuda(rl), origin=(5, 20)))
    F = oracle.compose(L, R, lab, B.astype(np.float64), lr, rl, (5, 20), oracle.Params())
    _check(got, F, lab, np.uint8)


def test_strip_canvas_area3_equals_blend_pair_bit_for_bit():
    h, ws, m = 48, 80, 8
    w = ws + 2 * m
    L, R = _image(h, w, 3, np.uint8, 8), _image(h, w, 3, np.uint8, 9)
    lab = np.full((h, w), 3, np.uint8)
    lab[:, :m], lab[:, m + ws:] = 1, 2
    B = oracle.blend_coeff(lab).astype(np.float32)
    g = np.random.default_rng(10)
    lr = g.uniform(-1.5, 1.5, (h, ws, 2)).astype(np.float32)
    rl = g.uniform(-1.5, 1.5, (h, ws, 2)).astype(np.float32)
    for f in (lr, rl):       # every sample stays inside the strip
        f[:, :3], f[:, -3:], f[:3], f[-3:] = 0, 0, 0, 0
    got = host(binding.compose_pair(cuda(L), cuda(R), cuda(lab), cuda(B), cuda(lr), cuda(rl), origin=(0, m)))
    Ld, Rd = cuda(L), cuda(R)
    with binding.FlowContext(binding.Params(), max_h=h, max_w=ws, max_c=3) as ctx:
        strip = host(ctx.blend_pair(Ld[:, m:m + ws], Rd[:, m:m + ws], cuda(lr), cuda(rl),
                                    blend=cuda(B[:, m:m + ws])))
    assert np.array_equal(got[:, m:m + ws], strip)
    assert np.array_equal(got[:, :m], L[:, :m]) and np.array_equal(got[:, m + ws:], R[:, m + ws:])


def test_compose_bad_arguments_raise():
    L = torch.zeros((16, 16, 3), dtype=torch.uint8, device=DEV)
    lab = torch.full((16, 16), 3, dtype=torch.uint8, device=DEV)
    B = torch.zeros((16, 16), dtype=torch.float32, device=DEV)
    f = torch.zeros((16, 8, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(binding.PanoError) as e:
        binding.compose_pair(L, L, lab, B, f, f, origin=(0, 9))        # crop leaves the canvas
    assert e.value.status == binding.PANO_ERR_INVALID_ARG
    with pytest.raises(binding.PanoError):
        binding.compose_pair(L, L, lab, B, f, f, out=L)                # F is an input


def test_stitch_canvas_runs_eq1_flow_and_code1_in_order():
    # a synthetic overlap pair with Area1 / Area2 margins around it
    pair = synth.pair_fullres_rgb(seed=4, h=160, w=240, dmax=8.0, levels=4)
    h, ws = pair.shape
    m = 40
    L = np.concatenate([_image(h, m, 3, np.uint8, 13), pair.L, pair.L[:, -m:]], 1)
    R = np.concatenate([pair.R[:, :m], pair.R, _image(h, m, 3, np.uint8, 14)], 1)
    lab = np.full((h, ws + 2 * m), 3, np.uint8)
    lab[:, :m], lab[:, m + ws:] = 1, 2
    p = binding.Params(levels=4)
    with binding.FlowContext(p, max_h=h, max_w=ws, max_c=3) as ctx:
        lr, rl, B, F = ctx.stitch_canvas(cuda(L), cuda(R), cuda(lab), (0, m, h, ws))
    lr, rl, B, F = host(lr), host(rl), host(B), host(F)
    np.testing.assert_allclose(B, oracle.blend_coeff(lab), rtol=0, atol=1e-6)
    olr, orl = oracle.flow_pair(L[:, m:m + ws], R[:, m:m + ws], oracle.Params(levels=4))
    assert np.hypot(*(lr - olr).transpose(2, 0, 1)).mean() <= 0.05
    assert np.hypot(*(rl - orl).transpose(2, 0, 1)).mean() <= 0.05
    Fo = oracle.compose(L, R, lab, B.astype(np.float64), lr, rl, (0, m), oracle.Params(levels=4))
    _check(F, Fo, lab, np.uint8)


@pytest.mark.slow
def test_full_size_canvas_around_the_benchmark_pair():
    """4000 x 3000 RGB u8 canvas: Area1 | the 4000 x 1500 overlap of the
    benchmark pair | Area2, flows from pano_flow_pair on the overlap crop."""
    pair = synth.pair_fullres_rgb()
    h, ws = pair.shape
    m = 750
    w = ws + 2 * m
    L = np.concatenate([_image(h, m, 3, np.uint8, 11), pair.L, pair.L[:, -m:][:, ::-1]], 1)
    R = np.concatenate([pair.R[:, :m][:, ::-1], pair.R, _image(h, m, 3, np.uint8, 12)], 1)
    lab = np.full((h, w), 3, np.uint8)
    lab[:, :m], lab[:, m + ws:] = 1, 2
    B = np.tile(np.concatenate([np.zeros(m), (np.arange(ws) + 1) / (ws + 1), np.ones(m)]).astype(np.float32), (h, 1))
    Ld, Rd = cuda(L), cuda(R)
    with binding.FlowContext(binding.Params(levels=6), max_h=h, max_w=ws, max_c=3) as ctx:
        lr, rl = ctx.flow_pair(Ld[:, m:m + ws].contiguous(), Rd[:, m:m + ws].contiguous())
    got = host(binding.compose_pair(Ld, Rd, cuda(lab), cuda(B), lr, rl, origin=(0, m),
                                    params=binding.Params(levels=6)))
    F = oracle.compose(L, R, lab, B.astype(np.float64), host(lr), host(rl), (0, m), oracle.Params(levels=6))
    _check(got, F, lab, np.uint8)
