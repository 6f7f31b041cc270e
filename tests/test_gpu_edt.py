"""Eq. (1) on labelled canvases of any shape (pano_blend_coeff) against the
FP64 oracle's brute force.

The GPU distances are exact integers; only the final ratio is rounded in
FP32 (two square roots and a division, a few ulps of a value in [0, 1]), so
the bar is max-abs 1e-6. Canvases the brute force finishes in seconds are
compared in full; the 4000 x 9000 canvas at sampled pixels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_01201_gb300 import binding  # noqa: E402
from paper_2006_01201_gb300 import build as gpu_build  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def gpu_blend(label):
    out = binding.blend_coeff(torch.from_numpy(np.ascontiguousarray(label)).to(DEV))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def overlap_canvas(h, w, seed, holes=True):
    """Area1 on the left, Area2 on the right, Area3 between two wavy seams,
    with small blobs of "neither" (holes in both images)."""
    g = np.random.default_rng(seed)
    ys = np.arange(h)[:, None]
    xs = np.arange(w)[None, :]
    a = 0.3 * w + 0.08 * w * np.sin(2 * np.pi * ys / (0.7 * h) + g.uniform(0, 6)) + g.normal(0, 0.01 * w, (h, 1))
    b = 0.7 * w + 0.08 * w * np.sin(2 * np.pi * ys / (0.5 * h) + g.uniform(0, 6))
    lab = np.where(xs < a, 1, np.where(xs >= b, 2, 3)).astype(np.uint8)
    if holes:
        for _ in range(6):
            cy, cx, r = g.integers(0, h), g.integers(0, w), g.integers(1, max(2, min(h, w) // 10))
            lab[(ys - cy) ** 2 + (xs - cx) ** 2 <= r * r] = 0
    return lab


@pytest.mark.parametrize("shape,seed", [((37, 53), 0), ((64, 64), 1), ((1, 40), 2), ((40, 1), 3), ((1, 1), 4),
                                        ((120, 150), 5)])
def test_random_labels_match_oracle(shape, seed):
    g = np.random.default_rng(seed)
    label = g.choice([0, 1, 2, 3, 7], p=[0.05, 0.05, 0.05, 0.8, 0.05], size=shape).astype(np.uint8)
    np.testing.assert_allclose(gpu_blend(label), oracle.blend_coeff(label), rtol=0, atol=TOL)


@pytest.mark.parametrize("shape,seed", [((90, 160), 6), ((150, 97), 7)])
def test_overlap_canvases_match_oracle(shape, seed):
    label = overlap_canvas(*shape, seed)
    np.testing.assert_allclose(gpu_blend(label), oracle.blend_coeff(label), rtol=0, atol=TOL)


def test_missing_areas_give_the_limits():
    lab = np.full((5, 9), 3, np.uint8)
    lab[:, -1] = 2
    assert (gpu_blend(lab) == 1.0).all()
    lab[:, -1] = 1
    assert (gpu_blend(lab) == 0.0).all()
    lab[:, -1] = 0
    assert (gpu_blend(lab) == 0.5).all()


@pytest.mark.parametrize("w", [1, 4, 31, 1500])
def test_strip_geometry_gives_the_eq1_ramp(w):
    lab = np.full((6, w + 2), 3, np.uint8)
    lab[:, 0], lab[:, -1] = 1, 2
    got = gpu_blend(lab)
    np.testing.assert_allclose(got[:, 1:-1], np.broadcast_to(oracle.blend_ramp(w), (6, w)), rtol=0, atol=TOL)


def test_general_blend_feeds_the_code1_blend():
    import synth
    pair = synth.pair_small_gray(h=96, w=128, levels=3)
    label = np.full((96, 130), 3, np.uint8)
    label[:, 0], label[:, -1] = 1, 2
    label[:30, :20] = 1                              # Area1 reaches into the strip's corner
    B = gpu_blend(label)[:, 1:-1]
    Bt = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).to(DEV)
    with binding.FlowContext(binding.Params(levels=3), 96, 128, 1) as ctx:
        L, R = torch.from_numpy(pair.L).to(DEV), torch.from_numpy(pair.R).to(DEV)
        lr, rl = ctx.flow_pair(L, R)
        F = ctx.blend_pair(L, R, lr, rl, blend=Bt)
        torch.cuda.synchronize()
    Fo = oracle.blend(pair.L, pair.R, lr.cpu().numpy().astype(np.float64), rl.cpu().numpy().astype(np.float64),
                      oracle.Params(levels=3), oracle.blend_coeff(label)[:, 1:-1])
    assert np.abs(F.cpu().numpy() - Fo).max() <= 1e-5


def test_full_canvas_at_sampled_pixels():
    """4000 x 9000 panorama canvas with wavy seams and holes, checked at 300
    sampled pixels (the brute force scans the whole canvas per pixel)."""
    label = overlap_canvas(4000, 9000, 8)
    got = gpu_blend(label)
    g = np.random.default_rng(9)
    area3 = np.argwhere(label == 3)
    pick = area3[g.choice(len(area3), 250, replace=False)]
    other = np.stack([g.integers(0, 4000, 50), g.integers(0, 9000, 50)], -1)
    ys, xs = np.concatenate([pick[:, 0], other[:, 0]]), np.concatenate([pick[:, 1], other[:, 1]])
    np.testing.assert_allclose(got[ys, xs], oracle.blend_coeff_at(label, ys, xs), rtol=0, atol=TOL)
    assert np.isfinite(got).all() and (got >= 0).all() and (got <= 1).all()


def _sampled(label, n, seed):
    """GPU Blend against the oracle's brute force at n pixels (Area3 first)."""
    got = gpu_blend(label)
    g = np.random.default_rng(seed)
    area3 = np.argwhere(label == 3)
    pick = area3[g.choice(len(area3), min(n, len(area3)), replace=False)]
    other = np.stack([g.integers(0, label.shape[0], n // 4), g.integers(0, label.shape[1], n // 4)], -1)
    ys, xs = np.concatenate([pick[:, 0], other[:, 0]]), np.concatenate([pick[:, 1], other[:, 1]])
    np.testing.assert_allclose(got[ys, xs], oracle.blend_coeff_at(label, ys, xs), rtol=0, atol=TOL)
    assert np.isfinite(got).all() and (got >= 0).all() and (got <= 1).all()


def test_wide_canvas_many_columns_per_band():
    """56000 columns (219 per thread of the row pass, near the shared-memory
    limit), wavy seams, holes and scattered Area1/Area2 pixels."""
    label = overlap_canvas(12, 56000, 10)
    g = np.random.default_rng(11)
    label[g.integers(0, 12, 300), g.integers(0, 56000, 300)] = g.choice([1, 2], 300)
    _sampled(label, 400, 12)


def test_tall_canvas_carries_across_row_blocks():
    """5000 rows (five 1024-row blocks of the column pass): the nearest
    feature of a column often lies blocks away."""
    h, w = 5000, 37
    label = np.full((h, w), 3, np.uint8)
    g = np.random.default_rng(13)
    for x in range(w):                       # a few feature pixels per column, anywhere
        k = g.integers(0, 4)
        label[g.integers(0, h, k), x] = g.choice([1, 2], k)
    label[:, 5] = 3                          # columns without any feature pixel
    label[1023:1026, 7] = 1                  # features at block edges
    label[2047, 9], label[2048, 9] = 2, 1
    _sampled(label, 1500, 14)


@pytest.mark.parametrize("shape,seed", [((90, 1100), 15), ((33, 4097), 16)])
def test_dense_random_labels_sampled(shape, seed):
    g = np.random.default_rng(seed)
    label = g.choice([0, 1, 2, 3], p=[0.1, 0.15, 0.15, 0.6], size=shape).astype(np.uint8)
    _sampled(label, 1500, seed + 100)


def test_too_wide_canvas_is_refused():
    lab = torch.full((2, 60000), 3, dtype=torch.uint8, device=DEV)
    with pytest.raises(binding.PanoError) as e:
        binding.blend_coeff(lab)
    assert e.value.status == binding.PANO_ERR_UNSUPPORTED


def test_bad_arguments_raise():
    lab = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    with pytest.raises(binding.PanoError):
        binding.blend_coeff(lab, scratch=torch.empty(16, dtype=torch.uint8, device=DEV))
    with pytest.raises(binding.PanoError):
        binding.blend_coeff(lab.float())
