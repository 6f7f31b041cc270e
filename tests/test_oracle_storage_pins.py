"""Pins of the oracle's 16-bit storage of pyramid levels.

The rounding to bfloat16 / binary16 is checked against conversions that do
not share its code: numpy's double -> float16 (round to nearest even,
subnormals and overflow included) and torch's float32 -> bfloat16 (on
float32 inputs, where no double rounding can occur), plus hand-made ties.
The stored pyramid is checked by properties: every stored value is
representable, and the stored levels stay within the rounding bound of the
exact pyramid."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _samples(seed=0, n=20000):
    g = np.random.default_rng(seed)
    mag = 10.0 ** g.uniform(-9, 5.5, n)            # binary16 subnormals .. beyond 65504
    x = mag * g.choice([-1.0, 1.0], n)
    unit = g.uniform(0, 1, n)                      # the range of a luma pyramid
    return np.concatenate([x, unit, [0.0, -0.0, 1.0, 65504.0, 65519.99, 65520.0, 6.0e-8, 2.0 ** -24]])


def test_binary16_rounding_matches_numpy():
    x = _samples()
    got = oracle.round_storage(x, oracle.FMT_F16)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, ref)


def test_bfloat16_rounding_matches_torch_on_float32_inputs():
    x = _samples(1).astype(np.float32)
    x = x[np.isfinite(x)]
    got = oracle.round_storage(x.astype(np.float64), oracle.FMT_BF16)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, ref)


def test_ties_go_to_the_even_neighbour():
    # bfloat16 has 7 fraction bits: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    t = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 2.0 ** -133 * 1.5])
    got = oracle.round_storage(t, oracle.FMT_BF16)
    assert list(got) == [1.0, 1 + 2.0 ** -6, -1.0, 2.0 ** -132]
    # binary16 has 10 fraction bits
    u = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -25, 3 * 2.0 ** -25])
    assert list(oracle.round_storage(u, oracle.FMT_F16)) == [1.0, 1 + 2.0 ** -9, 0.0, 2.0 ** -23]


def test_exact_format_is_the_identity():
    x = _samples(2)
    assert np.array_equal(oracle.round_storage(x, oracle.FMT_EXACT), x)


@pytest.mark.parametrize("fmt,p", [(oracle.FMT_BF16, 8), (oracle.FMT_F16, 11)])
def test_stored_pyramid_is_representable_and_close_to_the_exact_one(fmt, p):
    g = np.random.default_rng(3)
    from scipy import ndimage
    Y = ndimage.gaussian_filter(g.uniform(0, 1, (67, 93)), 1.5)
    exact = oracle.pyramid(Y, 4)
    stored = oracle.pyramid(Y, 4, fmt)
    for l, (a, b) in enumerate(zip(exact, stored)):
        assert np.array_equal(oracle.round_storage(b, fmt), b)
        # each level adds at most half an ulp of rounding to an average of
        # values already within the bound of the levels below (REDUCE has
        # positive weights summing to one): l + 1 half-ulps relative to 1
        assert np.abs(a - b).max() <= (l + 1) * 2.0 ** -p * 1.0001, l
        if fmt == oracle.FMT_F16:
            assert not np.array_equal(a, b)


def test_stored_flow_with_exact_format_equals_flow_pair_and_bf16_stays_close():
    import synth
    pair = synth.pair_small_gray(h=96, w=128, amp_x=2.0, amp_y=1.0, levels=3)
    p0 = oracle.Params(levels=3)
    lr0, rl0 = oracle.flow_pair(pair.L, pair.R, p0)
    lr1, rl1 = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=3, pyr_fmt=oracle.FMT_F16))
    lr2, _ = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=3, pyr_fmt=oracle.FMT_BF16))
    e16 = np.hypot(*(lr1 - lr0).transpose(2, 0, 1))
    ebf = np.hypot(*(lr2 - lr0).transpose(2, 0, 1))
    assert 0 < e16.mean() < ebf.mean() < 0.05
