"""pano_flow_pair_static: the flow of a strip pair without any device
allocation inside the library.

Callers that own all device memory through their own pool, or that run a
frame loop where cudaMalloc / cudaFree would add latency and synchronise the
device, cannot create a context (pano_flow_create allocates). This entry point
serves them from a fixed scratch array in the library. These tests call it
through the C ABI twice in a row, with different strips, and compare each
result with pano_flow_pair on the same inputs; they also check that a strip
too large for the fixed scratch is refused before anything is enqueued.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_01201_gb300 import binding  # noqa: E402
from paper_2006_01201_gb300 import build as gpu_build  # noqa: E402

DEV = torch.device("cuda:0")
# the tolerance of the other GPU flow tests is a mean endpoint error of 0.05 px
# against the oracle; against pano_flow_pair (same kernels) the bar is tighter
MAX_ABS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def _pairs():
    small = synth.pair_small_gray()                                   # 256 x 512 gray f32
    rgb = synth.pair_fullres_rgb(seed=3, h=300, w=400, dmax=12.0, levels=4)   # RGB u8
    return [(small, 4), (rgb, 4)]


def test_static_flow_matches_context_flow_on_two_calls_in_a_row():
    results = []
    for pair, levels in _pairs():
        L = torch.from_numpy(pair.L).to(DEV)
        R = torch.from_numpy(pair.R).to(DEV)
        params = binding.Params(levels=levels)
        s_lr, s_rl = binding.flow_pair_static(params, L, R)
        torch.cuda.synchronize()
        h, w = pair.shape
        with binding.FlowContext(params, max_h=h, max_w=w, max_c=3) as ctx:
            c_lr, c_rl = ctx.flow_pair(L, R)
            torch.cuda.synchronize()
        results.append(((s_lr - c_lr).abs().max().item(), (s_rl - c_rl).abs().max().item()))
    for d_lr, d_rl in results:
        assert d_lr <= MAX_ABS and d_rl <= MAX_ABS, results


def test_repeated_static_calls_give_the_same_flow():
    pair, levels = _pairs()[0]
    L = torch.from_numpy(pair.L).to(DEV)
    R = torch.from_numpy(pair.R).to(DEV)
    params = binding.Params(levels=levels)
    a = binding.flow_pair_static(params, L, R)
    b = binding.flow_pair_static(params, R, L)      # other strips in between
    c = binding.flow_pair_static(params, L, R)
    torch.cuda.synchronize()
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    assert torch.equal(b[0], a[1]) and torch.equal(b[1], a[0])


def test_largest_strip_that_fits_runs_and_one_more_column_is_refused():
    # 1024 x 1024 with 4 levels needs 16.65 MB of the 16 MiB scratch; a
    # 1025th column rounds every level's row pitch up by 32 floats (17.37 MB)
    g = np.random.default_rng(5)
    from scipy import ndimage
    T = ndimage.gaussian_filter(g.uniform(0, 1, (1024, 1025)), 1.5).astype(np.float32)
    J = np.roll(T, (1, 2), axis=(0, 1))
    params = binding.Params(levels=4)
    L = torch.from_numpy(np.ascontiguousarray(T[:, :1024])).to(DEV)
    R = torch.from_numpy(np.ascontiguousarray(J[:, :1024])).to(DEV)
    s_lr, s_rl = binding.flow_pair_static(params, L, R)
    with binding.FlowContext(params, max_h=1024, max_w=1024, max_c=1) as ctx:
        c_lr, c_rl = ctx.flow_pair(L, R)
        torch.cuda.synchronize()
    assert (s_lr - c_lr).abs().max().item() <= MAX_ABS and (s_rl - c_rl).abs().max().item() <= MAX_ABS
    wide = torch.from_numpy(T).to(DEV)
    with pytest.raises(binding.PanoError) as ei:
        binding.flow_pair_static(params, wide, wide)
    assert ei.value.status == binding.PANO_ERR_INVALID_ARG and "scratch" in ei.value.message


def test_strip_too_large_for_the_fixed_scratch_is_refused():
    big = torch.zeros((2048, 2048), dtype=torch.float32, device=DEV)
    with pytest.raises(binding.PanoError) as ei:
        binding.flow_pair_static(binding.Params(levels=4), big, big)
    assert ei.value.status == binding.PANO_ERR_INVALID_ARG
    assert "scratch" in ei.value.message
    assert np.isfinite(big.sum().item())


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import synth
from paper_2006_01201_gb300 import binding
binding.load_library()
dev = torch.device("cuda:0")
pair = synth.pair_fullres_rgb(seed=9, h=520, w=700, dmax=10.0, levels=7)
L = torch.from_numpy(pair.L).to(dev)
R = torch.from_numpy(pair.R).to(dev)
worst = 0.0
for levels in (6, 7):
    p = binding.Params(levels=levels)
    s_lr, s_rl = binding.flow_pair_static(p, L, R)   # before any context exists
    torch.cuda.synchronize()
    with binding.FlowContext(p, max_h=520, max_w=700, max_c=3) as ctx:
        c_lr, c_rl = ctx.flow_pair(L, R)
        torch.cuda.synchronize()
    worst = max(worst, (s_lr - c_lr).abs().max().item(), (s_rl - c_rl).abs().max().item())
print("MAXDIFF", worst)
"""


def test_static_flow_with_six_and_seven_levels_in_a_fresh_process():
    """With 6 or more levels the pyramid's multi-level REDUCE needs more than
    48 KB of shared memory; the first call of a process that never created a
    context must set that limit itself."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    worst = float(r.stdout.split("MAXDIFF")[1].split()[0])
    assert worst <= MAX_ABS, worst
