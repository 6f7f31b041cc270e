"""Index checks of the LK kernels on odd shapes.

The check variant of the library (build variant "check") checks every
shared-memory and global index of the streamed and the tiled LK kernels
before the access; an index outside its array is recorded and clamped
instead of trapping (pano_debug_bounds). Every run below must leave the
record empty and give exactly the flows of the release library: the checks
change no arithmetic.
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


@pytest.fixture(scope="module")
def libs():
    release = binding.open_library(gpu_build.build())
    check = binding.open_library(gpu_build.build(variant="check"))
    return release, check


def _run_both(libs, monkeypatch, fn):
    """fn() with the release library, then with the check variant; returns
    both results and the check variant's index record."""
    release, check = libs
    monkeypatch.setattr(binding, "_lib", release)
    a = fn()
    torch.cuda.synchronize()
    monkeypatch.setattr(binding, "_lib", check)
    binding.debug_bounds()          # start from an empty record
    b = fn()
    torch.cuda.synchronize()
    return a, b, binding.debug_bounds()


def _texture(h, w, c, seed):
    from scipy import ndimage
    g = np.random.default_rng(seed)
    planes = [ndimage.gaussian_filter(g.uniform(0, 1, (h, w)), 1.2) for _ in range(c)]
    img = np.stack(planes, -1) if c > 1 else planes[0]
    return (np.round(255 * (img - img.min()) / (img.max() - img.min()))).astype(np.uint8) if c == 3 \
        else img.astype(np.float32)


@pytest.mark.parametrize("h,w,c,levels,pyr", [(17, 33, 1, 2, "f32"), (37, 61, 3, 3, "f32"), (101, 203, 3, 4, "f32"),
                                              (230, 317, 1, 4, "f32"), (5, 7, 1, 1, "f32"), (2, 300, 1, 2, "f32"),
                                              (300, 2, 3, 2, "f32"), (230, 317, 3, 4, "bf16"),
                                              (61, 97, 1, 3, "f16")])
def test_flow_pair_keeps_every_index_in_bounds(libs, monkeypatch, h, w, c, levels, pyr):
    L = _texture(h, w, c, 1)
    R = np.roll(L, (1, -2), axis=(0, 1))
    Ld, Rd = torch.from_numpy(L).to(DEV), torch.from_numpy(R).to(DEV)
    dtype = {"f32": binding.PANO_F32, "bf16": binding.PANO_BF16, "f16": binding.PANO_F16}[pyr]
    params = binding.Params(levels=levels, pyr_dtype=dtype)

    def run():
        with binding.FlowContext(params, max_h=h, max_w=w, max_c=c) as ctx:
            out = ctx.flow_pair(Ld, Rd)
            torch.cuda.synchronize()
        return out

    (a_lr, a_rl), (b_lr, b_rl), rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    assert torch.equal(a_lr, b_lr) and torch.equal(a_rl, b_rl)


@pytest.mark.parametrize("kernel", [binding.PANO_LK_STREAM, binding.PANO_LK_TILE])
@pytest.mark.parametrize("radius,iters", [(1, 1), (2, 3), (2, 5), (3, 5), (3, 2)])
@pytest.mark.parametrize("h,w,start", [(53, 97, "coarse"), (230, 317, "zero"), (9, 250, "given")])
def test_each_lk_kernel_keeps_every_index_in_bounds(libs, monkeypatch, kernel, radius, iters, h, w, start):
    T = _texture(h, w, 1, 2)
    J = np.roll(T, (2, 3), axis=(0, 1)).astype(np.float32)
    g = np.random.default_rng(3)
    if start == "coarse":
        uin = torch.from_numpy(g.normal(0, 4, ((h + 1) // 2, (w + 1) // 2, 2)).astype(np.float32)).to(DEV)
    elif start == "given":
        uin = torch.from_numpy(g.normal(0, 30, (h, w, 2)).astype(np.float32)).to(DEV)   # far outside the box
    else:
        uin = None
    Td, Jd = torch.from_numpy(T).to(DEV), torch.from_numpy(J).to(DEV)

    def run():
        return binding.stage_lk(Td, Jd, uin, upsample=start == "coarse", iters=iters, radius=radius, lam=1e-2,
                                kernel=kernel)

    a, b, rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    assert torch.equal(a, b)


def test_rig_keeps_every_index_in_bounds(libs, monkeypatch):
    widths = [97, 150, 233]
    h = 120
    pairs = [synth.pair_fullres_rgb(seed=40 + k, h=h, w=wk, dmax=6.0, levels=3) for k, wk in enumerate(widths)]
    Ls = [torch.from_numpy(p.L).to(DEV) for p in pairs]
    Rs = [torch.from_numpy(p.R).to(DEV) for p in pairs]

    def run():
        with binding.Rig(binding.Params(levels=3), h, widths, 3, canvas_hw=(h, 400), canvas_x0=[0, 90, 230]) as rig:
            cv = rig.new_canvas()
            rig.run(Ls, Rs, canvas=cv)
            torch.cuda.synchronize()
            return [rig.flows(k) for k in range(len(widths))], cv

    (fa, ca), (fb, cb), rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    assert torch.equal(ca, cb)
    for (alr, arl), (blr, brl) in zip(fa, fb):
        assert torch.equal(alr, blr) and torch.equal(arl, brl)
