"""Index checks of every kernel of the library on odd shapes.

The check variant of the library (build variant "check") checks every
shared-memory and global index of the streamed and the tiled LK kernels,
the pyramid kernels, the distance transform of Eq. (1) and the energy and
adjoint kernels, and the bilinear gathers of the warp, the strip blend and
the canvas compose, before the access; an index outside its array is recorded
and clamped instead of trapping (pano_debug_bounds). Every run below must
leave the record empty and give exactly the results of the release library:
the checks change no arithmetic.
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


@pytest.mark.parametrize("h,w,nlev", [(17, 33, 4), (5, 7, 3), (263, 129, 6), (1, 300, 2), (96, 1, 2)])
def test_pyramid_keeps_every_index_in_bounds(libs, monkeypatch, h, w, nlev):
    img = torch.from_numpy(_texture(h, w, 3, 5)).to(DEV)

    def run():
        Y, Y1 = binding.stage_luma_pyr(img)
        return [Y, Y1] + binding.stage_pyramid(Y, nlev)

    a, b, rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("h,w,c", [(37, 61, 3), (9, 250, 1), (120, 97, 3)])
def test_blends_and_warp_keep_every_index_in_bounds(libs, monkeypatch, h, w, c):
    m = 6
    canvas_L = torch.from_numpy(_texture(h, w + 2 * m, c, 6)).to(DEV)
    canvas_R = torch.from_numpy(_texture(h, w + 2 * m, c, 7)).to(DEV)
    L, R = canvas_L[:, m:m + w], canvas_R[:, m:m + w]            # strided strips
    g = np.random.default_rng(8)
    lr = torch.from_numpy(g.normal(0, 25, (h, w, 2)).astype(np.float32)).to(DEV)   # samples far outside
    rl = torch.from_numpy(g.normal(0, 25, (h, w, 2)).astype(np.float32)).to(DEV)
    lab = np.full((h, w + 2 * m), 3, np.uint8)
    lab[:, :m], lab[:, m + w:] = 1, 2
    lab[0, :3] = 0
    labd = torch.from_numpy(lab).to(DEV)
    B = torch.from_numpy(np.tile(np.linspace(0, 1, w + 2 * m, dtype=np.float32), (h, 1))).to(DEV)

    def run():
        with binding.FlowContext(binding.Params(), max_h=h, max_w=w, max_c=c) as ctx:
            F = ctx.blend_pair(L, R, lr, rl)
        G = binding.compose_pair(canvas_L, canvas_R, labd, B, lr, rl, origin=(0, m))
        Wp = binding.stage_warp(L, lr, 0.7)
        return F, G, Wp

    a, b, rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("h,w,kind", [(37, 61, "blobs"), (1, 200, "blobs"), (150, 1, "blobs"), (40, 90, "no_area1"),
                                      (33, 47, "area3_only"), (64, 300, "single_sites"), (2100, 7, "single_sites"),
                                      (3, 9000, "blobs"), (5, 40000, "single_sites")])
def test_distance_transform_keeps_every_index_in_bounds(libs, monkeypatch, h, w, kind):
    g = np.random.default_rng(9)
    if kind == "blobs":
        lab = g.choice(np.array([0, 1, 2, 3, 3, 3], np.uint8), size=(h, w))
    elif kind == "no_area1":
        lab = np.where(g.uniform(size=(h, w)) < 0.05, 2, 3).astype(np.uint8)
    elif kind == "area3_only":
        lab = np.full((h, w), 3, np.uint8)
    else:   # one Area1 and one Area2 pixel per row, so every envelope has one site per column band
        lab = np.full((h, w), 3, np.uint8)
        lab[np.arange(h), g.integers(0, w, h)] = 1
        lab[np.arange(h), g.integers(0, w, h)] = 2
    canvas = torch.zeros((h, w + 5), dtype=torch.uint8, device=DEV)
    canvas[:, 2:2 + w] = torch.from_numpy(lab).to(DEV)
    label = canvas[:, 2:2 + w]                                  # a strided label

    a, b, rec = _run_both(libs, monkeypatch, lambda: binding.blend_coeff(label))
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    assert torch.equal(a, b)


@pytest.mark.parametrize("h,w", [(29, 45), (1, 70), (64, 1), (130, 257)])
def test_energy_and_adjoint_keep_every_index_in_bounds(libs, monkeypatch, h, w):
    T = torch.from_numpy(_texture(h, w, 1, 11)).to(DEV)
    J = torch.from_numpy(_texture(h, w, 1, 12)).to(DEV)
    g = np.random.default_rng(13)
    u = torch.from_numpy(g.normal(0, 40, (h, w, 2)).astype(np.float32)).to(DEV)   # samples far outside
    gd = torch.from_numpy(g.normal(0, 1, ((h + 1) // 2, (w + 1) // 2)).astype(np.float32)).to(DEV)

    def run():
        E, gu, gt, gj = binding.energy_grad(T, J, u, 0.3)
        return E, gu, gt, gj, binding.stage_pyr_down_adjoint(gd, h, w)

    (Ea, gua, gta, gja, ada), (Eb, gub, gtb, gjb, adb), rec = _run_both(libs, monkeypatch, run)
    assert rec[0] == 0, f"{rec[0]} indices out of bounds, first at site {rec[1]}: {rec[2]} of {rec[3]}"
    assert torch.equal(gua, gub) and torch.equal(gta, gtb) and torch.equal(ada, adb)
    # E and dE/dJ are sums by atomics, in no fixed order
    torch.testing.assert_close(Eb, Ea, rtol=1e-12, atol=0)
    torch.testing.assert_close(gjb, gja, rtol=1e-5, atol=1e-6)
