"""A whole rig through one pano_rig object against the single-pair path and
the FP64 oracle.

With the default tuning the rig's flows must equal pano_flow_pair's bit for
bit (same kernels, same tiles and segments, batched differently), and its
canvas must equal the single-pair blends placed by the rule of the header:
strip k at columns (x0[k] + x) mod canvas_w, the highest pair index wins
where spans overlap, every other canvas pixel untouched. Other tunings change
only FP32 rounding; they are held to the end-to-end bound against the oracle
(mean endpoint error <= 0.05 px) and to 1e-3 px mean against the default.
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
SENTINEL = 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def epe(a, b):
    return np.hypot(*(a - b).transpose(2, 0, 1))


# h = 400: level 0 of the 100-wide pair has 40000 pixels (tiled kernel), of
# the others 96000 and 70400 (streamed kernel), so level 0 is split over both
# kernel kinds; at level 1 the 100-wide pair drops below 16000 pixels and
# gets the small tiles while the others keep the default ones (two tiled
# launches). The third span wraps around the canvas seam and covers the
# start of the first.
GEOM = dict(h=400, widths=(240, 100, 176), x0=(0, 200, 520), canvas=(420, 600), y0=10, levels=4)


@pytest.fixture(scope="module")
def small_rig_pairs():
    return [synth.pair_fullres_rgb(seed=40 + k, h=GEOM["h"], w=w, dmax=6.0, levels=GEOM["levels"])
            for k, w in enumerate(GEOM["widths"])]


def make_rig(pairs, geom=GEOM, dtype=torch.uint8, c=3):
    return binding.Rig(binding.Params(levels=geom["levels"]), geom["h"], geom["widths"], c=c, dtype=dtype,
                       canvas_hw=geom["canvas"], canvas_x0=geom["x0"], canvas_y0=geom["y0"])


def per_pair(pairs, geom=GEOM):
    """Flows and F of every pair through pano_flow_pair / pano_blend_pair."""
    out = []
    with binding.FlowContext(binding.Params(levels=geom["levels"]), geom["h"], max(geom["widths"]), 3) as ctx:
        for p in pairs:
            L, R = cuda(p.L), cuda(p.R)
            lr, rl, F = ctx.stitch_pair(L, R)
            out.append((lr, rl, F))
        torch.cuda.synchronize()
    return out


def place(canvas, Fs, geom=GEOM):
    """The placement rule on the host: pairs in index order, later ones overwrite."""
    cw = geom["canvas"][1]
    y0, h = geom["y0"], geom["h"]
    for F, x0 in zip(Fs, geom["x0"]):
        cols = (x0 + np.arange(F.shape[1])) % cw
        canvas[y0:y0 + h, cols] = F
    return canvas


def test_default_tuning_equals_single_pair_path_and_places_canvas(small_rig_pairs):
    pairs = small_rig_pairs
    ref = per_pair(pairs)
    with make_rig(pairs) as rig:
        Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
        flows = [(torch.empty(p.L.shape[:2] + (2,), device=DEV), torch.empty(p.L.shape[:2] + (2,), device=DEV))
                 for p in pairs]
        canvas = rig.new_canvas().fill_(SENTINEL)
        rig.run(Ls, Rs, flows=flows, canvas=canvas)
        torch.cuda.synchronize()
        for k, ((lr, rl), (rlr, rrl, _)) in enumerate(zip(flows, ref)):
            assert torch.equal(lr, rlr) and torch.equal(rl, rrl), k
        expect = np.full(canvas.shape, SENTINEL, np.uint8)
        place(expect, [F.cpu().numpy() for _, _, F in ref])
        got = canvas.cpu().numpy()
        assert np.array_equal(got, expect)
        # columns 300..519 lie in no span and rows outside the strips are untouched
        assert (got[:, 300:520] == SENTINEL).all()
        assert (got[:GEOM["y0"]] == SENTINEL).all() and (got[GEOM["y0"] + GEOM["h"]:] == SENTINEL).all()


def test_rig_flows_match_oracle(small_rig_pairs):
    pairs = small_rig_pairs
    with make_rig(pairs) as rig:
        rig.run([cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs])
        torch.cuda.synchronize()
        prm = oracle.Params(levels=GEOM["levels"])
        for k in (0, 1):
            olr, orl = oracle.flow_pair(pairs[k].L, pairs[k].R, prm)
            lr, rl = (t.cpu().numpy() for t in rig.flows(k))
            assert epe(lr, olr).mean() <= 0.05 and epe(rl, orl).mean() <= 0.05, k


def test_graph_replay_equals_eager_and_recaptures_on_new_buffers(small_rig_pairs):
    pairs = small_rig_pairs
    with make_rig(pairs) as rig:
        Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
        c_eager = rig.new_canvas()
        rig.run(Ls, Rs, canvas=c_eager)
        f_eager = [rig.flows(k) for k in range(3)]
        n0 = rig.launches
        c_graph = rig.new_canvas()
        rig.run(Ls, Rs, canvas=c_graph, use_graph=True)
        n1 = rig.launches
        c_graph.zero_()
        rig.run(Ls, Rs, canvas=c_graph, use_graph=True)
        torch.cuda.synchronize()
        assert rig.graph_captures == 1
        assert rig.launches - n1 == n1 - n0 > 0
        assert torch.equal(c_graph, c_eager)
        for k in range(3):
            a, b = rig.flows(k)
            assert torch.equal(a, f_eager[k][0]) and torch.equal(b, f_eager[k][1])
        c_other = rig.new_canvas()
        rig.run(Ls, Rs, canvas=c_other, use_graph=True)  # new canvas pointer: new graph
        assert rig.graph_captures == 2
        for _ in range(3):                                # both graphs stay cached
            rig.run(Ls, Rs, canvas=c_graph, use_graph=True)
            rig.run(Ls, Rs, canvas=c_other, use_graph=True)
        assert rig.graph_captures == 2
        torch.cuda.synchronize()
        assert torch.equal(c_graph, c_other)
        rig.set_tuning(0, binding.PANO_LK_TILE, tile_w=32, tile_h=8)
        rig.run(Ls, Rs, canvas=c_other, use_graph=True)  # new tuning: new graph
        assert rig.graph_captures == 3
        torch.cuda.synchronize()


def test_host_pipeline_matches_direct_calls(small_rig_pairs):
    """Double-buffered host pipelines (copies of neighbouring items overlap
    the kernels of the current one) give the results of direct calls."""
    pairs = small_rig_pairs
    with make_rig(pairs) as rig:
        Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
        ref = rig.new_canvas()
        rig.run(Ls, Rs, canvas=ref, use_graph=True)
        torch.cuda.synchronize()
        pipe = binding.RigHostPipeline(rig)
        Lh = [torch.from_numpy(p.L).pin_memory() for p in pairs]
        Rh = [torch.from_numpy(p.R).pin_memory() for p in pairs]
        outs = [torch.empty(tuple(ref.shape), dtype=ref.dtype).pin_memory() for _ in range(4)]
        for k in range(4):
            pipe.submit(k, Lh, Rh, outs[k])
        pipe.drain()
        for o in outs:
            assert torch.equal(o, ref.cpu())
        assert rig.graph_captures <= 3
    p = pairs[0]
    h, w = p.L.shape[:2]
    with binding.FlowContext(binding.Params(levels=GEOM["levels"]), h, w, 3) as ctx:
        _, _, F = ctx.stitch_pair(cuda(p.L), cuda(p.R))
        torch.cuda.synchronize()
        pipe = ctx.host_pipeline(p.L.shape, torch.uint8)
        Lh, Rh = torch.from_numpy(p.L).pin_memory(), torch.from_numpy(p.R).pin_memory()
        outs = [torch.empty(p.L.shape, dtype=torch.uint8).pin_memory() for _ in range(3)]
        for k in range(3):
            pipe.submit(k, Lh, Rh, outs[k])
        pipe.drain()
        for o in outs:
            assert torch.equal(o, F.cpu())


@pytest.mark.parametrize("kernel,seg,tile", [(binding.PANO_LK_STREAM, 0, (0, 0)),
                                             (binding.PANO_LK_STREAM, 64, (0, 0)),
                                             (binding.PANO_LK_TILE, 0, (64, 8)),
                                             (binding.PANO_LK_TILE, 0, (16, 16))])
def test_forced_kernels_agree_with_default(small_rig_pairs, kernel, seg, tile):
    pairs = small_rig_pairs
    Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
    with make_rig(pairs) as rig:
        rig.run(Ls, Rs)
        base = [rig.flows(k) for k in range(3)]
        for l in range(GEOM["levels"]):
            rig.set_tuning(l, kernel, seg_rows=seg, tile_w=tile[0], tile_h=tile[1])
        rig.run(Ls, Rs, use_graph=True)
        torch.cuda.synchronize()
        for k in range(3):
            for a, b in zip(rig.flows(k), base[k]):
                d = (a - b).abs()
                assert float(d.mean()) <= 1e-3 and float(d.max()) <= 0.25, (k, float(d.mean()), float(d.max()))


def test_autotune_sets_valid_tunings_and_keeps_results(small_rig_pairs):
    pairs = small_rig_pairs
    Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
    with make_rig(pairs) as rig:
        rig.run(Ls, Rs)
        base = [rig.flows(k) for k in range(3)]
        tunings = rig.autotune(Ls, Rs, reps=2)
        assert len(tunings) == GEOM["levels"]
        for t in tunings:
            assert t["kernel"] in (binding.PANO_LK_AUTO, binding.PANO_LK_STREAM, binding.PANO_LK_TILE)
            assert t["ms"] > 0.0
        rig.run(Ls, Rs, use_graph=True)
        torch.cuda.synchronize()
        for k in range(3):
            for a, b in zip(rig.flows(k), base[k]):
                assert float((a - b).abs().mean()) <= 1e-3


def test_float_gray_rig_equals_single_pair_path():
    geom = dict(h=160, widths=(96, 130), x0=(0, 90), canvas=(160, 300), y0=0, levels=3)
    pairs = [synth.pair_small_gray(seed=50 + k, h=160, w=w, levels=3) for k, w in enumerate(geom["widths"])]
    with binding.FlowContext(binding.Params(levels=3), 160, 130, 1) as ctx:
        ref = [ctx.stitch_pair(cuda(p.L), cuda(p.R)) for p in pairs]
        torch.cuda.synchronize()
    with make_rig(pairs, geom, dtype=torch.float32, c=1) as rig:
        canvas = rig.new_canvas().fill_(-1.0)
        rig.run([cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs], canvas=canvas, use_graph=True)
        torch.cuda.synchronize()
        for k in range(2):
            a, b = rig.flows(k)
            assert torch.equal(a, ref[k][0]) and torch.equal(b, ref[k][1])
        expect = np.full(canvas.shape, -1.0, np.float32)
        place(expect, [F.cpu().numpy() for _, _, F in ref], geom)
        assert np.array_equal(canvas.cpu().numpy(), expect)


def test_bad_arguments_raise(small_rig_pairs):
    pairs = small_rig_pairs
    with make_rig(pairs) as rig:
        Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
        with pytest.raises(binding.PanoError) as ei:
            rig.run(Ls[::-1], Rs[::-1])                    # widths in the wrong order
        assert ei.value.status == binding.PANO_ERR_INVALID_ARG
        with pytest.raises(binding.PanoError):
            rig.run(Ls, Rs, canvas=torch.zeros((420, 600, 3), dtype=torch.float32, device=DEV))
        with pytest.raises(binding.PanoError):
            rig.run(Ls, Rs, canvas=torch.zeros((420, 599, 3), dtype=torch.uint8, device=DEV))
        with pytest.raises(binding.PanoError):
            rig.set_tuning(0, 5)
        with pytest.raises(binding.PanoError):
            rig.set_tuning(GEOM["levels"], binding.PANO_LK_AUTO)
        with pytest.raises(binding.PanoError):
            rig.set_tuning(0, binding.PANO_LK_TILE, tile_w=512, tile_h=512)   # shared memory


@pytest.mark.slow
def test_full_rig_equals_single_pair_path_and_oracle():
    """8 pairs of 4000 x {800..2000} RGB u8, 6 levels, on the 9000 x 4000
    canvas at columns 1125 k: the rig workload of the benchmark, replayed from
    its graph."""
    widths = synth.RIG_WIDTHS
    geom = dict(h=4000, widths=widths, x0=tuple(1125 * k for k in range(8)), canvas=(4000, 9000), y0=0,
                levels=6)
    pairs = synth.rig_pairs()
    ref = per_pair(pairs, geom)
    with make_rig(pairs, geom) as rig:
        canvas = rig.new_canvas()
        Ls, Rs = [cuda(p.L) for p in pairs], [cuda(p.R) for p in pairs]
        rig.run(Ls, Rs, canvas=canvas, use_graph=True)
        torch.cuda.synchronize()
        for k in range(8):
            a, b = rig.flows(k)
            assert torch.equal(a, ref[k][0]) and torch.equal(b, ref[k][1]), k
        expect = np.zeros(canvas.shape, np.uint8)
        place(expect, [F.cpu().numpy() for _, _, F in ref], geom)
        assert np.array_equal(canvas.cpu().numpy(), expect)
        prm = oracle.Params(levels=6)
        olr, orl = oracle.flow_pair(pairs[0].L, pairs[0].R, prm)
        lr, rl = (t.cpu().numpy() for t in rig.flows(0))
        assert epe(lr, olr).mean() <= 0.05 and epe(rl, orl).mean() <= 0.05
