"""PANO_DEBUG: the allocation-failure path of the create calls (a failure
made on the host, no GPU fault) and the synchronising debug mode."""
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpu_build.build()
    binding.load_library()


def test_failed_device_allocation_is_reported_and_recoverable(monkeypatch):
    monkeypatch.setenv("PANO_DEBUG", "fail_alloc")
    with pytest.raises(binding.PanoError) as ei:
        binding.FlowContext(binding.Params(levels=3), 64, 64, 1)
    assert ei.value.status == binding.PANO_ERR_OOM and "cudaMalloc" in ei.value.message
    with pytest.raises(binding.PanoError) as ei:
        binding.Rig(binding.Params(levels=3), 64, [32, 40], canvas_hw=(64, 100), canvas_x0=[0, 50])
    assert ei.value.status == binding.PANO_ERR_OOM
    monkeypatch.setenv("PANO_DEBUG", "")
    with binding.FlowContext(binding.Params(levels=3), 64, 64, 1) as ctx:
        z = torch.zeros((64, 64), dtype=torch.float32, device=DEV)
        lr, rl = ctx.flow_pair(z, z)
        torch.cuda.synchronize()
        assert torch.count_nonzero(lr) == 0


def test_sync_mode_gives_the_same_results(monkeypatch):
    pair = synth.pair_small_gray(h=96, w=128, levels=3)
    L, R = torch.from_numpy(pair.L).to(DEV), torch.from_numpy(pair.R).to(DEV)
    with binding.FlowContext(binding.Params(levels=3), 96, 128, 1) as ctx:
        ref = ctx.stitch_pair(L, R)
        torch.cuda.synchronize()
        monkeypatch.setenv("PANO_DEBUG", "sync,unknown_word")
        got = ctx.stitch_pair(L, R)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    with binding.Rig(binding.Params(levels=3), 96, [128], c=1, dtype=torch.float32, canvas_hw=(96, 128),
                     canvas_x0=[0]) as rig:
        canvas = rig.new_canvas()
        rig.run([L], [R], canvas=canvas)                 # eager, synchronised per call
        rig.run([L], [R], canvas=canvas, use_graph=True)  # capture: no synchronisation inside it
        torch.cuda.synchronize()
        assert torch.equal(canvas, ref[2])
