"""The u8 RGB blend and the float blend evaluate the same FP32 operations on
the same values (a byte b is the float b), so the u8 result must equal the
float result rounded half to even and clamped, bit for bit: for strips whose
rows start at every byte offset modulo 4 (strided views), and for flows that
clamp samples at every edge."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _u8_of(F):
    return torch.round(F.clamp(0.0, 255.0)).to(torch.uint8)  # torch.round: half to even


@pytest.mark.parametrize("h,w,off,amp", [(67, 131, 0, 3.0), (40, 97, 1, 30.0), (33, 64, 2, 0.7), (21, 255, 3, 300.0),
                                          (1, 9, 1, 2.0), (9, 1, 2, 2.0)])
def test_u8_blend_equals_rounded_float_blend(h, w, off, amp):
    g = np.random.default_rng(h * 1000 + w)
    canvas_L = torch.from_numpy(g.integers(0, 256, (h, w + 4, 3), dtype=np.uint8)).to(DEV)
    canvas_R = torch.from_numpy(g.integers(0, 256, (h, w + 4, 3), dtype=np.uint8)).to(DEV)
    L, R = canvas_L[:, off:off + w], canvas_R[:, off:off + w]        # rows start at byte offset 3 * off
    lr = torch.from_numpy(g.normal(0, amp, (h, w, 2)).astype(np.float32)).to(DEV)
    rl = torch.from_numpy(g.normal(0, amp, (h, w, 2)).astype(np.float32)).to(DEV)
    with binding.FlowContext(binding.Params(), max_h=h, max_w=w, max_c=3) as ctx:
        F8 = ctx.blend_pair(L, R, lr, rl)
        Ff = ctx.blend_pair(L.float().contiguous(), R.float().contiguous(), lr, rl)
        B = torch.from_numpy(g.uniform(0, 1, (h, w)).astype(np.float32)).to(DEV)
        G8 = ctx.blend_pair(L, R, lr, rl, blend=B)
        Gf = ctx.blend_pair(L.float().contiguous(), R.float().contiguous(), lr, rl, blend=B)
    torch.cuda.synchronize()
    assert F8.dtype == torch.uint8 and Ff.dtype == torch.float32
    assert torch.equal(F8, _u8_of(Ff))
    assert torch.equal(G8, _u8_of(Gf))
