"""ctypes binding of ``libpanoflow.so`` (the C ABI in ``include/pano_flow.h``
and ``include/pano_rig.h``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch supplies device memory (tensors) and streams. There is no
fallback: if the library is missing, loading raises ``PanoError``.

Tensor conventions
  * an image is a CUDA tensor (H, W) or (H, W, C), C in {1, 3}, dtype uint8
    or float32, whose channels and columns are contiguous (stride(-1) == 1
    and stride(1) == C); any row stride is accepted;
  * a flow is a contiguous float32 CUDA tensor (H, W, 2), [..., 0] = column
    offset, [..., 1] = row offset; FlowAtoB lives on A's grid with
    A(p) ~ B(p + FlowAtoB(p)).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpanoflow.so")

PANO_OK, PANO_ERR_INVALID_ARG, PANO_ERR_UNSUPPORTED, PANO_ERR_OOM, PANO_ERR_CUDA, PANO_ERR_TIMEOUT = range(6)
PANO_U8, PANO_F32, PANO_BF16, PANO_F16 = range(4)

STATUS_NAMES = {0: "PANO_OK", 1: "PANO_ERR_INVALID_ARG", 2: "PANO_ERR_UNSUPPORTED", 3: "PANO_ERR_OOM",
                4: "PANO_ERR_CUDA", 5: "PANO_ERR_TIMEOUT"}

# Every function the header declares, with its ctypes signature.
_VP, _I, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float


class PanoImage(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("h", ctypes.c_int), ("w", ctypes.c_int), ("c", ctypes.c_int),
                ("pitch_bytes", ctypes.c_size_t), ("dtype", ctypes.c_int)]


class PanoParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("iters", ctypes.c_int), ("radius", ctypes.c_int),
                ("lam", ctypes.c_float), ("soft_sharpness", ctypes.c_float),
                ("flow_mag_coef", ctypes.c_float), ("pyr_dtype", ctypes.c_int)]


class PanoTraceRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("level", ctypes.c_int), ("ms", ctypes.c_float)]


RIG_MAX_PAIRS = 8
PANO_LK_AUTO, PANO_LK_STREAM, PANO_LK_TILE = 0, 1, 2


class PanoRigDesc(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int), ("h", ctypes.c_int), ("w", ctypes.c_int * RIG_MAX_PAIRS),
                ("c", ctypes.c_int), ("dtype", ctypes.c_int), ("canvas_h", ctypes.c_int),
                ("canvas_w", ctypes.c_int), ("canvas_y0", ctypes.c_int),
                ("canvas_x0", ctypes.c_int * RIG_MAX_PAIRS)]


class PanoRigTuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("seg_rows", ctypes.c_int), ("tile_w", ctypes.c_int),
                ("tile_h", ctypes.c_int), ("ms", ctypes.c_float)]


_IMG = ctypes.POINTER(PanoImage)
_PAR = ctypes.POINTER(PanoParams)
_PP = ctypes.POINTER(ctypes.c_void_p)

PANO_TRACE_LUMA, PANO_TRACE_PYR_DOWN, PANO_TRACE_LK, PANO_TRACE_BLEND = 0x1, 0x2, 0x4, 0x8
PANO_TRACE_LUMA_REDUCE = 0x10
PANO_TRACE_PYR_TAIL = 0x20

SIGNATURES = {
    "pano_flow_params_default": ([_PAR], None),
    "pano_flow_create": ([_PAR, _I, _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "pano_flow_pair": ([_VP, _IMG, _IMG, _VP, _VP, _VP], _I),
    "pano_blend_pair": ([_VP, _IMG, _IMG, _VP, _VP, _VP, _IMG, _VP], _I),
    "pano_debug_bounds": ([ctypes.POINTER(ctypes.c_uint)], _I),
    "pano_compose_pair": ([_PAR, _IMG, _IMG, _VP, ctypes.c_size_t, _VP, _I, _VP, _VP, _I, _I, _I, _I, _IMG, _VP], _I),
    "pano_flow_destroy": ([_VP], _I),
    "pano_last_error": ([_VP], ctypes.c_char_p),
    "pano_trace_enable": ([_VP, ctypes.c_uint, _I], _I),
    "pano_trace_read": ([_VP, ctypes.POINTER(PanoTraceRecord), _I, ctypes.POINTER(ctypes.c_int)], _I),
    "pano_flow_launches": ([_VP], ctypes.c_ulonglong),
    "pano_flow_pair_static": ([_PAR, _IMG, _IMG, _VP, _VP, _VP], _I),
    "pano_energy_grad": ([_VP, _VP, _I, _I, _I, _VP, _F, _VP, _VP, _VP, _VP, _VP], _I),
    "pano_stage_pyr_down_adjoint": ([_VP, _I, _I, _I, _VP, _I, _VP], _I),
    "pano_stage_luma": ([_IMG, _VP, _I, _VP], _I),
    "pano_stage_pyr_down": ([_VP, _I, _I, _I, _VP, _I, _VP], _I),
    "pano_stage_luma_pyr": ([_IMG, _VP, _I, _VP, _I, _VP], _I),
    "pano_stage_pyramid": ([_VP, _I, _I, _I, _PP, ctypes.POINTER(ctypes.c_int), _I, _VP], _I),
    "pano_stage_lk": ([_VP, _VP, _I, _I, _I, _VP, _I, _I, _I, _VP, _I, _I, _F, _VP], _I),
    "pano_stage_lk_kernel": ([_VP, _VP, _I, _I, _I, _VP, _I, _I, _I, _VP, _I, _I, _F, _I, _VP], _I),
    "pano_stage_warp": ([_IMG, _VP, _F, _IMG, _VP], _I),
    "pano_blend_coeff_scratch_bytes": ([_I, _I], ctypes.c_size_t),
    "pano_blend_coeff": ([_VP, _I, _I, ctypes.c_size_t, _VP, _I, _VP, ctypes.c_size_t, _VP], _I),
    "pano_rig_create": ([_PAR, ctypes.POINTER(PanoRigDesc), _PP], _I),
    "pano_rig_run": ([_VP, _IMG, _IMG, _PP, _PP, _IMG, _I, _VP], _I),
    "pano_rig_autotune": ([_VP, _IMG, _IMG, _I, _VP], _I),
    "pano_rig_get_tuning": ([_VP, _I, ctypes.POINTER(PanoRigTuning)], _I),
    "pano_rig_set_tuning": ([_VP, _I, ctypes.POINTER(PanoRigTuning)], _I),
    "pano_rig_flows": ([_VP, _I, _PP, _PP], _I),
    "pano_rig_trace_enable": ([_VP, ctypes.c_uint, _I], _I),
    "pano_rig_trace_read": ([_VP, ctypes.POINTER(PanoTraceRecord), _I, ctypes.POINTER(ctypes.c_int)], _I),
    "pano_rig_launches": ([_VP], ctypes.c_ulonglong),
    "pano_rig_graph_captures": ([_VP], _I),
    "pano_rig_destroy": ([_VP], _I),
}

_lib = None


class PanoError(RuntimeError):
    """A non-OK status from the library, or a missing library."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def open_library(path: str) -> ctypes.CDLL:
    """A library file of this project (the release or the check variant) with
    every C-ABI signature set; does not make it the one the binding uses."""
    if not os.path.exists(path):
        raise PanoError(-1, f"CUDA library not built: {path} is missing "
                            "(run paper_2006_01201_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path)
    return _lib


def debug_bounds():
    """(count, site, index, bound) of the index checks of the check variant
    since the last read (pano_debug_bounds); synchronise before calling."""
    out = (ctypes.c_uint * 4)()
    _check(load_library().pano_debug_bounds(out))
    return tuple(out)


def _check(status: int) -> None:
    if status != PANO_OK:
        msg = load_library().pano_last_error(None)
        raise PanoError(status, msg.decode() if msg else "")


@dataclass
class Params:
    """Mirror of ``pano_flow_params`` (defaults: those of the library)."""

    levels: int = 4
    iters: int = 5
    radius: int = 2
    lam: float = 1e-2
    soft_sharpness: float = 10.0
    flow_mag_coef: float = 20.0
    pyr_dtype: int = PANO_F32     # storage of the pyramid levels: PANO_F32, PANO_BF16 or PANO_F16

    def to_c(self) -> PanoParams:
        return PanoParams(self.levels, self.iters, self.radius, self.lam, self.soft_sharpness,
                          self.flow_mag_coef, self.pyr_dtype)


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def image_desc(t) -> PanoImage:
    """pano_image for an (H, W) or (H, W, C) CUDA tensor."""
    torch = _torch()
    if not t.is_cuda:
        raise PanoError(PANO_ERR_INVALID_ARG, "image tensor must be on a CUDA device")
    if t.dtype == torch.uint8:
        dt, es = PANO_U8, 1
    elif t.dtype == torch.float32:
        dt, es = PANO_F32, 4
    else:
        raise PanoError(PANO_ERR_UNSUPPORTED, f"image dtype {t.dtype}")
    if t.dim() == 2:
        h, w, c = t.shape[0], t.shape[1], 1
        ok = t.stride(1) == 1
    elif t.dim() == 3:
        h, w, c = t.shape
        ok = t.stride(2) == 1 and t.stride(1) == c
    else:
        raise PanoError(PANO_ERR_INVALID_ARG, "image must be (H, W) or (H, W, C)")
    if not ok:
        raise PanoError(PANO_ERR_INVALID_ARG, "image columns and channels must be contiguous")
    pitch = t.stride(0) * es if h > 1 else w * c * es
    return PanoImage(t.data_ptr(), h, w, c, pitch, dt)


def _flow_ptr(f, h, w, name) -> int:
    torch = _torch()
    if f.dtype != torch.float32 or not f.is_cuda or tuple(f.shape) != (h, w, 2) or not f.is_contiguous():
        raise PanoError(PANO_ERR_INVALID_ARG, f"{name} must be a contiguous float32 CUDA tensor of shape {(h, w, 2)}")
    return f.data_ptr()


class FlowContext:
    """A library context: scratch for strips up to max_h x max_w x max_c."""

    def __init__(self, params: Optional[Params] = None, max_h: int = 4096, max_w: int = 4096, max_c: int = 3):
        lib = load_library()
        self.params = params or Params()
        self.max_h, self.max_w, self.max_c = max_h, max_w, max_c
        h = ctypes.c_void_p()
        p = self.params.to_c()
        _check(lib.pano_flow_create(ctypes.byref(p), max_h, max_w, max_c, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load_library().pano_flow_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def flow_pair(self, L, R, out: Optional[Tuple] = None, stream=None):
        """(FlowLtoR, FlowRtoL) of two strips, Section III-C-1."""
        torch = _torch()
        dl, dr = image_desc(L), image_desc(R)
        h, w = dl.h, dl.w
        if out is None:
            out = (torch.empty((h, w, 2), dtype=torch.float32, device=L.device),
                   torch.empty((h, w, 2), dtype=torch.float32, device=L.device))
        lr = _flow_ptr(out[0], h, w, "flow_LtoR")
        rl = _flow_ptr(out[1], h, w, "flow_RtoL")
        _check(load_library().pano_flow_pair(self._h, ctypes.byref(dl), ctypes.byref(dr), lr, rl,
                                             _stream_ptr(stream)))
        return out

    def blend_pair(self, L, R, flow_LtoR, flow_RtoL, blend=None, out=None, stream=None):
        """F of Code 1 (Section III-C-3); blend None means the Eq. (1) strip ramp."""
        torch = _torch()
        dl, dr = image_desc(L), image_desc(R)
        if out is None:
            out = torch.empty_like(L)
        df = image_desc(out)
        bp = None
        if blend is not None:
            if blend.dtype != torch.float32 or not blend.is_contiguous() or tuple(blend.shape) != (dl.h, dl.w):
                raise PanoError(PANO_ERR_INVALID_ARG, "blend must be a contiguous float32 (H, W) tensor")
            bp = blend.data_ptr()
        _check(load_library().pano_blend_pair(
            self._h, ctypes.byref(dl), ctypes.byref(dr), _flow_ptr(flow_LtoR, dl.h, dl.w, "flow_LtoR"),
            _flow_ptr(flow_RtoL, dl.h, dl.w, "flow_RtoL"), bp, ctypes.byref(df), _stream_ptr(stream)))
        return out

    def stitch_pair(self, L, R, stream=None):
        """flow_pair followed by blend_pair; returns (FlowLtoR, FlowRtoL, F)."""
        lr, rl = self.flow_pair(L, R, stream=stream)
        return lr, rl, self.blend_pair(L, R, lr, rl, stream=stream)

    def stitch_canvas(self, L, R, label, crop, blend=None, out=None, stream=None):
        """Section III-C on a canvas, in the paper's order: Blend of Eq. (1) on
        the label canvas (pano_blend_coeff, unless `blend` is given), the flows
        of the overlap crop (pano_flow_pair on the crop of L and R), and
        Code 1 on the whole canvas (pano_compose_pair). crop = (row, column,
        height, width) of the overlap on the canvas, within the context's
        maxima. Returns (FlowLtoR, FlowRtoL, Blend, F)."""
        y0, x0, ch, cw = (int(v) for v in crop)
        if blend is None:
            blend = blend_coeff(label, stream=stream)
        lr, rl = self.flow_pair(L[y0:y0 + ch, x0:x0 + cw], R[y0:y0 + ch, x0:x0 + cw], stream=stream)
        F = compose_pair(L, R, label, blend, lr, rl, origin=(y0, x0), params=self.params, out=out, stream=stream)
        return lr, rl, blend, F

    def stitch_host(self, L_host, R_host, F_host, work, stream=None):
        """Whole path from host strips to a host F on one stream.

        L_host, R_host, F_host: CPU tensors (pinned for asynchronous copies).
        work: dict of preallocated device tensors ``L``, ``R``, ``lr``, ``rl``,
        ``F`` of matching shapes. Enqueues H2D copies, flow_pair, blend_pair
        and the D2H copy of F; returns without synchronising.
        """
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            work["L"].copy_(L_host, non_blocking=True)
            work["R"].copy_(R_host, non_blocking=True)
            self.flow_pair(work["L"], work["R"], out=(work["lr"], work["rl"]), stream=s)
            self.blend_pair(work["L"], work["R"], work["lr"], work["rl"], out=work["F"], stream=s)
            F_host.copy_(work["F"], non_blocking=True)
        return F_host

    def host_pipeline(self, shape, dtype, device="cuda"):
        """A HostPipeline of this context for strips of `shape` and `dtype`."""
        return HostPipeline(self, shape, dtype, device)

    # -- tracing -------------------------------------------------------------

    def trace_enable(self, kind_mask: int, capacity: int) -> None:
        """Bracket launches of the selected kinds with CUDA events."""
        _check(load_library().pano_trace_enable(self._h, kind_mask, capacity))

    def trace_read(self, max_records: int = 4096):
        """[(kind, level, ms), ...] of the launches recorded since the last read."""
        buf = (PanoTraceRecord * max_records)()
        n = ctypes.c_int()
        _check(load_library().pano_trace_read(self._h, buf, max_records, ctypes.byref(n)))
        return [(buf[i].kind, buf[i].level, buf[i].ms) for i in range(n.value)]

    @property
    def launches(self) -> int:
        """Kernel launches enqueued by this context so far."""
        return int(load_library().pano_flow_launches(self._h))


class _Pipeline:
    """Two device buffer sets used in turn. Item k: the host->device copies of
    its inputs run on the input stream once buffer set k % 2 is free again,
    the kernels on the compute stream once its inputs have arrived, and the
    device->host copy of its result on the output stream once they are done;
    so the copies of items k + 1 and k - 1 overlap the kernels of item k.
    Host buffers must be pinned, and each item's host output must stay
    untouched until `wait(k)` (or `drain()`) returns."""

    def __init__(self, bufs, compute_stream=None):
        torch = _torch()
        self.bufs = bufs
        self.s_in = torch.cuda.Stream()
        self.s_out = torch.cuda.Stream()
        self.s_comp = compute_stream if compute_stream is not None else torch.cuda.Stream()
        self.free = [None, None]          # event: buffer set b drained by the output stream
        self.done = {}                    # item -> event recorded after its output copy

    def _submit(self, k, upload, compute, download):
        torch = _torch()
        b = k % 2
        buf = self.bufs[b]
        if self.free[b] is not None:
            self.s_in.wait_event(self.free[b])
        with torch.cuda.stream(self.s_in):
            upload(buf)
            ev_in = torch.cuda.Event()
            ev_in.record(self.s_in)
        self.s_comp.wait_event(ev_in)
        compute(buf, self.s_comp)
        ev_c = torch.cuda.Event()
        ev_c.record(self.s_comp)
        self.s_out.wait_event(ev_c)
        with torch.cuda.stream(self.s_out):
            download(buf)
            ev_out = torch.cuda.Event()
            ev_out.record(self.s_out)
        self.free[b] = ev_out
        self.done[k] = ev_out
        self.done.pop(k - 2, None)
        return ev_out

    def wait(self, k):
        ev = self.done.get(k)
        if ev is not None:
            ev.synchronize()

    def drain(self):
        for ev in list(self.done.values()):
            ev.synchronize()


class HostPipeline(_Pipeline):
    """Strip pairs from pinned host memory to blended strips in pinned host
    memory through one FlowContext, with the copies of neighbouring pairs
    overlapping the kernels of the current one (see _Pipeline)."""

    def __init__(self, ctx: "FlowContext", shape, dtype, device="cuda", compute_stream=None):
        torch = _torch()
        h, w = shape[0], shape[1]
        bufs = [{"L": torch.empty(shape, dtype=dtype, device=device), "R": torch.empty(shape, dtype=dtype, device=device),
                 "lr": torch.empty((h, w, 2), dtype=torch.float32, device=device),
                 "rl": torch.empty((h, w, 2), dtype=torch.float32, device=device),
                 "F": torch.empty(shape, dtype=dtype, device=device)} for _ in range(2)]
        super().__init__(bufs, compute_stream)
        self.ctx = ctx

    def submit(self, k: int, L_host, R_host, F_host):
        """Enqueue pair k; returns the event that completes with its F_host."""
        def upload(buf):
            buf["L"].copy_(L_host, non_blocking=True)
            buf["R"].copy_(R_host, non_blocking=True)

        def compute(buf, s):
            self.ctx.flow_pair(buf["L"], buf["R"], out=(buf["lr"], buf["rl"]), stream=s)
            self.ctx.blend_pair(buf["L"], buf["R"], buf["lr"], buf["rl"], out=buf["F"], stream=s)

        def download(buf):
            F_host.copy_(buf["F"], non_blocking=True)

        return self._submit(k, upload, compute, download)


class RigHostPipeline(_Pipeline):
    """Every pair of a rig from pinned host strips to a pinned host canvas,
    overlapped as HostPipeline does (graph replays on the compute stream)."""

    def __init__(self, rig: "Rig", device="cuda", compute_stream=None):
        torch = _torch()
        shapes = [(rig.h, w, rig.c) if rig.c > 1 else (rig.h, w) for w in rig.widths]
        bufs = [{"L": [torch.empty(sh, dtype=rig.dtype, device=device) for sh in shapes],
                 "R": [torch.empty(sh, dtype=rig.dtype, device=device) for sh in shapes],
                 "canvas": rig.new_canvas(device)} for _ in range(2)]
        super().__init__(bufs, compute_stream)
        self.rig = rig

    def submit(self, k: int, L_hosts, R_hosts, canvas_host, use_graph: bool = True):
        def upload(buf):
            for d, h_ in zip(buf["L"], L_hosts):
                d.copy_(h_, non_blocking=True)
            for d, h_ in zip(buf["R"], R_hosts):
                d.copy_(h_, non_blocking=True)

        def compute(buf, s):
            self.rig.run(buf["L"], buf["R"], canvas=buf["canvas"], use_graph=use_graph, stream=s)

        def download(buf):
            canvas_host.copy_(buf["canvas"], non_blocking=True)

        return self._submit(k, upload, compute, download)


def compose_pair(L, R, label, blend, flow_LtoR, flow_RtoL, origin=(0, 0), params: Optional[Params] = None,
                 out=None, stream=None):
    """Code 1 on a whole canvas (pano_compose_pair): Area1 (label 1) from L,
    Area2 (label 2) from R, Area3 (label 3) blended with the flows of the
    overlap crop whose pixel (0, 0) is canvas pixel `origin`, zero elsewhere.
    L, R: canvas images; label: (H, W) uint8; blend: (H, W) float32 (Eq. 1)."""
    torch = _torch()
    dl, dr = image_desc(L), image_desc(R)
    if out is None:
        out = torch.empty_like(L)
    df = image_desc(out)
    if label.dtype != torch.uint8 or label.dim() != 2 or label.stride(1) != 1:
        raise PanoError(PANO_ERR_INVALID_ARG, "label must be a uint8 (H, W) tensor with contiguous rows")
    if blend.dtype != torch.float32 or blend.dim() != 2 or blend.stride(1) != 1:
        raise PanoError(PANO_ERR_INVALID_ARG, "blend must be a float32 (H, W) tensor with contiguous rows")
    if tuple(label.shape) != (dl.h, dl.w) or tuple(blend.shape) != (dl.h, dl.w):
        raise PanoError(PANO_ERR_INVALID_ARG, "label and blend must have the canvas size")
    for f, n in ((flow_LtoR, "flow_LtoR"), (flow_RtoL, "flow_RtoL")):
        if f.dtype != torch.float32 or f.dim() != 3 or f.shape[2] != 2 or not f.is_contiguous():
            raise PanoError(PANO_ERR_INVALID_ARG, f"{n} must be a contiguous float32 (h, w, 2) tensor")
    if flow_LtoR.shape != flow_RtoL.shape:
        raise PanoError(PANO_ERR_INVALID_ARG, "the two flows differ in size")
    fh, fw = flow_LtoR.shape[0], flow_LtoR.shape[1]
    p = (params or Params()).to_c()
    lp = label.stride(0) if dl.h > 1 else dl.w
    bp = blend.stride(0) if dl.h > 1 else dl.w
    _check(load_library().pano_compose_pair(ctypes.byref(p), ctypes.byref(dl), ctypes.byref(dr), label.data_ptr(),
                                            lp, blend.data_ptr(), bp, flow_LtoR.data_ptr(), flow_RtoL.data_ptr(),
                                            int(origin[0]), int(origin[1]), fh, fw, ctypes.byref(df),
                                            _stream_ptr(stream)))
    return out


def flow_pair_static(params: Params, L, R, out=None, stream=None):
    """(FlowLtoR, FlowRtoL) like FlowContext.flow_pair, without any device allocation
    inside the library: its scratch is a fixed in-library array (strips up to
    about one megapixel). For callers that may not allocate device memory;
    calls that overlap on the GPU share that array and must be ordered."""
    torch = _torch()
    dl, dr = image_desc(L), image_desc(R)
    h, w = dl.h, dl.w
    if out is None:
        out = (torch.empty((h, w, 2), dtype=torch.float32, device=L.device),
               torch.empty((h, w, 2), dtype=torch.float32, device=L.device))
    p = params.to_c()
    _check(load_library().pano_flow_pair_static(ctypes.byref(p), ctypes.byref(dl), ctypes.byref(dr),
                                                _flow_ptr(out[0], h, w, "flow_LtoR"),
                                                _flow_ptr(out[1], h, w, "flow_RtoL"), _stream_ptr(stream)))
    return out


class Rig:
    """Every overlap pair of a 360-degree rig per call (``include/pano_rig.h``).

    widths: strip widths of the pairs (all strips are h rows high); strip k
    lands on canvas columns (canvas_x0[k] + x) mod canvas_w, rows canvas_y0..;
    where spans overlap, the pair with the higher index writes the canvas.
    """

    def __init__(self, params: Optional[Params], h: int, widths, c: int = 3, dtype=None,
                 canvas_hw: Tuple[int, int] = (4000, 9000), canvas_x0=None, canvas_y0: int = 0):
        torch = _torch()
        lib = load_library()
        self.params = params or Params()
        self.h, self.widths, self.c = h, list(widths), c
        self.dtype = dtype if dtype is not None else torch.uint8
        n = len(self.widths)
        if not 1 <= n <= RIG_MAX_PAIRS:
            raise PanoError(PANO_ERR_INVALID_ARG, f"{n} pairs (1..{RIG_MAX_PAIRS})")
        self.canvas_hw = tuple(canvas_hw)
        self.canvas_x0 = list(canvas_x0) if canvas_x0 is not None else [0] * n
        self.canvas_y0 = canvas_y0
        d = PanoRigDesc()
        d.n_pairs, d.h, d.c = n, h, c
        d.dtype = PANO_U8 if self.dtype == torch.uint8 else PANO_F32
        d.canvas_h, d.canvas_w = self.canvas_hw
        d.canvas_y0 = canvas_y0
        for k in range(n):
            d.w[k] = self.widths[k]
            d.canvas_x0[k] = self.canvas_x0[k]
        self.desc = d
        hdl = ctypes.c_void_p()
        p = self.params.to_c()
        _check(lib.pano_rig_create(ctypes.byref(p), ctypes.byref(d), ctypes.byref(hdl)))
        self._h = hdl

    @property
    def n_pairs(self) -> int:
        return len(self.widths)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load_library().pano_rig_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _strips(self, Ls, Rs):
        if len(Ls) != self.n_pairs or len(Rs) != self.n_pairs:
            raise PanoError(PANO_ERR_INVALID_ARG, f"expected {self.n_pairs} L and R strips")
        L = (PanoImage * self.n_pairs)(*[image_desc(t) for t in Ls])
        R = (PanoImage * self.n_pairs)(*[image_desc(t) for t in Rs])
        return L, R

    def new_canvas(self, device="cuda"):
        torch = _torch()
        hc, wc = self.canvas_hw
        shape = (hc, wc, self.c) if self.c > 1 else (hc, wc)
        return torch.zeros(shape, dtype=self.dtype, device=device)

    def run(self, Ls, Rs, flows=None, canvas=None, use_graph: bool = False, stream=None):
        """Flows of every pair (list of (FlowLtoR, FlowRtoL) tensors, or None to keep
        them in the rig) and, with a canvas tensor, the blended strips placed on it."""
        L, R = self._strips(Ls, Rs)
        lr = rl = None
        if flows is not None:
            if len(flows) != self.n_pairs:
                raise PanoError(PANO_ERR_INVALID_ARG, f"expected {self.n_pairs} flow pairs")
            lr = (ctypes.c_void_p * self.n_pairs)(*[_flow_ptr(f[0], self.h, w, "flow_LtoR")
                                                     for f, w in zip(flows, self.widths)])
            rl = (ctypes.c_void_p * self.n_pairs)(*[_flow_ptr(f[1], self.h, w, "flow_RtoL")
                                                     for f, w in zip(flows, self.widths)])
        dc = ctypes.byref(image_desc(canvas)) if canvas is not None else None
        _check(load_library().pano_rig_run(self._h, L, R, lr, rl, dc, int(bool(use_graph)), _stream_ptr(stream)))
        return canvas

    def run_host(self, L_host, R_host, canvas_host, work, use_graph: bool = True, stream=None):
        """Whole rig from host strips to a host canvas on one stream: H2D copies of
        every strip into ``work["L"]``/``work["R"]`` (lists of device tensors), the
        rig run into ``work["canvas"]`` and the D2H copy of the canvas. Returns
        without synchronising."""
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            for dst, src in zip(work["L"], L_host):
                dst.copy_(src, non_blocking=True)
            for dst, src in zip(work["R"], R_host):
                dst.copy_(src, non_blocking=True)
            self.run(work["L"], work["R"], canvas=work["canvas"], use_graph=use_graph, stream=s)
            canvas_host.copy_(work["canvas"], non_blocking=True)
        return canvas_host

    def flows(self, k: int, copy: bool = True):
        """(FlowLtoR, FlowRtoL) of pair k kept in the rig: copies, or (copy=False)
        views of the rig's buffers, valid while the rig lives."""
        torch = _torch()
        a, b = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load_library().pano_rig_flows(self._h, k, ctypes.byref(a), ctypes.byref(b)))
        shape = (self.h, self.widths[k], 2)
        out = tuple(torch.as_tensor(_DeviceArray(ptr, shape), device="cuda") for ptr in (a.value, b.value))
        return tuple(t.clone() for t in out) if copy else out

    def autotune(self, Ls, Rs, reps: int = 5, stream=None):
        L, R = self._strips(Ls, Rs)
        _check(load_library().pano_rig_autotune(self._h, L, R, reps, _stream_ptr(stream)))
        return [self.get_tuning(l) for l in range(self.params.levels)]

    def get_tuning(self, level: int) -> dict:
        t = PanoRigTuning()
        _check(load_library().pano_rig_get_tuning(self._h, level, ctypes.byref(t)))
        return {"kernel": t.kernel, "seg_rows": t.seg_rows, "tile_w": t.tile_w, "tile_h": t.tile_h, "ms": t.ms}

    def set_tuning(self, level: int, kernel: int = PANO_LK_AUTO, seg_rows: int = 0, tile_w: int = 0,
                   tile_h: int = 0) -> None:
        t = PanoRigTuning(kernel, seg_rows, tile_w, tile_h, 0.0)
        _check(load_library().pano_rig_set_tuning(self._h, level, ctypes.byref(t)))

    def trace_enable(self, kind_mask: int, capacity: int) -> None:
        _check(load_library().pano_rig_trace_enable(self._h, kind_mask, capacity))

    def trace_read(self, max_records: int = 4096):
        buf = (PanoTraceRecord * max_records)()
        n = ctypes.c_int()
        _check(load_library().pano_rig_trace_read(self._h, buf, max_records, ctypes.byref(n)))
        return [(buf[i].kind, buf[i].level, buf[i].ms) for i in range(n.value)]

    @property
    def launches(self) -> int:
        return int(load_library().pano_rig_launches(self._h))

    @property
    def graph_captures(self) -> int:
        return int(load_library().pano_rig_graph_captures(self._h))


AREA1, AREA2, AREA3 = 1, 2, 3   # labels of pano_blend_coeff


def blend_coeff(label, out=None, scratch=None, stream=None):
    """Eq. (1) on a labelled canvas: label is a uint8 CUDA tensor (H, W) with
    1 = Area1, 2 = Area2, 3 = Area3 (overlap), other = neither; returns the
    float32 (H, W) Blend array. scratch: optional uint8 device tensor of
    pano_blend_coeff_scratch_bytes(H, W) bytes, reused across calls."""
    torch = _torch()
    if label.dtype != torch.uint8 or label.dim() != 2 or not label.is_cuda or label.stride(1) != 1:
        raise PanoError(PANO_ERR_INVALID_ARG, "label must be a uint8 (H, W) CUDA tensor with contiguous rows")
    h, w = label.shape
    lib = load_library()
    need = int(lib.pano_blend_coeff_scratch_bytes(h, w))
    if out is None:
        out = torch.empty((h, w), dtype=torch.float32, device=label.device)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=label.device)
    if out.dtype != torch.float32 or out.dim() != 2 or out.stride(1) != 1 or tuple(out.shape) != (h, w):
        raise PanoError(PANO_ERR_INVALID_ARG, "out must be a float32 (H, W) tensor with contiguous rows")
    lp = label.stride(0) if h > 1 else w
    bp = out.stride(0) if h > 1 else w
    _check(lib.pano_blend_coeff(label.data_ptr(), h, w, lp, out.data_ptr(), bp, scratch.data_ptr(),
                                scratch.numel() * scratch.element_size(), _stream_ptr(stream)))
    return out


class _DeviceArray:
    """A float32 device buffer of the library, exposed through the CUDA array
    interface so that torch can view it without a copy."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


# ---------------------------------------------------------------------------
# Stage entry points
# ---------------------------------------------------------------------------

def stage_luma(img, stream=None):
    torch = _torch()
    d = image_desc(img)
    Y = torch.empty((d.h, d.w), dtype=torch.float32, device=img.device)
    _check(load_library().pano_stage_luma(ctypes.byref(d), Y.data_ptr(), d.w, _stream_ptr(stream)))
    return Y


def stage_luma_pyr(img, stream=None):
    """(level 0, level 1) of an image in one launch, as the flow path forms them."""
    torch = _torch()
    d = image_desc(img)
    Y = torch.empty((d.h, d.w), dtype=torch.float32, device=img.device)
    Y1 = torch.empty(((d.h + 1) // 2, (d.w + 1) // 2), dtype=torch.float32, device=img.device)
    _check(load_library().pano_stage_luma_pyr(ctypes.byref(d), Y.data_ptr(), d.w, Y1.data_ptr(), Y1.shape[1],
                                              _stream_ptr(stream)))
    return Y, Y1


def stage_pyramid(Y, nlev: int, stream=None):
    """[level 1, ..., level nlev-1] of a float32 (H, W) CUDA tensor, with the
    launch sequence of the flow path."""
    torch = _torch()
    if Y.dtype != torch.float32 or Y.dim() != 2 or Y.stride(1) != 1:
        raise PanoError(PANO_ERR_INVALID_ARG, "Y must be a float32 (H, W) tensor with contiguous rows")
    h, w = Y.shape
    outs = []
    for _ in range(nlev - 1):
        h, w = (h + 1) // 2, (w + 1) // 2
        outs.append(torch.empty((h, w), dtype=torch.float32, device=Y.device))
    ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    pitches = (ctypes.c_int * len(outs))(*[o.shape[1] for o in outs])
    pitch = Y.stride(0) if Y.shape[0] > 1 else Y.shape[1]
    _check(load_library().pano_stage_pyramid(Y.data_ptr(), Y.shape[0], Y.shape[1], pitch, ptrs, pitches, nlev,
                                             _stream_ptr(stream)))
    return outs


def stage_pyr_down(src, stream=None):
    torch = _torch()
    if src.dtype != torch.float32 or src.dim() != 2 or src.stride(1) != 1:
        raise PanoError(PANO_ERR_INVALID_ARG, "src must be a float32 (H, W) tensor with contiguous rows")
    h, w = src.shape
    dst = torch.empty(((h + 1) // 2, (w + 1) // 2), dtype=torch.float32, device=src.device)
    _check(load_library().pano_stage_pyr_down(src.data_ptr(), h, w, src.stride(0), dst.data_ptr(),
                                              dst.stride(0), _stream_ptr(stream)))
    return dst


def stage_lk(T, J, flow_in=None, upsample=False, iters=5, radius=2, lam=1e-2, stream=None, kernel=None):
    """One LK level (pano_stage_lk); `kernel` (a PANO_LK_* value) selects the
    kernel through pano_stage_lk_kernel."""
    torch = _torch()
    for t, n in ((T, "T"), (J, "J")):
        if t.dtype != torch.float32 or t.dim() != 2 or not t.is_contiguous():
            raise PanoError(PANO_ERR_INVALID_ARG, f"{n} must be a contiguous float32 (H, W) tensor")
    h, w = T.shape
    if tuple(J.shape) != (h, w):
        raise PanoError(PANO_ERR_INVALID_ARG, "T and J differ in size")
    out = torch.empty((h, w, 2), dtype=torch.float32, device=T.device)
    fin, ih, iw = None, 0, 0
    if flow_in is not None:
        if flow_in.dtype != torch.float32 or not flow_in.is_contiguous() or flow_in.dim() != 3:
            raise PanoError(PANO_ERR_INVALID_ARG, "flow_in must be a contiguous float32 (h, w, 2) tensor")
        ih, iw = flow_in.shape[0], flow_in.shape[1]
        if not upsample and (ih, iw) != (h, w):
            raise PanoError(PANO_ERR_INVALID_ARG, "flow_in must match T unless upsample is set")
        fin = flow_in.data_ptr()
    if kernel is None:
        _check(load_library().pano_stage_lk(T.data_ptr(), J.data_ptr(), h, w, w, fin, ih, iw, int(bool(upsample)),
                                            out.data_ptr(), iters, radius, lam, _stream_ptr(stream)))
    else:
        _check(load_library().pano_stage_lk_kernel(T.data_ptr(), J.data_ptr(), h, w, w, fin, ih, iw,
                                                   int(bool(upsample)), out.data_ptr(), iters, radius, lam,
                                                   int(kernel), _stream_ptr(stream)))
    return out


def stage_warp(src, flow, scale=1.0, stream=None):
    torch = _torch()
    d = image_desc(src)
    dst = torch.empty(src.shape, dtype=torch.float32, device=src.device)
    dd = image_desc(dst)
    _check(load_library().pano_stage_warp(ctypes.byref(d), _flow_ptr(flow, d.h, d.w, "flow"), float(scale),
                                          ctypes.byref(dd), _stream_ptr(stream)))
    return dst


def energy_grad(T, J, u, alpha: float, want_energy=True, want_u=True, want_T=True, want_J=True, stream=None):
    """(E as a float64 0-d tensor or None, dE/du, dE/dT, dE/dJ) on the GPU."""
    torch = _torch()
    for t, n in ((T, "T"), (J, "J")):
        if t.dtype != torch.float32 or t.dim() != 2 or not t.is_contiguous():
            raise PanoError(PANO_ERR_INVALID_ARG, f"{n} must be a contiguous float32 (H, W) tensor")
    h, w = T.shape
    uptr = _flow_ptr(u, h, w, "u")
    dev = T.device
    E = torch.empty((), dtype=torch.float64, device=dev) if want_energy else None
    gu = torch.empty((h, w, 2), dtype=torch.float32, device=dev) if want_u else None
    gt = torch.empty((h, w), dtype=torch.float32, device=dev) if want_T else None
    gj = torch.empty((h, w), dtype=torch.float32, device=dev) if want_J else None
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(load_library().pano_energy_grad(T.data_ptr(), J.data_ptr(), h, w, w, uptr, float(alpha), ptr(E),
                                           ptr(gu), ptr(gt), ptr(gj), _stream_ptr(stream)))
    return E, gu, gt, gj


def stage_pyr_down_adjoint(gdst, h: int, w: int, stream=None):
    """Gradient of the (h, w) input of a REDUCE from the gradient of its output."""
    torch = _torch()
    if gdst.dtype != torch.float32 or tuple(gdst.shape) != ((h + 1) // 2, (w + 1) // 2) or not gdst.is_contiguous():
        raise PanoError(PANO_ERR_INVALID_ARG, "gdst must be a contiguous float32 (ceil(h/2), ceil(w/2)) tensor")
    out = torch.empty((h, w), dtype=torch.float32, device=gdst.device)
    _check(load_library().pano_stage_pyr_down_adjoint(gdst.data_ptr(), h, w, gdst.shape[1], out.data_ptr(), w,
                                                      _stream_ptr(stream)))
    return out
