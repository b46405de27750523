"""GB300-native frame-group video enhancement (NNVISR's hot path) -- Python binding.

Argument marshalling over the C ABI of ``include/nvisr.h`` (ctypes): every
step of the path runs in libnvisr.so's CUDA kernels.  The library is built
in-tree (``paper_2308_03121_gb300/build.py``); importing this package loads it
and raises if it is missing -- there is no fallback implementation.

Names follow the C ABI (``nvisr_push``, ``nvisr_pull`` ...); ``Engine`` and
``Filter`` wrap them for numpy (host) and torch (device) planes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "Batch", "Engine", "Filter", "NvisrError", "Server", "PREC", "Status", "fmt", "lib", "load",
    "nvisr_conv2d", "nvisr_conv2d_static", "nvisr_dcn2d", "nvisr_resblock2d", "nvisr_fig1_layout", "nvisr_group_outputs",
    "nvisr_group_runs",
    "nvisr_ingest", "nvisr_network_check", "nvisr_requant", "nvisr_selftest",
    "nvisr_tuple_map",
]


class Status:
    OK, AGAIN, FULL, EOS = 0, 1, 2, 3
    INVALID_ARG, UNSUPPORTED_FORMAT, OUT_OF_MEMORY, OVER_BUDGET = -1, -2, -3, -4
    CUDA_ERROR, DEVICE_TIMEOUT, BAD_NETWORK, INTERNAL = -5, -6, -7, -8


PREC = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}
SUB = {"420": 0, "444": 1}
RANGE = {"limited": 0, "full": 1}
LOC = {"left": 0, "center": 1, "point": 2}
SCENE_CUT = 1


class NvisrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


class Format(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
                ("subsampling", ctypes.c_int32), ("range", ctypes.c_int32), ("matrix", ctypes.c_int32),
                ("chroma_loc", ctypes.c_int32), ("transfer", ctypes.c_int32)]


class Planes(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p * 3), ("pitch", ctypes.c_int64 * 3),
                ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("queue_p50_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("admitted", ctypes.c_int64), ("pending", ctypes.c_int64), ("active", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("outputs", ctypes.c_int64), ("deferred_steps", ctypes.c_int64)]


class EngineDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_filters", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class FilterDesc(ctypes.Structure):
    _fields_ = [("network_text", ctypes.c_char_p), ("weights", ctypes.POINTER(ctypes.c_float)),
                ("weights_count", ctypes.c_int64), ("in_fmt", Format), ("out_fmt", Format),
                ("scale_w", ctypes.c_int32), ("scale_h", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("calib_frames", ctypes.c_int32), ("options", ctypes.c_uint32)]


OPT_UNFUSED_OUTPUT = 1
OPT_UNFUSED_BLOCKS = 2
OPT_GUARD_BANDS = 4


class FrameInfo(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("src_first", ctypes.c_int64), ("src_last", ctypes.c_int64),
                ("scene", ctypes.c_int32), ("kind", ctypes.c_int32)]


OUT_NETWORK, OUT_PASSTHROUGH = 0, 1


KINDS = ("ingest", "pack", "conv_head", "conv_body", "conv_tail", "requant", "dcn", "conv_other", "resample")


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(KINDS)), ("launches", ctypes.c_int64 * len(KINDS))]

_LIB = None
_VP, _I32, _I64, _F32P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_float)
_I32P, _U8P = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8)

# name -> (restype, argtypes)
_SIGS = {
    "nvisr_engine_create": (_I32, [ctypes.POINTER(EngineDesc), ctypes.POINTER(_VP)]),
    "nvisr_engine_destroy": (None, [_VP]),
    "nvisr_engine_stream": (_VP, [_VP]),
    "nvisr_engine_bytes_in_use": (_I64, [_VP]),
    "nvisr_filter_create": (_I32, [_VP, ctypes.POINTER(FilterDesc), ctypes.POINTER(_VP)]),
    "nvisr_filter_destroy": (None, [_VP]),
    "nvisr_push": (_I32, [_VP, ctypes.POINTER(Planes), ctypes.c_uint32]),
    "nvisr_flush": (_I32, [_VP]),
    "nvisr_pull": (_I32, [_VP, ctypes.POINTER(Planes), ctypes.POINTER(FrameInfo)]),
    "nvisr_filter_ready": (_I64, [_VP]),
    "nvisr_engine_step": (_I32, [_VP, _I32, _I32P]),
    "nvisr_filter_profile": (_I32, [_VP, _I32]),
    "nvisr_filter_profile_read": (_I32, [_VP, ctypes.POINTER(Profile)]),
    "nvisr_filter_cache_stats": (_I32, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "nvisr_filter_check_guards": (_I32, [_VP, ctypes.POINTER(_I32)]),
    "nvisr_test_poke_guard": (_I32, [_VP, _I32]),
    "nvisr_status_string": (ctypes.c_char_p, [_I32]),
    "nvisr_last_error": (ctypes.c_char_p, [_VP]),
    "nvisr_network_check": (_I32, [ctypes.c_char_p, _I64]),
    "nvisr_ingest": (_I32, [ctypes.POINTER(Format), ctypes.POINTER(Planes), _VP, _I64, _VP]),
    "nvisr_requant": (_I32, [ctypes.POINTER(Format), _VP, _I64, ctypes.POINTER(Planes), _VP]),
    "nvisr_tuple_map": (_I32, [_U8P, _I32, _I32, _I32P]),
    "nvisr_group_runs": (_I32, [_I32, _I32, _I32, _I32, _I32, _I32P, _I32P, _I32P, _I32P]),
    "nvisr_group_outputs": (_I32, [_U8P, _I32, _I32, _I32, _I32, _I32, _I32, _I32P, _I32P, _I32P, _I32P, _I32P]),
    "nvisr_fig1_layout": (_I32, [_I32, _I32, _I32P, _I32P, _I32P]),
    "nvisr_conv2d": (_I32, [_I32, _VP, _I32, _I32, _I32, _VP, _VP, _I32, _I32, _I32, _VP, _VP, _VP]),
    "nvisr_conv2d_static": (_I32, [_I32, _VP, _I32, _I32, _I32, _VP, _VP, _I32, _I32, _I32, _VP, _VP, _VP]),
    "nvisr_resblock2d": (_I32, [_I32, _VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _I32, _VP]),
    "nvisr_dcn2d": (_I32, [_I32, _VP, _I32, _I32, _I32, _VP, _VP, _I32, _VP, _VP, _I32, _VP, _VP]),
    "nvisr_selftest": (_I32, [_I32P, _I32P]),
    "nvisr_test_starve": (_I32, [_I32]),
    "nvisr_selftest_swizzle": (_I32, [_I32P]),
    "nvisr_batch_create": (_I32, [_VP, ctypes.POINTER(_VP), _I32, ctypes.POINTER(_VP)]),
    "nvisr_batch_step": (_I32, [_VP, _I32P]),
    "nvisr_batch_info": (_I32, [_VP, _I32P, _I32P, _I32P]),
    "nvisr_batch_destroy": (None, [_VP]),
    "nvisr_server_create": (_I32, [_VP, _I32, ctypes.POINTER(_VP)]),
    "nvisr_server_submit": (_I32, [_VP, ctypes.POINTER(FilterDesc), ctypes.POINTER(_I64)]),
    "nvisr_server_push": (_I32, [_VP, _I64, ctypes.POINTER(Planes), ctypes.c_uint32]),
    "nvisr_server_flush": (_I32, [_VP, _I64]),
    "nvisr_server_step": (_I32, [_VP, _I32P]),
    "nvisr_server_pull": (_I32, [_VP, _I64, ctypes.POINTER(Planes), ctypes.POINTER(FrameInfo)]),
    "nvisr_server_close": (_I32, [_VP, _I64]),
    "nvisr_server_stats": (_I32, [_VP, ctypes.POINTER(ServerStats)]),
    "nvisr_server_destroy": (None, [_VP]),
    "nvisr_abi_version": (_I32, []),
    "nvisr_build_info": (ctypes.c_char_p, []),
}


def load(build: bool = True):
    """Load libnvisr.so (building it in-tree first when ``build``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libnvisr.so not found at {path}; run paper_2308_03121_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def lib():
    return load()


def _check(status, what):
    if status < 0:
        msg = _LIB.nvisr_last_error(None).decode(errors="replace")
        raise NvisrError(status, f"{what}: {msg}")
    return status


MATRIX = {"bt709": 0, "bt2020": 1, "rgb": 2}
TRANSFER = {"none": 0, "pq": 1, "hlg": 2}


def fmt(width, height, bit_depth, subsampling="420", range_="limited", chroma_loc="left", matrix="bt709",
        transfer="none"):
    return Format(width, height, bit_depth, SUB[subsampling], RANGE[range_], MATRIX[matrix], LOC[chroma_loc],
                  TRANSFER[transfer])


def _ptr(t):
    """Device or host address of a torch tensor or numpy array."""
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _pitch(t):
    return int(t.stride(0) * t.element_size()) if hasattr(t, "stride") and callable(t.stride) else int(t.strides[0])


def planes_of(arrs, on_device):
    p = Planes()
    for i, a in enumerate(arrs):
        p.data[i] = _ptr(a)
        p.pitch[i] = _pitch(a)
    p.on_device = 1 if on_device else 0
    return p


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream) if isinstance(stream, int) else stream.cuda_stream


# ------------------------------------------------------------------ stage entry points

def nvisr_ingest(format_, y, u, v, out_rgb, stream=None):
    """Device planes (torch uint8/int16 tensors) -> out_rgb float32 [3][H][pitch] (torch)."""
    load()
    pl = planes_of((y, u, v), True)
    _check(_LIB.nvisr_ingest(ctypes.byref(format_), ctypes.byref(pl), out_rgb.data_ptr(),
                             out_rgb.stride(1), _stream_ptr(stream)), "nvisr_ingest")


def nvisr_requant(format_, rgb, y, u, v, stream=None):
    load()
    pl = planes_of((y, u, v), True)
    _check(_LIB.nvisr_requant(ctypes.byref(format_), rgb.data_ptr(), rgb.stride(1), ctypes.byref(pl),
                              _stream_ptr(stream)), "nvisr_requant")


def nvisr_conv2d(precision, x, weight, bias, act=0, res=None, stream=None):
    """x [cin][H][W] float32 cuda -> y [cout][H][W]; weight [cout][cin][k][k]."""
    import torch
    load()
    cin, h, w = x.shape
    cout, _, k, _ = weight.shape
    y = torch.empty((cout, h, w), dtype=torch.float32, device=x.device)
    _check(_LIB.nvisr_conv2d(PREC.get(precision, precision), x.data_ptr(), cin, h, w, weight.data_ptr(),
                             bias.data_ptr() if bias is not None else None, cout, k, act,
                             res.data_ptr() if res is not None else None, y.data_ptr(), _stream_ptr(stream)),
           "nvisr_conv2d")
    return y


def nvisr_conv2d_static(precision, x, weight, bias, act=0, res=None, stream=None, out=None):
    """nvisr_conv2d through the allocation-free entry point (fixed device scratch area).
    out: optional preallocated [cout][H][W] float32 cuda tensor."""
    load()
    cin, h, w = x.shape
    cout, _, k, _ = weight.shape
    if out is None:
        import torch
        out = torch.empty((cout, h, w), dtype=torch.float32, device=x.device)
    _check(_LIB.nvisr_conv2d_static(PREC.get(precision, precision), x.data_ptr(), cin, h, w, weight.data_ptr(),
                                    bias.data_ptr() if bias is not None else None, cout, k, act,
                                    res.data_ptr() if res is not None else None, out.data_ptr(),
                                    _stream_ptr(stream)), "nvisr_conv2d_static")
    return out


def nvisr_resblock2d(precision, x, w1, b1, w2, b2, fused=True, stream=None):
    """x [64][H][W] float32 cuda -> x + conv2(LeakyReLU(conv1(x) + b1)) + b2; w1, w2 [64][64][3][3].
    fused: one launch of 2-CTA clusters (else two single-layer launches)."""
    import torch
    load()
    _, h, w = x.shape
    y = torch.empty_like(x)
    _check(_LIB.nvisr_resblock2d(PREC.get(precision, precision), x.data_ptr(), h, w, w1.data_ptr(),
                                 b1.data_ptr() if b1 is not None else None, w2.data_ptr(),
                                 b2.data_ptr() if b2 is not None else None, y.data_ptr(), 1 if fused else 0,
                                 _stream_ptr(stream)), "nvisr_resblock2d")
    return y


def nvisr_dcn2d(precision, x, offsets, mask, weight, bias, groups, stream=None):
    import torch
    load()
    cin, h, w = x.shape
    cout = weight.shape[0]
    y = torch.empty((cout, h, w), dtype=torch.float32, device=x.device)
    _check(_LIB.nvisr_dcn2d(PREC.get(precision, precision), x.data_ptr(), cin, h, w, offsets.data_ptr(),
                            mask.data_ptr(), groups, weight.data_ptr(),
                            bias.data_ptr() if bias is not None else None, cout, y.data_ptr(),
                            _stream_ptr(stream)), "nvisr_dcn2d")
    return y


def nvisr_tuple_map(flags, T):
    load()
    flags = np.ascontiguousarray(np.asarray(flags, np.uint8))
    out = np.zeros((len(flags), T), np.int32)
    _check(_LIB.nvisr_tuple_map(flags.ctypes.data_as(_U8P), len(flags), T, out.ctypes.data_as(_I32P)),
           "nvisr_tuple_map")
    return out


def nvisr_group_runs(s0, s1, n, extra):
    """[(inputs, skip, count)] of the runs covering scene [s0, s1] (host only)."""
    load()
    need = n + (1 if extra else 0)
    maxr = (s1 - s0) // n + 2
    ins = np.zeros(maxr * need, np.int32)
    skip = np.zeros(maxr, np.int32)
    cnt = np.zeros(maxr, np.int32)
    nr = ctypes.c_int32(0)
    _check(_LIB.nvisr_group_runs(s0, s1, n, int(extra), maxr, ins.ctypes.data_as(_I32P),
                                 skip.ctypes.data_as(_I32P), cnt.ctypes.data_as(_I32P), ctypes.byref(nr)),
           "nvisr_group_runs")
    return [(list(map(int, ins[i * need:(i + 1) * need])), int(skip[i]), int(cnt[i])) for i in range(nr.value)]


def nvisr_group_outputs(flags, n, extra, interp, double):
    """Every output of a flushed group-network stream: [(kind, src_first, src_last, net_k)] (host only)."""
    load()
    flags = np.ascontiguousarray(np.asarray(flags, np.uint8))
    cap = 2 * len(flags) + 1
    arrs = [np.zeros(cap, np.int32) for _ in range(4)]
    nout = ctypes.c_int32(0)
    _check(_LIB.nvisr_group_outputs(flags.ctypes.data_as(_U8P), len(flags), n, int(extra), int(interp),
                                    int(double), cap, *[a.ctypes.data_as(_I32P) for a in arrs],
                                    ctypes.byref(nout)), "nvisr_group_outputs")
    return [tuple(int(a[o]) for a in arrs) for o in range(nout.value)]


def nvisr_fig1_layout(n, b):
    load()
    cells = np.zeros((n + 1) * b, np.int32)
    slots = np.zeros(n + 1, np.int32)
    copy = np.zeros(2, np.int32)
    _check(_LIB.nvisr_fig1_layout(n, b, cells.ctypes.data_as(_I32P), slots.ctypes.data_as(_I32P),
                                  copy.ctypes.data_as(_I32P)), "nvisr_fig1_layout")
    return cells, slots, copy


def nvisr_network_check(text, count):
    load()
    st = _LIB.nvisr_network_check(text.encode(), int(count))
    return st, _LIB.nvisr_last_error(None).decode()


def nvisr_test_starve(on):
    """Fault drill (tests only): tensor-core kernels of this thread load no input while on."""
    load()
    _check(_LIB.nvisr_test_starve(1 if on else 0), "nvisr_test_starve")


def nvisr_selftest():
    load()
    a, b = ctypes.c_int32(-1), ctypes.c_int32(-1)
    _check(_LIB.nvisr_selftest(ctypes.byref(a), ctypes.byref(b)), "nvisr_selftest")
    return a.value, b.value


def nvisr_selftest_swizzle():
    load()
    out = np.zeros(16, np.int32)
    _check(_LIB.nvisr_selftest_swizzle(out.ctypes.data_as(_I32P)), "nvisr_selftest_swizzle")
    return out


# ------------------------------------------------------------------ engine / filter

class Engine:
    """One GPU's engine: owns the stream, the HBM budget and its filters."""

    def __init__(self, device=0, hbm_budget_bytes=0, max_filters=0, stream=None):
        load()
        d = EngineDesc(device, max_filters, int(hbm_budget_bytes), stream)
        h = ctypes.c_void_p()
        _check(_LIB.nvisr_engine_create(ctypes.byref(d), ctypes.byref(h)), "nvisr_engine_create")
        self.h = h
        self.filters = []

    @property
    def stream(self):
        return _LIB.nvisr_engine_stream(self.h)

    def bytes_in_use(self):
        return int(_LIB.nvisr_engine_bytes_in_use(self.h))

    def last_error(self):
        """Message of the most recent failed call on this engine or its filters."""
        return _LIB.nvisr_last_error(self.h).decode(errors="replace")

    def step(self, max_outputs=1 << 30):
        n = ctypes.c_int32(0)
        _check(_LIB.nvisr_engine_step(self.h, max_outputs, ctypes.byref(n)), "nvisr_engine_step")
        return n.value

    def filter(self, net_text, blob, in_fmt, out_fmt, precision="fp32", scale=2, calib_frames=0, options=0):
        return Filter(self, net_text, blob, in_fmt, out_fmt, precision, scale, calib_frames, options)

    def batch(self, filters):
        return Batch(self, filters)

    def close(self):
        if self.h:
            for b in list(getattr(self, "batches", [])):
                b.close()
            for f in self.filters:
                f.h = None
            self.filters = []
            _LIB.nvisr_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched multi-stream stepping over filters of one engine (shared launches + CUDA graphs)."""

    def __init__(self, engine, filters):
        self.engine = engine
        self.filters = list(filters)
        arr = (_VP * len(self.filters))(*[f.h for f in self.filters])
        h = ctypes.c_void_p()
        _check(_LIB.nvisr_batch_create(engine.h, arr, len(self.filters), ctypes.byref(h)), "nvisr_batch_create")
        self.h = h
        if not hasattr(engine, "batches"):
            engine.batches = []
        engine.batches.append(self)

    def step(self):
        n = ctypes.c_int32(0)
        _check(_LIB.nvisr_batch_step(self.h, ctypes.byref(n)), "nvisr_batch_step")
        return n.value

    def info(self):
        s, g, r = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(_LIB.nvisr_batch_info(self.h, ctypes.byref(s), ctypes.byref(g), ctypes.byref(r)), "nvisr_batch_info")
        return {"shared": bool(s.value), "graphs": g.value, "rows_per_strip": r.value}

    def close(self):
        if self.h:
            _LIB.nvisr_batch_destroy(self.h)
            self.h = None
            if self in getattr(self.engine, "batches", []):
                self.engine.batches.remove(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving runtime on one engine: submit clips at any time; admitted clips share batched steps."""

    def __init__(self, engine, max_active=0):
        self.engine = engine
        h = ctypes.c_void_p()
        _check(_LIB.nvisr_server_create(engine.h, max_active, ctypes.byref(h)), "nvisr_server_create")
        self.h = h
        self.fmts = {}

    def submit(self, net_text, blob, in_fmt, out_fmt, precision="bf16", scale=2, calib_frames=0):
        blob = np.ascontiguousarray(np.asarray(blob, np.float32))
        text = net_text.encode()
        sw, sh = scale if isinstance(scale, tuple) else (scale, scale)  # (horizontal, vertical)
        d = FilterDesc(text, blob.ctypes.data_as(_F32P), blob.size, in_fmt, out_fmt, sw, sh,
                       PREC[precision] if isinstance(precision, str) else precision, calib_frames, 0)
        cid = ctypes.c_int64(0)
        _check(_LIB.nvisr_server_submit(self.h, ctypes.byref(d), ctypes.byref(cid)), "nvisr_server_submit")
        self.fmts[cid.value] = out_fmt
        return cid.value

    def push(self, clip, planes, cut=False):
        dev = hasattr(planes[0], "is_cuda") and planes[0].is_cuda
        p = planes_of(planes, dev)
        return _check(_LIB.nvisr_server_push(self.h, clip, ctypes.byref(p), SCENE_CUT if cut else 0),
                      "nvisr_server_push")

    def flush(self, clip):
        return _check(_LIB.nvisr_server_flush(self.h, clip), "nvisr_server_flush")

    def step(self):
        n = ctypes.c_int32(0)
        _check(_LIB.nvisr_server_step(self.h, ctypes.byref(n)), "nvisr_server_step")
        return n.value

    def pull(self, clip, out):
        dev = hasattr(out[0], "is_cuda") and out[0].is_cuda
        p = planes_of(out, dev)
        info = FrameInfo()
        st = _check(_LIB.nvisr_server_pull(self.h, clip, ctypes.byref(p), ctypes.byref(info)), "nvisr_server_pull")
        return st, info

    def alloc_out_host(self, clip):
        f = self.fmts[clip]
        dt = np.uint8 if f.bit_depth <= 8 else np.uint16
        cw, ch = (f.width // 2, f.height // 2) if f.subsampling == 0 else (f.width, f.height)
        return (np.zeros((f.height, f.width), dt), np.zeros((ch, cw), dt), np.zeros((ch, cw), dt))

    def close_clip(self, clip):
        _check(_LIB.nvisr_server_close(self.h, clip), "nvisr_server_close")
        self.fmts.pop(clip, None)

    def stats(self):
        st = ServerStats()
        _check(_LIB.nvisr_server_stats(self.h, ctypes.byref(st)), "nvisr_server_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _LIB.nvisr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Filter:
    """A filter: push integer frames, pull enhanced frames in presentation order."""

    def __init__(self, engine, net_text, blob, in_fmt, out_fmt, precision="fp32", scale=2, calib_frames=0,
                 options=0):
        self.engine = engine
        self._blob = np.ascontiguousarray(np.asarray(blob, np.float32))
        self._text = net_text.encode()
        sw, sh = scale if isinstance(scale, tuple) else (scale, scale)  # (horizontal, vertical)
        d = FilterDesc(self._text, self._blob.ctypes.data_as(_F32P), self._blob.size, in_fmt, out_fmt,
                       sw, sh, PREC[precision] if isinstance(precision, str) else precision, calib_frames, options)
        h = ctypes.c_void_p()
        _check(_LIB.nvisr_filter_create(engine.h, ctypes.byref(d), ctypes.byref(h)), "nvisr_filter_create")
        self.h = h
        self.in_fmt, self.out_fmt = in_fmt, out_fmt
        engine.filters.append(self)

    def push(self, planes, cut=False):
        """planes: (Y, U, V) numpy arrays (host) or torch cuda tensors (device)."""
        dev = hasattr(planes[0], "is_cuda") and planes[0].is_cuda
        p = planes_of(planes, dev)
        return _check(_LIB.nvisr_push(self.h, ctypes.byref(p), SCENE_CUT if cut else 0), "nvisr_push")

    def flush(self):
        _check(_LIB.nvisr_flush(self.h), "nvisr_flush")

    def ready(self):
        return int(_LIB.nvisr_filter_ready(self.h))

    def pull(self, out):
        """out: (Y, U, V) numpy arrays or torch cuda tensors; returns (status, FrameInfo)."""
        dev = hasattr(out[0], "is_cuda") and out[0].is_cuda
        p = planes_of(out, dev)
        info = FrameInfo()
        st = _check(_LIB.nvisr_pull(self.h, ctypes.byref(p), ctypes.byref(info)), "nvisr_pull")
        return st, info

    def profile(self, enable=True):
        _check(_LIB.nvisr_filter_profile(self.h, 1 if enable else 0), "nvisr_filter_profile")

    def check_guards(self):
        """Number of buffers whose guard bands were overwritten (filters created
        with OPT_GUARD_BANDS); 0 when every band holds its pattern."""
        bad = _I32(0)
        st = _LIB.nvisr_filter_check_guards(self.h, ctypes.byref(bad))
        if st not in (Status.OK, Status.CUDA_ERROR):
            _check(st, "nvisr_filter_check_guards")
        return bad.value

    def poke_guard(self, index):
        _check(_LIB.nvisr_test_poke_guard(self.h, index), "nvisr_test_poke_guard")

    def cache_stats(self):
        """(hits, misses) of the extract-stage cache (two-frame group networks)."""
        h, m = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(_LIB.nvisr_filter_cache_stats(self.h, ctypes.byref(h), ctypes.byref(m)), "nvisr_filter_cache_stats")
        return h.value, m.value

    def profile_read(self):
        """{kind: (total ms, launches)} since profiling was enabled."""
        p = Profile()
        _check(_LIB.nvisr_filter_profile_read(self.h, ctypes.byref(p)), "nvisr_filter_profile_read")
        return {k: (p.ms[i], int(p.launches[i])) for i, k in enumerate(KINDS)}

    def alloc_out_host(self):
        f = self.out_fmt
        dt = np.uint8 if f.bit_depth <= 8 else np.uint16
        cw, ch = (f.width // 2, f.height // 2) if f.subsampling == 0 else (f.width, f.height)
        return (np.zeros((f.height, f.width), dt), np.zeros((ch, cw), dt), np.zeros((ch, cw), dt))

    def close(self):
        if self.h:
            for b in list(getattr(self.engine, "batches", [])):
                if self in b.filters:
                    b.close()
            _LIB.nvisr_filter_destroy(self.h)
            self.h = None
            if self in self.engine.filters:
                self.engine.filters.remove(self)
