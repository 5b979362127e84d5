"""Thin ctypes binding of libgattn (include/gattn.h): STORM global propagation
attention (STORM-GPA, arXiv 2604.16590, Sec. III-C) on GB300.

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels.  PyTorch is used for device memory and streams.  There is no
fallback: if ``libgattn.so`` has not been built, importing the library
raises.

The functions ``gattn_*`` mirror the C ABI one to one (same names, same
arguments; tensors may be passed where the C side takes device pointers).
``GlobalAttention`` wraps forward and backward as a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgattn.so")

GATTN_BF16, GATTN_FP32 = 0, 1
GATTN_WINDOW_HANN, GATTN_WINDOW_FLAT = 0, 1
GATTN_FLAG_DEBUG_BOUNDS = 0x1
GATTN_FLAG_TEST_STALL = 0x2

STATUS = {
    0: "GATTN_OK",
    1: "GATTN_ERR_INVALID_ARG",
    2: "GATTN_ERR_UNSUPPORTED",
    3: "GATTN_ERR_WORKSPACE",
    4: "GATTN_ERR_CUDA",
    5: "GATTN_ERR_TIMEOUT",
    6: "GATTN_ERR_OOM",
    7: "GATTN_ERR_BUSY",
    8: "GATTN_ERR_DEVICE_BOUNDS",
    9: "GATTN_ERR_NOT_FOUND",
}
_DTYPES = {"bf16": GATTN_BF16, "fp32": GATTN_FP32, torch.bfloat16: GATTN_BF16, torch.float32: GATTN_FP32}
_TORCH_DTYPE = {GATTN_BF16: torch.bfloat16, GATTN_FP32: torch.float32}


class GattnError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS.get(self.status, self.status)}")


class gattn_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class gattn_serve_cfg(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("Y", ctypes.c_int32),
        ("X", ctypes.c_int32),
        ("core", ctypes.c_int32 * 3),
        ("halo", ctypes.c_int32 * 3),
        ("window", ctypes.c_int32),
        ("steps", ctypes.c_int32),
        ("c", ctypes.c_float),
        ("max_active", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("hbm_budget", ctypes.c_size_t),
    ]


class gattn_request(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("nh", ctypes.c_int32), ("z0", ctypes.c_void_p), ("z0_on_device", ctypes.c_int32)]


class gattn_serve_stats_t(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("admitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("rejected", ctypes.c_int64),
        ("active", ctypes.c_int64),
        ("waiting", ctypes.c_int64),
        ("iterations", ctypes.c_int64),
        ("p50_latency_s", ctypes.c_double),
        ("p99_latency_s", ctypes.c_double),
        ("mean_latency_s", ctypes.c_double),
        ("max_latency_s", ctypes.c_double),
        ("token_steps", ctypes.c_double),
        ("gpu_busy_s", ctypes.c_double),
        ("wall_s", ctypes.c_double),
        ("hbm_in_use", ctypes.c_size_t),
        ("hbm_peak", ctypes.c_size_t),
    ]


class gattn_desc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int32),
        ("nh", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("Y", ctypes.c_int32),
        ("X", ctypes.c_int32),
        ("core", ctypes.c_int32 * 3),
        ("halo", ctypes.c_int32 * 3),
        ("window", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
        ("out_dtype", ctypes.c_int32),
        ("scale", ctypes.c_float),
        ("flags", ctypes.c_uint32),
    ]


class gattn_linear_desc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int32),
        ("nh", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("N", ctypes.c_int64),
        ("in_dtype", ctypes.c_int32),
        ("out_dtype", ctypes.c_int32),
    ]


class gattn_dps_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("sigma_next", ctypes.c_float), ("lam", ctypes.c_float)]


class gattn_compress_desc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int32),
        ("nh", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("S", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
        ("out_dtype", ctypes.c_int32),
        ("scale", ctypes.c_float),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgattn.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_2604_16590_gb300.build` "
            "(the operator has no non-CUDA implementation)"
        )
    lib = ctypes.CDLL(path)
    P, S, D = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(gattn_desc)
    sig = {
        "gattn_abi_version": ([], ctypes.c_int32),
        "gattn_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "gattn_validate": ([D], ctypes.c_int),
        "gattn_num_tiles": ([D], ctypes.c_int64),
        "gattn_block_shape": ([D, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "gattn_saved_bytes": ([D], S),
        "gattn_bwd_workspace_bytes": ([D], S),
        "gattn_fwd": ([D, P, P, P, P, P, S, P], ctypes.c_int),
        "gattn_bwd": ([D, P, P, P, P, P, P, S, P, P, P, P, S, P], ctypes.c_int),
        "gattn_stream_status": ([P], ctypes.c_int),
        "gattn_fwd_noalloc": ([D, P, P, P, P, P], ctypes.c_int),
        "gattn_serve_request_bytes": ([ctypes.POINTER(gattn_serve_cfg), ctypes.c_int32, ctypes.c_int32], S),
        "gattn_serve_create": ([ctypes.POINTER(gattn_serve_cfg), P, ctypes.POINTER(P)], ctypes.c_int),
        "gattn_serve_submit": ([P, ctypes.POINTER(gattn_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "gattn_serve_step": ([P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "gattn_serve_poll": (
            [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), P],
            ctypes.c_int,
        ),
        "gattn_serve_release": ([P, ctypes.c_uint64], ctypes.c_int),
        "gattn_serve_take_async": ([P, ctypes.c_uint64, P], ctypes.c_int),
        "gattn_serve_copied": ([P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "gattn_serve_stats": ([P, ctypes.POINTER(gattn_serve_stats_t)], ctypes.c_int),
        "gattn_serve_destroy": ([P], None),
        "gattn_linear_workspace_bytes": ([ctypes.POINTER(gattn_linear_desc)], S),
        "gattn_linear_fwd": ([ctypes.POINTER(gattn_linear_desc), P, P, P, P, P, S, P], ctypes.c_int),
        "gattn_linear_bwd_workspace_bytes": ([ctypes.POINTER(gattn_linear_desc)], S),
        "gattn_linear_bwd": ([ctypes.POINTER(gattn_linear_desc), P, P, P, P, P, S, P, P, P, P, S, P], ctypes.c_int),
        "gattn_dps_workspace_bytes": ([D], S),
        "gattn_dps_step": ([D, ctypes.POINTER(gattn_dps_params), P, P, P, P, P, P, S, P], ctypes.c_int),
        "gattn_gated_workspace_bytes": ([D], S),
        "gattn_gated_fwd": ([D, P, P, P, P, P, P, P, P, S, P], ctypes.c_int),
        "gattn_compress_workspace_bytes": ([ctypes.POINTER(gattn_compress_desc)], S),
        "gattn_compress_fwd": ([ctypes.POINTER(gattn_compress_desc), P, P, P, P, P, P, S, P], ctypes.c_int),
        "gattn_profile_enable": ([ctypes.c_int32], ctypes.c_int),
        "gattn_profile_read": ([ctypes.POINTER(gattn_kernel_stat), ctypes.c_int32], ctypes.c_int32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _nbytes(x, given):
    if given is not None:
        return int(given)
    return x.numel() * x.element_size()


def make_desc(B, nh, d, grid, core, halo, window="hann", in_dtype="bf16", out_dtype=None, scale=0.0, flags=0):
    """Build a gattn_desc.  grid = (T, Y, X); core/halo along (t, y, x)."""
    desc = gattn_desc()
    desc.B, desc.nh, desc.d = int(B), int(nh), int(d)
    desc.T, desc.Y, desc.X = (int(g) for g in grid)
    for a in range(3):
        desc.core[a] = int(core[a])
        desc.halo[a] = int(halo[a])
    desc.window = GATTN_WINDOW_HANN if window == "hann" else GATTN_WINDOW_FLAT
    desc.in_dtype = _DTYPES[in_dtype]
    desc.out_dtype = _DTYPES[out_dtype if out_dtype is not None else in_dtype]
    desc.scale = float(scale or 0.0)
    desc.flags = int(flags)
    return desc


# ---------------------------------------------------------------- the C ABI, one to one
def gattn_abi_version() -> int:
    return load_library().gattn_abi_version()


def gattn_status_string(status: int) -> str:
    return load_library().gattn_status_string(int(status)).decode()


def gattn_validate(desc) -> int:
    return load_library().gattn_validate(ctypes.byref(desc))


def gattn_num_tiles(desc) -> int:
    return load_library().gattn_num_tiles(ctypes.byref(desc))


def gattn_block_shape(desc):
    """(status, (bt, by, bx)): the token box the tensor-core kernels use."""
    arr = (ctypes.c_int32 * 3)()
    st = load_library().gattn_block_shape(ctypes.byref(desc), arr)
    return st, (int(arr[0]), int(arr[1]), int(arr[2]))


def gattn_saved_bytes(desc) -> int:
    return load_library().gattn_saved_bytes(ctypes.byref(desc))


def gattn_bwd_workspace_bytes(desc) -> int:
    return load_library().gattn_bwd_workspace_bytes(ctypes.byref(desc))


def gattn_fwd(desc, q, k, v, out, saved, saved_bytes=None, stream=None) -> int:
    return load_library().gattn_fwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(out), _ptr(saved), _nbytes(saved, saved_bytes), _stream(stream)
    )


def gattn_bwd(desc, q, k, v, out, dout, saved, dq, dk, dv, ws, saved_bytes=None, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_bwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(out), _ptr(dout), _ptr(saved), _nbytes(saved, saved_bytes),
        _ptr(dq), _ptr(dk), _ptr(dv), _ptr(ws), _nbytes(ws, ws_bytes), _stream(stream),
    )


GATTN_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def gattn_fwd_noalloc(desc, q, k, v, out, stream=None) -> int:
    """Forward whose scratch is the library's own device array (no allocation);
    see include/gattn.h for the size limit and the sharing rules."""
    return load_library().gattn_fwd_noalloc(ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(out), _stream(stream))


def gattn_stream_status(stream=None) -> int:
    return load_library().gattn_stream_status(_stream(stream))


def gattn_linear_workspace_bytes(desc) -> int:
    return load_library().gattn_linear_workspace_bytes(ctypes.byref(desc))


def gattn_linear_fwd(desc, q, k, v, out, ws, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_linear_fwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(out), _ptr(ws), _nbytes(ws, ws_bytes), _stream(stream)
    )


def gattn_linear_bwd_workspace_bytes(desc) -> int:
    return load_library().gattn_linear_bwd_workspace_bytes(ctypes.byref(desc))


def gattn_linear_bwd(desc, q, k, v, dout, saved, dq, dk, dv, ws, saved_bytes=None, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_linear_bwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(dout), _ptr(saved), _nbytes(saved, saved_bytes),
        _ptr(dq), _ptr(dk), _ptr(dv), _ptr(ws), _nbytes(ws, ws_bytes), _stream(stream),
    )


def linear_desc(q):
    B, nh, N, d = q.shape
    desc = gattn_linear_desc()
    desc.B, desc.nh, desc.d, desc.N = int(B), int(nh), int(d), int(N)
    desc.in_dtype = desc.out_dtype = _DTYPES[q.dtype]
    return desc


def linear_forward(q, k, v, stream=None, keep_summary=False):
    """Factorised linear attention (phi = elu + 1) of BF16 [B, heads, N, 64]
    tensors; with keep_summary, also the workspace that holds the summary the
    backward reads."""
    _require_cuda(q, k, v)
    if not (q.shape == k.shape == v.shape) or q.dtype != torch.bfloat16:
        raise ValueError("q, k, v must be BF16 tensors of one shape [B, heads, N, 64]")
    desc = linear_desc(q)
    out = torch.empty_like(q)
    ws = torch.empty(gattn_linear_workspace_bytes(desc), dtype=torch.uint8, device=q.device)
    check(gattn_linear_fwd(desc, q, k, v, out, ws, stream=stream), "gattn_linear_fwd")
    return (out, ws) if keep_summary else out


def linear_backward(q, k, v, dout, saved, stream=None):
    """(dq, dk, dv) of sum(out * dout) for the factorised linear attention;
    `saved` is the workspace linear_forward(..., keep_summary=True) returned."""
    _require_cuda(q, k, v, dout, saved)
    if dout.shape != q.shape or dout.dtype != torch.bfloat16:
        raise ValueError("dout must be BF16 of the shape of q")
    desc = linear_desc(q)
    dq, dk, dv = torch.empty_like(q), torch.empty_like(q), torch.empty_like(q)
    ws = torch.empty(gattn_linear_bwd_workspace_bytes(desc), dtype=torch.uint8, device=q.device)
    check(gattn_linear_bwd(desc, q, k, v, dout, saved, dq, dk, dv, ws, stream=stream), "gattn_linear_bwd")
    return dq, dk, dv


class LinearAttention(torch.autograd.Function):
    """Factorised linear attention as an autograd op: forward and hand-written
    backward in CUDA (the summary is kept from the forward, feature maps are
    recomputed)."""

    @staticmethod
    def forward(ctx, q, k, v):
        out, saved = linear_forward(q, k, v, keep_summary=True)
        ctx.save_for_backward(q, k, v, saved)
        return out

    @staticmethod
    def backward(ctx, dout):
        q, k, v, saved = ctx.saved_tensors
        return linear_backward(q, k, v, dout.contiguous().to(torch.bfloat16), saved)


def linear_attention(q, k, v):
    return LinearAttention.apply(q, k, v)


def gattn_dps_workspace_bytes(desc) -> int:
    return load_library().gattn_dps_workspace_bytes(ctypes.byref(desc))


def gattn_dps_step(desc, params, z, zb, y, mask, eps, ws, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_dps_step(
        ctypes.byref(desc), ctypes.byref(params), _ptr(z), _ptr(zb), _ptr(y), _ptr(mask), _ptr(eps), _ptr(ws),
        _nbytes(ws, ws_bytes), _stream(stream),
    )


def gattn_gated_workspace_bytes(desc) -> int:
    return load_library().gattn_gated_workspace_bytes(ctypes.byref(desc))


def gattn_gated_fwd(desc, q, k, v, kc, vc, gate, out, ws, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_gated_fwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(kc), _ptr(vc), _ptr(gate), _ptr(out), _ptr(ws),
        _nbytes(ws, ws_bytes), _stream(stream),
    )


def gattn_compress_workspace_bytes(desc) -> int:
    return load_library().gattn_compress_workspace_bytes(ctypes.byref(desc))


def gattn_compress_fwd(desc, q, k, v, out, lse, ws, ws_bytes=None, stream=None) -> int:
    return load_library().gattn_compress_fwd(
        ctypes.byref(desc), _ptr(q), _ptr(k), _ptr(v), _ptr(out), _ptr(lse), _ptr(ws),
        0 if ws is None else _nbytes(ws, ws_bytes), _stream(stream),
    )


def gattn_profile_enable(enable: bool) -> int:
    return load_library().gattn_profile_enable(1 if enable else 0)


def gattn_profile_read() -> dict:
    """{kernel name: (launches, total device ms)} since the last enable."""
    arr = (gattn_kernel_stat * 32)()
    n = load_library().gattn_profile_read(arr, 32)
    if n < 0:
        raise GattnError(-n, "gattn_profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n, 32))}


# ---------------------------------------------------------------- serving ABI, one to one
def gattn_serve_request_bytes(cfg, T, nh) -> int:
    return load_library().gattn_serve_request_bytes(ctypes.byref(cfg), int(T), int(nh))


def gattn_serve_create(cfg, stream=None):
    """Returns (status, server handle); stream None lets the server own a stream."""
    h = ctypes.c_void_p()
    st = load_library().gattn_serve_create(ctypes.byref(cfg), None if stream is None else _stream(stream), ctypes.byref(h))
    return st, h


def gattn_serve_submit(server, req):
    """Returns (status, request id)."""
    rid = ctypes.c_uint64()
    st = load_library().gattn_serve_submit(server, ctypes.byref(req), ctypes.byref(rid))
    return st, rid.value


def gattn_serve_step(server):
    """Returns (status, n_active, n_waiting)."""
    a, w = ctypes.c_int32(), ctypes.c_int32()
    st = load_library().gattn_serve_step(server, ctypes.byref(a), ctypes.byref(w))
    return st, a.value, w.value


def gattn_serve_poll(server, rid, result_host=None):
    """Returns (status, done, latency_s)."""
    done, lat = ctypes.c_int32(), ctypes.c_double()
    st = load_library().gattn_serve_poll(server, ctypes.c_uint64(rid), ctypes.byref(done), ctypes.byref(lat), _ptr(result_host))
    return st, bool(done.value), lat.value


def gattn_serve_release(server, rid) -> int:
    return load_library().gattn_serve_release(server, ctypes.c_uint64(rid))


def gattn_serve_take_async(server, rid, dst) -> int:
    return load_library().gattn_serve_take_async(server, ctypes.c_uint64(rid), _ptr(dst))


def gattn_serve_copied(server, rid):
    """Returns (status, copied)."""
    c = ctypes.c_int32()
    st = load_library().gattn_serve_copied(server, ctypes.c_uint64(rid), ctypes.byref(c))
    return st, bool(c.value)


def gattn_serve_stats(server) -> gattn_serve_stats_t:
    out = gattn_serve_stats_t()
    check(load_library().gattn_serve_stats(server, ctypes.byref(out)), "gattn_serve_stats")
    return out


def gattn_serve_destroy(server) -> None:
    load_library().gattn_serve_destroy(server)


def serve_cfg(d=64, Y=32, X=64, core=(1, 16, 16), halo=(0, 4, 4), window="hann", steps=20, c=0.5, max_active=256,
              use_graph=True, hbm_budget=150 * 10**9):
    cfg = gattn_serve_cfg()
    cfg.d, cfg.Y, cfg.X = int(d), int(Y), int(X)
    for a in range(3):
        cfg.core[a] = int(core[a])
        cfg.halo[a] = int(halo[a])
    cfg.window = GATTN_WINDOW_HANN if window == "hann" else GATTN_WINDOW_FLAT
    cfg.steps, cfg.c, cfg.max_active = int(steps), float(c), int(max_active)
    cfg.use_graph = 1 if use_graph else 0
    cfg.hbm_budget = int(hbm_budget)
    return cfg


class Server:
    """Owns a gattn_server; submit BF16 states (CPU or CUDA tensors [nh, N, d])."""

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        st, self.h = gattn_serve_create(cfg, stream)
        check(st, "gattn_serve_create")
        self._keep = {}
        self._numel = {}  # result size of each submitted request

    def submit(self, z0: torch.Tensor) -> int:
        nh, N, d = z0.shape
        if z0.dtype != torch.bfloat16 or d != self.cfg.d or N % (self.cfg.Y * self.cfg.X):
            raise ValueError("z0 must be BF16 [nh, T*Y*X, d]")
        z0 = z0.contiguous()
        req = gattn_request()
        req.T, req.nh, req.z0 = N // (self.cfg.Y * self.cfg.X), nh, z0.data_ptr()
        req.z0_on_device = 1 if z0.is_cuda else 0
        st, rid = gattn_serve_submit(self.h, req)
        check(st, "gattn_serve_submit")
        if z0.is_cuda:
            self._keep[rid] = z0  # read at admission
        self._numel[rid] = z0.numel()
        return rid

    def step(self):
        st, a, w = gattn_serve_step(self.h)
        check(st, "gattn_serve_step")
        return a, w

    def result(self, rid, shape=None, out=None):
        """(final state, latency) of a finished request, else (None, None).
        The state is copied into `out` (a BF16 tensor on the host or the
        device) or a new host tensor of `shape`; a result can be taken once."""
        st, done, _ = gattn_serve_poll(self.h, rid, None)
        check(st, "gattn_serve_poll")
        if not done:
            return None, None
        if out is None:
            out = torch.empty(shape, dtype=torch.bfloat16)
        if out.dtype != torch.bfloat16 or not out.is_contiguous() or out.numel() != self._numel.get(rid, out.numel()):
            raise ValueError("result: out must be a contiguous BF16 tensor of the request's size")
        st, done, lat = gattn_serve_poll(self.h, rid, out)
        check(st, "gattn_serve_poll")
        self._keep.pop(rid, None)
        return out, lat

    def release(self, rid):
        """Drops the final state of a finished request without copying it."""
        check(gattn_serve_release(self.h, rid), "gattn_serve_release")

    def take_async(self, rid, out):
        """Starts copying the final state of a finished request into `out` (a
        BF16 tensor, pinned host or device memory) and returns; `out` holds the
        result once copied(rid) is True."""
        if out.dtype != torch.bfloat16 or not out.is_contiguous() or out.numel() != self._numel.get(rid, -1):
            raise ValueError("take_async: out must be a contiguous BF16 tensor of the request's size")
        check(gattn_serve_take_async(self.h, rid, out), "gattn_serve_take_async")
        self._keep.pop(rid, None)

    def copied(self, rid) -> bool:
        st, c = gattn_serve_copied(self.h, rid)
        check(st, "gattn_serve_copied")
        return c

    def done(self, rid) -> bool:
        st, done, _ = gattn_serve_poll(self.h, rid, None)
        check(st, "gattn_serve_poll")
        if done:
            self._keep.pop(rid, None)
        return done

    def stats(self):
        return gattn_serve_stats(self.h)

    def close(self):
        if self.h:
            gattn_serve_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def check(status: int, what: str = "gattn") -> None:
    if status != 0:
        raise GattnError(status, what)


# ---------------------------------------------------------------- torch-level API
@dataclass(frozen=True)
class Tiling:
    """Token grid and tile spec of a GPA call (all along (t, y, x))."""

    grid: tuple
    core: tuple
    halo: tuple
    window: str = "hann"
    scale: float = 0.0

    @property
    def N(self) -> int:
        T, Y, X = self.grid
        return T * Y * X


def desc_for(q: torch.Tensor, tiling: Tiling, out_dtype=None, flags: int = 0):
    if q.dim() != 4:
        raise ValueError("expected [B, heads, N, d]")
    B, nh, N, d = q.shape
    if N != tiling.N:
        raise ValueError(f"N={N} does not match grid {tiling.grid}")
    return make_desc(
        B, nh, d, tiling.grid, tiling.core, tiling.halo, tiling.window, q.dtype,
        out_dtype if out_dtype is not None else q.dtype, tiling.scale, flags,
    )


def _require_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("gattn needs contiguous CUDA tensors")


def forward(q, k, v, tiling: Tiling, out_dtype=None, stream=None):
    """Out = GPA(q, k, v) and the saved state the backward needs."""
    _require_cuda(q, k, v)
    desc = desc_for(q, tiling, out_dtype)
    out = torch.empty(q.shape, dtype=_TORCH_DTYPE[desc.out_dtype], device=q.device)
    saved = torch.empty(gattn_saved_bytes(desc), dtype=torch.uint8, device=q.device)
    check(gattn_fwd(desc, q, k, v, out, saved, stream=stream), "gattn_fwd")
    return out, saved


def backward(q, k, v, out, dout, saved, tiling: Tiling, stream=None):
    """(dq, dk, dv) of sum(out * dout)."""
    _require_cuda(q, k, v, out, dout, saved)
    desc = desc_for(q, tiling, out.dtype)
    if dout.dtype != q.dtype:
        raise ValueError("dout must have the input dtype")
    dq = torch.empty_like(out)
    dk = torch.empty_like(out)
    dv = torch.empty_like(out)
    ws = torch.empty(gattn_bwd_workspace_bytes(desc), dtype=torch.uint8, device=q.device)
    check(gattn_bwd(desc, q, k, v, out, dout, saved, dq, dk, dv, ws, stream=stream), "gattn_bwd")
    return dq, dk, dv


class GlobalAttention(torch.autograd.Function):
    """STORM-GPA as an autograd op: forward and hand-written backward in CUDA."""

    @staticmethod
    def forward(ctx, q, k, v, tiling: Tiling):
        out, saved = forward(q, k, v, tiling)
        ctx.tiling = tiling
        ctx.save_for_backward(q, k, v, out, saved)
        return out

    @staticmethod
    def backward(ctx, dout):
        q, k, v, out, saved = ctx.saved_tensors
        dout = dout.contiguous()
        if dout.dtype != q.dtype:
            raise ValueError("upstream gradient must have the input dtype")
        dq, dk, dv = backward(q, k, v, out, dout, saved, ctx.tiling)
        return dq, dk, dv, None


def global_attention(q, k, v, tiling: Tiling):
    return GlobalAttention.apply(q, k, v, tiling)


def gated_forward(q, k, v, kc, vc, gate, tiling: Tiling, out_dtype=None, stream=None):
    """Noise-gated blend gate[h] * GPA(q, k, v) + (1 - gate[h]) * GPA(q, kc, vc);
    gate: FP32 CUDA tensor [nh]."""
    _require_cuda(q, k, v, kc, vc, gate)
    if gate.dtype != torch.float32 or gate.shape != (q.shape[1],):
        raise ValueError("gate must be FP32 [heads]")
    desc = desc_for(q, tiling, out_dtype)
    out = torch.empty(q.shape, dtype=_TORCH_DTYPE[desc.out_dtype], device=q.device)
    ws = torch.empty(gattn_gated_workspace_bytes(desc), dtype=torch.uint8, device=q.device)
    check(gattn_gated_fwd(desc, q, k, v, kc, vc, gate, out, ws, stream=stream), "gattn_gated_fwd")
    return out


# ---------------------------------------------------------------- temporal compression
def compress_desc(k: torch.Tensor, out_dtype=None, scale: float = 0.0):
    """gattn_compress_desc for history keys/values k of shape [B, nh, S, M, d]."""
    if k.dim() != 5:
        raise ValueError("expected [B, heads, S, M, d]")
    B, nh, S, M, d = k.shape
    desc = gattn_compress_desc()
    desc.B, desc.nh, desc.d, desc.S, desc.M = int(B), int(nh), int(d), int(S), int(M)
    desc.in_dtype = _DTYPES[k.dtype]
    desc.out_dtype = _DTYPES[out_dtype if out_dtype is not None else k.dtype]
    desc.scale = float(scale or 0.0)
    return desc


def compress_forward(q, k, v, scale: float = 0.0, out_dtype=None, with_lse: bool = True, stream=None):
    """Temporal compression: (out [B, nh, M, d], lse [B, nh, M] or None).

    q [nh, d] FP32 learned queries; k, v [B, nh, S, M, d] (BF16 or FP32)."""
    _require_cuda(q, k, v)
    if q.dtype != torch.float32 or k.dtype != v.dtype or k.shape != v.shape:
        raise ValueError("q must be FP32 [nh, d]; k and v the same dtype and shape")
    desc = compress_desc(k, out_dtype, scale)
    if tuple(q.shape) != (desc.nh, desc.d):
        raise ValueError("q must be [nh, d]")
    B, nh, S, M, d = k.shape
    out = torch.empty((B, nh, M, d), dtype=_TORCH_DTYPE[desc.out_dtype], device=k.device)
    lse = torch.empty((B, nh, M), dtype=torch.float32, device=k.device) if with_lse else None
    nws = gattn_compress_workspace_bytes(desc)
    ws = torch.empty(nws, dtype=torch.uint8, device=k.device) if nws else None
    check(gattn_compress_fwd(desc, q, k, v, out, lse, ws, stream=stream), "gattn_compress_fwd")
    return out, lse


# ---------------------------------------------------------------- posterior sampling
def sigma_schedule(n: int, sigma_max: float = 2.0, sigma_min: float = 0.02, rho: float = 7.0):
    """n + 1 decreasing noise levels, sigma_max ... sigma_min, then 0 (the
    rho-spaced schedule of Karras et al. 2022, whose diffusion model the paper
    uses)."""
    out = []
    for i in range(n):
        f = i / max(n - 1, 1)
        out.append((sigma_max ** (1 / rho) + f * (sigma_min ** (1 / rho) - sigma_max ** (1 / rho))) ** rho)
    return out + [0.0]


class PosteriorSampler:
    """Diffusion posterior sampling with the GPA denoiser (one gattn_dps_step
    per noise level).  z: FP32 CUDA state [B, nh, N, d]; attention in
    ``attn_dtype`` ("bf16": tensor-core form on a BF16 copy of z, "fp32")."""

    def __init__(self, z, tiling: Tiling, attn_dtype="bf16"):
        _require_cuda(z)
        if z.dtype != torch.float32:
            raise ValueError("the state is FP32")
        self.z = z
        self.zb = z.to(torch.bfloat16) if attn_dtype == "bf16" else None
        self.desc = desc_for(self.zb if self.zb is not None else z, tiling, torch.float32)
        self.ws = torch.empty(gattn_dps_workspace_bytes(self.desc), dtype=torch.uint8, device=z.device)

    def step(self, y, mask, eps, sigma, sigma_next, lam, stream=None):
        p = gattn_dps_params()
        p.sigma, p.sigma_next, p.lam = float(sigma), float(sigma_next), float(lam)
        check(gattn_dps_step(self.desc, p, self.z, self.zb, y, mask, eps, self.ws, stream=stream), "gattn_dps_step")
        return self.z
