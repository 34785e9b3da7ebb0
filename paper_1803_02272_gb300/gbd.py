"""Thin Python binding of the gbd C ABI (include/gbd.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no compute:
all of the path (packing, scheduling, DP, conversion, stores) runs in libgbd.so's CUDA
kernels.  PyTorch is used for device memory and streams: output buffers are torch
tensors and `stream` defaults to torch's current CUDA stream.

Importing this module loads libgbd.so and raises if it has not been built -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgbd.so")

GBD_OK, GBD_EINVAL, GBD_ENOMEM, GBD_EBUDGET, GBD_ETIMEDOUT, GBD_ECUDA, GBD_ENOTFOUND = range(7)
GBD_CONV_MAX, GBD_CONV_MIN, GBD_CONV_SCORE, GBD_CONV_NORM = 0, 1, 2, 3
GBD_KERNEL_AUTO, GBD_KERNEL_GENERAL, GBD_KERNEL_SYSTOLIC = 0, 1, 2
PROBE_OPS = ["VIMAX3_S16X2_RELU", "VIADDMAX_S16X2", "VIADDMAX_S16X2_RELU", "VIMAX_S16X2_RELU",
             "VMAXS2", "PRMT", "IADD3", "LOP3", "IMAX", "HMAX2", "HADD2", "CELL_MIX",
             "VIMAX3_S16X2", "FMAX", "FMAX3", "FADD", "MIX_DPX_HMAX2", "MIX_DPX_FMAX3",
             "MIX_DPX_IADD3", "VIMAX3_U16X2", "VMINU2", "VSETLEU2", "VIBMIN_U16X2"]

# every symbol include/gbd.h declares (checked by the tests)
EXPORTS = [
    "gbd_default_params", "gbd_params_size", "gbd_create", "gbd_destroy", "gbd_trim", "gbd_load_reads", "gbd_free_set",
    "gbd_set_size", "gbd_set_max_len", "gbd_set_pair_cells", "gbd_all_pairs", "gbd_tile",
    "gbd_batch", "gbd_server_create", "gbd_server_submit", "gbd_server_poll",
    "gbd_server_wait", "gbd_server_destroy", "gbd_last_error", "gbd_probe_op_rate",
    "gbd_kernel_launches", "gbd_tile_noalloc", "gbd_sqdist_square", "gbd_gram_apply", "gbd_mds",
    "gbd_tile_hits", "gbd_threshold_components", "gbd_tri_components", "gbd_batch_tuning",
    "gbd_rect_hits", "gbd_bounds_check", "gbd_debug_output_limit", "gbd_all_pairs_to_host",
]


class GbdParams(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int16), ("mismatch", ctypes.c_int16),
                ("gap", ctypes.c_int16), ("conversion", ctypes.c_int16),
                ("kernel", ctypes.c_int32), ("hbm_budget", ctypes.c_uint64),
                ("timeout_us", ctypes.c_uint32), ("gap_open", ctypes.c_int16),
                ("band_entries", ctypes.c_uint64)]


class GbdThreshold(ctypes.Structure):
    """Hit rule d <= abs_max and d * den <= num * max(la, lb) (97 % homology: 3/100)."""
    _fields_ = [("num", ctypes.c_uint32), ("den", ctypes.c_uint32), ("abs_max", ctypes.c_uint32)]


class GbdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gbd error {code}: {msg}")
        self.code = code


def _declare(lib):
    vp, u64, u32, ci = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "gbd_default_params": ([ctypes.POINTER(GbdParams)], None),
        "gbd_params_size": ([], u64),
        "gbd_create": ([pp, ci, ctypes.POINTER(GbdParams)], ci),
        "gbd_destroy": ([vp], None),
        "gbd_trim": ([vp], ci),
        "gbd_load_reads": ([vp, vp, vp, u64, pp, vp], ci),
        "gbd_free_set": ([vp], None),
        "gbd_set_size": ([vp], u64),
        "gbd_set_max_len": ([vp], u32),
        "gbd_set_pair_cells": ([vp], ctypes.c_double),
        "gbd_all_pairs": ([vp, vp, vp, u64, vp], ci),
        "gbd_all_pairs_to_host": ([vp, vp, vp, u64, u64, vp], ci),
        "gbd_tile": ([vp, vp, u64, u64, vp, u64, u64, vp, u64, vp], ci),
        "gbd_batch": ([vp, vp, u64, vp, vp], ci),
        "gbd_server_create": ([vp, vp, pp], ci),
        "gbd_server_submit": ([vp, vp, vp, u64, vp, ctypes.POINTER(u64)], ci),
        "gbd_server_poll": ([vp, u64, ctypes.POINTER(ci)], ci),
        "gbd_server_wait": ([vp, u64], ci),
        "gbd_server_destroy": ([vp], None),
        "gbd_last_error": ([], ctypes.c_char_p),
        "gbd_probe_op_rate": ([ci, u32, ctypes.POINTER(ctypes.c_double), vp], ci),
        "gbd_kernel_launches": ([], u64),
        "gbd_tile_noalloc": ([vp, vp, vp, u64, vp, vp, u64, u32, vp, u64, vp], ci),
        "gbd_sqdist_square": ([vp, vp, u64, vp, u64, ctypes.POINTER(ctypes.c_int32), vp], ci),
        "gbd_gram_apply": ([vp, vp, u64, u64, ctypes.c_int32, vp, u32, vp, vp], ci),
        "gbd_mds": ([vp, vp, u64, vp, u32, u32, u32, vp, vp, vp], ci),
        "gbd_tile_hits": ([vp, vp, u64, u64, vp, u64, u64, ctypes.POINTER(GbdThreshold), vp, u64, vp, u64,
                           vp, vp, vp, vp], ci),
        "gbd_threshold_components": ([vp, vp, ctypes.POINTER(GbdThreshold), vp, vp, vp, vp], ci),
        "gbd_rect_hits": ([vp, vp, u64, u64, vp, u64, u64, vp, u64, ctypes.POINTER(GbdThreshold), vp, u64,
                           vp, vp, vp, vp], ci),
        "gbd_tri_components": ([vp, vp, vp, ctypes.POINTER(GbdThreshold), vp, vp, vp], ci),
        "gbd_bounds_check": ([ctypes.POINTER(u64)], ci),
        "gbd_debug_output_limit": ([vp, u64], ci),
        "gbd_batch_tuning": ([vp, u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ci)], ci),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1803_02272_gb300.build.build() "
                           "(there is no CPU fallback)")
    return _declare(ctypes.CDLL(path))


_lib = load_library()


def _check(rc: int):
    if rc != GBD_OK:
        raise GbdError(rc, (_lib.gbd_last_error() or b"").decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ C names

def gbd_params_size() -> int:
    return _lib.gbd_params_size()


def gbd_default_params() -> GbdParams:
    p = GbdParams()
    _lib.gbd_default_params(ctypes.byref(p))
    return p


def gbd_create(device: int = 0, params: GbdParams | None = None) -> int:
    h = ctypes.c_void_p()
    _check(_lib.gbd_create(ctypes.byref(h), device, ctypes.byref(params) if params else None))
    return h.value


def gbd_destroy(ctx: int) -> None:
    _lib.gbd_destroy(ctx)


def gbd_trim(ctx: int) -> None:
    """Free the context's kept workspaces (MDS square, captured batch graph)."""
    _check(_lib.gbd_trim(ctx))


def gbd_load_reads(ctx: int, seq, offsets, n: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_lib.gbd_load_reads(ctx, _ptr(seq), _ptr(offsets), n, ctypes.byref(h), _stream(stream)))
    return h.value


def gbd_free_set(s: int) -> None:
    _lib.gbd_free_set(s)


def gbd_set_size(s: int) -> int:
    return _lib.gbd_set_size(s)


def gbd_set_max_len(s: int) -> int:
    return _lib.gbd_set_max_len(s)


def gbd_set_pair_cells(s: int) -> float:
    return _lib.gbd_set_pair_cells(s)


def gbd_all_pairs(ctx: int, s: int, d_tri, tri_len: int, stream=None) -> None:
    _check(_lib.gbd_all_pairs(ctx, s, _ptr(d_tri), tri_len, _stream(stream)))


def gbd_all_pairs_to_host(ctx: int, s: int, h_tri, tri_len: int, band_entries: int = 0, stream=None) -> None:
    """The triangle into host memory (a numpy array or a pinned torch tensor), band by band."""
    _check(_lib.gbd_all_pairs_to_host(ctx, s, _ptr(h_tri), tri_len, band_entries, _stream(stream)))


def gbd_tile(ctx: int, A: int, a0: int, a1: int, B: int, b0: int, b1: int, d_out, ld: int,
             stream=None) -> None:
    _check(_lib.gbd_tile(ctx, A, a0, a1, B, b0, b1, _ptr(d_out), ld, _stream(stream)))


def gbd_batch(ctx: int, samples, d_tris, stream=None) -> None:
    ns = len(samples)
    arr_s = (ctypes.c_void_p * max(ns, 1))(*samples)
    arr_o = (ctypes.c_void_p * max(ns, 1))(*[_ptr(t) for t in d_tris])
    _check(_lib.gbd_batch(ctx, ctypes.cast(arr_s, ctypes.c_void_p), ns,
                          ctypes.cast(arr_o, ctypes.c_void_p), _stream(stream)))


def gbd_batch_tuning(ctx: int) -> dict:
    """Autotuner state of the context's batched launch: per candidate its time (ms), work-unit
    scale and stream count, the chosen candidate (-1 while tuning) and whether tuning is done."""
    cap = 16
    ms = (ctypes.c_double * cap)()
    sc = (ctypes.c_double * cap)()
    streams = (ctypes.c_int32 * cap)()
    nt = ctypes.c_uint32()
    chosen = ctypes.c_int32()
    done = ctypes.c_int()
    _check(_lib.gbd_batch_tuning(ctx, cap, ms, sc, streams, ctypes.byref(nt), ctypes.byref(chosen),
                                 ctypes.byref(done)))
    k = nt.value
    return {"trial_ms": list(ms)[:k], "piece_scale": list(sc)[:k], "streams": list(streams)[:k],
            "chosen": chosen.value, "done": bool(done.value)}


def gbd_server_create(ctx: int, ref: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.gbd_server_create(ctx, ref, ctypes.byref(h)))
    return h.value


def gbd_server_submit(srv: int, seq, offsets, nq: int, d_rows) -> int:
    t = ctypes.c_uint64()
    _check(_lib.gbd_server_submit(srv, _ptr(seq), _ptr(offsets), nq, _ptr(d_rows), ctypes.byref(t)))
    return t.value


def gbd_server_poll(srv: int, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(_lib.gbd_server_poll(srv, ticket, ctypes.byref(d)))
    return bool(d.value)


def gbd_server_wait(srv: int, ticket: int) -> None:
    _check(_lib.gbd_server_wait(srv, ticket))


def gbd_server_destroy(srv: int) -> None:
    _lib.gbd_server_destroy(srv)


def gbd_last_error() -> str:
    return (_lib.gbd_last_error() or b"").decode()


def gbd_probe_op_rate(op: int, iters: int, stream=None) -> float:
    r = ctypes.c_double()
    _check(_lib.gbd_probe_op_rate(op, iters, ctypes.byref(r), _stream(stream)))
    return r.value


def gbd_tile_noalloc(ctx: int, seqA, offA, nA: int, seqB, offB, nB: int, max_len: int, d_out,
                     ld: int, stream=None) -> None:
    """Allocation-free rectangle (device inputs and output; see include/gbd.h)."""
    _check(_lib.gbd_tile_noalloc(ctx, _ptr(seqA), _ptr(offA), nA, _ptr(seqB), _ptr(offB), nB,
                                 max_len, _ptr(d_out), ld, _stream(stream)))


def gbd_sqdist_square(ctx: int, d_tri, n: int, d_w, ld: int, stream=None) -> int:
    """fp16 square of scaled squared distances from a triangle; returns the shift s."""
    s = ctypes.c_int32()
    _check(_lib.gbd_sqdist_square(ctx, _ptr(d_tri), n, _ptr(d_w), ld, ctypes.byref(s), _stream(stream)))
    return s.value


def gbd_gram_apply(ctx: int, d_w, n: int, ld: int, shift: int, d_x, k: int, d_y, stream=None) -> None:
    """Y = G X with G = -1/2 J (D o D) J (device float32 n x k)."""
    _check(_lib.gbd_gram_apply(ctx, _ptr(d_w), n, ld, shift, _ptr(d_x), k, _ptr(d_y), _stream(stream)))


def gbd_mds(ctx: int, d_tri, n: int, d_omega, k: int, r: int, q: int, d_lambda, d_coords,
            stream=None) -> None:
    """Classical MDS by randomized SVD: r eigenvalues and n x r coordinates (device)."""
    _check(_lib.gbd_mds(ctx, _ptr(d_tri), n, _ptr(d_omega), k, r, q, _ptr(d_lambda), _ptr(d_coords),
                        _stream(stream)))


def threshold(num: int = 3, den: int = 100, abs_max: int = 65535) -> GbdThreshold:
    return GbdThreshold(num, den, abs_max)


def gbd_tile_hits(ctx: int, A: int, a0: int, a1: int, B: int, b0: int, b1: int, th: GbdThreshold,
                  d_out=None, ld: int = 0, d_hits=None, hit_capacity: int = 0, d_hit_count=None,
                  d_ref_labels=None, d_row_labels=None, stream=None) -> None:
    """Rectangle with the threshold epilogue (hit list and/or row annotation)."""
    _check(_lib.gbd_tile_hits(ctx, A, a0, a1, B, b0, b1, ctypes.byref(th), _ptr(d_out), ld, _ptr(d_hits),
                              hit_capacity, _ptr(d_hit_count), _ptr(d_ref_labels), _ptr(d_row_labels),
                              _stream(stream)))


def gbd_rect_hits(ctx: int, A: int, a0: int, a1: int, B: int, b0: int, b1: int, d_rect, ld: int,
                  th: GbdThreshold, d_hits=None, hit_capacity: int = 0, d_hit_count=None, d_ref_labels=None,
                  d_row_labels=None, stream=None) -> None:
    """Threshold epilogue over an already computed rectangle."""
    _check(_lib.gbd_rect_hits(ctx, A, a0, a1, B, b0, b1, _ptr(d_rect), ld, ctypes.byref(th), _ptr(d_hits),
                              hit_capacity, _ptr(d_hit_count), _ptr(d_ref_labels), _ptr(d_row_labels),
                              _stream(stream)))


def gbd_threshold_components(ctx: int, s: int, th: GbdThreshold, d_labels, d_edges=None, d_tri=None,
                             stream=None) -> None:
    """Connected components of the threshold graph (labels = smallest read of each component)."""
    _check(_lib.gbd_threshold_components(ctx, s, ctypes.byref(th), _ptr(d_labels), _ptr(d_edges), _ptr(d_tri),
                                         _stream(stream)))


def gbd_tri_components(ctx: int, s: int, d_tri, th: GbdThreshold, d_labels, d_edges=None, stream=None) -> None:
    """Threshold-graph components from an already computed triangle of the set."""
    _check(_lib.gbd_tri_components(ctx, s, _ptr(d_tri), ctypes.byref(th), _ptr(d_labels), _ptr(d_edges),
                                   _stream(stream)))


def gbd_kernel_launches() -> int:
    return _lib.gbd_kernel_launches()


# ------------------------------------------------------------------ convenience wrappers

class ReadSetHandle:
    """Owns a gbd_set; frees it when garbage collected."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx, self.handle = ctx, handle

    @property
    def n(self) -> int:
        return gbd_set_size(self.handle)

    @property
    def max_len(self) -> int:
        return gbd_set_max_len(self.handle)

    @property
    def pair_cells(self) -> float:
        return gbd_set_pair_cells(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                gbd_free_set(self.handle)
            except Exception:
                pass
            self.handle = None


class Context:
    """A gbd context with torch-allocated outputs."""

    def __init__(self, device: int = 0, **params):
        p = gbd_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        self.device = device
        self.handle = gbd_create(device, p)

    def load_reads(self, seq, offsets, stream=None) -> ReadSetHandle:
        n = len(offsets) - 1
        return ReadSetHandle(self, gbd_load_reads(self.handle, seq, offsets, n, stream))

    def load(self, readset, stream=None) -> ReadSetHandle:
        """Load a synth.ReadSet (host numpy arrays)."""
        seq = np.ascontiguousarray(readset.seq, dtype=np.uint8)
        off = np.ascontiguousarray(readset.offsets, dtype=np.uint64)
        if seq.size == 0:
            seq = np.zeros(1, np.uint8)
        return self.load_reads(seq, off, stream)

    def all_pairs(self, s: ReadSetHandle, out=None, stream=None):
        import torch
        n = s.n
        m = n * (n - 1) // 2
        if out is None:
            out = torch.empty(max(m, 1), dtype=torch.int16, device=f"cuda:{self.device}")
        gbd_all_pairs(self.handle, s.handle, out, m, stream)
        return out[:m]

    def tile(self, A: ReadSetHandle, a0, a1, B: ReadSetHandle, b0, b1, out=None, ld=None,
             stream=None):
        import torch
        ld = (b1 - b0) if ld is None else ld
        if out is None:
            out = torch.empty(max((a1 - a0) * ld, 1), dtype=torch.int16,
                              device=f"cuda:{self.device}")
        gbd_tile(self.handle, A.handle, a0, a1, B.handle, b0, b1, out, ld, stream)
        return out[: (a1 - a0) * ld].view(a1 - a0, ld)

    def batch(self, sets, outs=None, stream=None):
        import torch
        if outs is None:
            outs = [torch.empty(max(s.n * (s.n - 1) // 2, 1), dtype=torch.int16,
                                device=f"cuda:{self.device}") for s in sets]
        gbd_batch(self.handle, [s.handle for s in sets], outs, stream)
        return [o[: s.n * (s.n - 1) // 2] for o, s in zip(outs, sets)]

    def close(self):
        if self.handle:
            gbd_destroy(self.handle)
            self.handle = None


class Server:
    """A serving loop over a resident reference set (gbd_server_*)."""

    def __init__(self, ctx: Context, ref: ReadSetHandle):
        self.ctx, self.ref = ctx, ref
        self.handle = gbd_server_create(ctx.handle, ref.handle)

    def submit(self, readset, out=None):
        """Queue a synth.ReadSet of queries; returns (ticket, output tensor nq x n_ref)."""
        import torch
        seq = np.ascontiguousarray(readset.seq, dtype=np.uint8)
        if seq.size == 0:
            seq = np.zeros(1, np.uint8)
        off = np.ascontiguousarray(readset.offsets, dtype=np.uint64)
        nq = len(off) - 1
        if out is None:
            out = torch.empty((nq, self.ref.n), dtype=torch.int16, device=f"cuda:{self.ctx.device}")
        t = gbd_server_submit(self.handle, seq, off, nq, out)
        return t, out

    def poll(self, ticket: int) -> bool:
        return gbd_server_poll(self.handle, ticket)

    def wait(self, ticket: int) -> None:
        gbd_server_wait(self.handle, ticket)

    def close(self):
        if self.handle:
            gbd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def as_uint16(t) -> np.ndarray:
    """Host numpy uint16 view of an int16 torch tensor holding uint16 distances."""
    return t.cpu().numpy().view(np.uint16)
