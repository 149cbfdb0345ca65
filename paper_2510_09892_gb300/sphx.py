"""Python binding of libsphx.so (include/sphx.h): argument marshalling only.

Every function here forwards to the C ABI of the same name. Tensors are
passed as raw device pointers; PyTorch only provides device memory and
streams. There is no CPU path: if the CUDA library cannot be loaded, the
import of this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphx.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sphx.h")

# sphx_status
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NOMEM, ERR_UNSUPPORTED = range(7)
# sphx_mode
(MODE_DIRECT_FP64, MODE_EFT_FP64, MODE_EFT_FF32, MODE_EFT_FP64_PRINTED, MODE_WIDE_INT,
 MODE_ADAPTIVE) = range(6)
MODES = {"direct": MODE_DIRECT_FP64, "eft": MODE_EFT_FP64, "ff32": MODE_EFT_FF32,
         "eft_printed": MODE_EFT_FP64_PRINTED, "wide": MODE_WIDE_INT, "adaptive": MODE_ADAPTIVE}
# sphx_compaction
COMPACT_AUTO, COMPACT_ATOMIC, COMPACT_ORDERED, COMPACT_FUSED = range(4)

HIT_DTYPE = [("edge", "<i8"), ("lat", "<i4"), ("root", "<i4"), ("x", "<f8"), ("y", "<f8")]
HIT_BYTES = 32


class SphxError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {status_string(status)}"
        if status == ERR_CUDA:
            msg += f" ({last_cuda_error()})"
        super().__init__(msg)


class Tuning(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("pairs_per_lane", ctypes.c_int32), ("compaction", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32

_SIGS = {
    "sphx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    "sphx_destroy": (None, [_vp]),
    "sphx_intersect_gca_constlat": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, ctypes.c_int, _vp]),
    "sphx_intersect_gca_constlat_adaptive": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp,
                                                            ctypes.c_double, _vp, _vp]),
    "sphx_intersect_gca_constlat_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp,
                                                        ctypes.c_int, _vp]),
    "sphx_host_join": (ctypes.c_int, [_vp, _vp]),
    "sphx_accux_intermediates": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "sphx_intersect_gca_gca": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp, ctypes.c_int,
                                              _vp]),
    "sphx_candidate_ranges": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp]),
    "sphx_intersect_ragged": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _i64, _vp, _vp, _i64, _vp, _vp,
                                             ctypes.c_int, _vp, _i64, _vp, _vp]),
    "sphx_intersect_ragged_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i64, _vp, _vp, _i64,
                                                     ctypes.c_int, _vp, _i64, _vp, _vp]),
    "sphx_noalloc_sync_status": (ctypes.c_int, [_vp]),
    "sphx_band_ranges": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp,
                                        _vp, _vp]),
    "sphx_band_areas": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp,
                                       _vp, ctypes.c_int, _vp, _i64, _vp]),
    "sphx_zonal_sums": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _vp]),
    "sphx_autotune_dense": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, ctypes.c_int, _vp,
                                           ctypes.POINTER(ctypes.c_double)]),
    "sphx_tuning_cache_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int64)]),
    "sphx_tuning_cache_clear": (ctypes.c_int, []),
    "sphx_sync_status": (ctypes.c_int, [_vp, _vp]),
    "sphx_set_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(Tuning)]),
    "sphx_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(Tuning)]),
    "sphx_autotune_ragged": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _i64, _vp, _vp, _i64,
                                            ctypes.c_int, _vp, _i64, _vp, _vp,
                                            ctypes.POINTER(ctypes.c_double)]),
    "sphx_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sphx_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sphx_last_cuda_error": (ctypes.c_char_p, []),
}


def header_symbols() -> list[str]:
    """Names of the functions include/sphx.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sphx_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded libsphx.so, built in-tree first if needed (never a fallback)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if not os.path.exists(LIB_PATH) or not _build.up_to_date():
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().sphx_status_string(status).decode()


def last_cuda_error() -> str:
    return lib().sphx_last_cuda_error().decode()


def _check(status: int, what: str):
    if status != OK:
        raise SphxError(status, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"expected a torch.Tensor or a device pointer, got {type(t)}")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _mode(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


def _dev_tensor(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# ------------------------------------------------------------------ dense --
def sphx_intersect_gca_constlat(A, B, z0, out_pts, out_count, mode="eft", stream=None):
    """Dense call: arc (A[i], B[i]) against latitude z0[i] (see include/sphx.h).

    A, B: (n, 3) float64 CUDA tensors; z0: (n,) float64; out_pts: (n, 2, 3)
    float64; out_count: (n,) int32. Stream-ordered, returns after enqueue.
    """
    n = int(z0.shape[0])
    _dev_tensor(A, torch.float64, "A", (n, 3))
    _dev_tensor(B, torch.float64, "B", (n, 3))
    _dev_tensor(z0, torch.float64, "z0", (n,))
    _dev_tensor(out_pts, torch.float64, "out_pts", (n, 2, 3))
    _dev_tensor(out_count, torch.int32, "out_count", (n,))
    st = lib().sphx_intersect_gca_constlat(_ptr(A), _ptr(B), _ptr(z0), n, _ptr(out_pts),
                                           _ptr(out_count), _mode(mode), _stream(stream))
    _check(st, "sphx_intersect_gca_constlat")


def sphx_intersect_gca_constlat_adaptive(A, B, z0, out_pts, out_count, gate_ulps=4.0,
                                         fallback_count=None, stream=None):
    """The dense call in the adaptive mode with a gate of gate_ulps ulp per
    component; fallback_count: optional (1,) int64 CUDA tensor to which the
    number of arcs re-evaluated by the accurate form is added."""
    n = int(z0.shape[0])
    _dev_tensor(A, torch.float64, "A", (n, 3))
    _dev_tensor(B, torch.float64, "B", (n, 3))
    _dev_tensor(z0, torch.float64, "z0", (n,))
    _dev_tensor(out_pts, torch.float64, "out_pts", (n, 2, 3))
    _dev_tensor(out_count, torch.int32, "out_count", (n,))
    if fallback_count is not None:
        _dev_tensor(fallback_count, torch.int64, "fallback_count", (1,))
    st = lib().sphx_intersect_gca_constlat_adaptive(_ptr(A), _ptr(B), _ptr(z0), n, _ptr(out_pts),
                                                    _ptr(out_count), float(gate_ulps),
                                                    _ptr(fallback_count), _stream(stream))
    _check(st, "sphx_intersect_gca_constlat_adaptive")


def sphx_intersect_gca_gca(A1, A2, B1, B2, out_pts, out_count, mode="wide", stream=None):
    """Intersection of arc (A1[i], A2[i]) with arc (B1[i], B2[i]) (see include/sphx.h):
    (n, 3) float64 CUDA tensors in, out_pts (n, 2, 3) float64 and out_count (n,) int32."""
    n = int(A1.shape[0])
    for t, name in ((A1, "A1"), (A2, "A2"), (B1, "B1"), (B2, "B2")):
        _dev_tensor(t, torch.float64, name, (n, 3))
    _dev_tensor(out_pts, torch.float64, "out_pts", (n, 2, 3))
    _dev_tensor(out_count, torch.int32, "out_count", (n,))
    st = lib().sphx_intersect_gca_gca(_ptr(A1), _ptr(A2), _ptr(B1), _ptr(B2), n, _ptr(out_pts),
                                      _ptr(out_count), _mode(mode), _stream(stream))
    _check(st, "sphx_intersect_gca_gca")


def sphx_accux_intermediates(A, B, z0, out_mid, stream=None):
    """Algorithm 8's intermediate pairs per arc (App. A): out_mid (n, 16) float64."""
    n = int(z0.shape[0])
    _dev_tensor(out_mid, torch.float64, "out_mid", (n, 16))
    st = lib().sphx_accux_intermediates(_ptr(A), _ptr(B), _ptr(z0), n, _ptr(out_mid),
                                        _stream(stream))
    _check(st, "sphx_accux_intermediates")


def intersect(A, B, z0, mode="eft", stream=None):
    """Allocate outputs and run the dense call; returns (out_pts, out_count)."""
    n = int(z0.shape[0])
    pts = torch.empty((n, 2, 3), dtype=torch.float64, device=z0.device)
    cnt = torch.empty((n,), dtype=torch.int32, device=z0.device)
    sphx_intersect_gca_constlat(A, B, z0, pts, cnt, mode, stream)
    return pts, cnt


# ----------------------------------------------------------------- ragged --
class Context:
    """Owns an sphx_context (scratch, status word, tuning, graphs) on one device."""

    def __init__(self, device: int = 0):
        h = _vp()
        _check(lib().sphx_create(ctypes.byref(h), int(device)), "sphx_create")
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            lib().sphx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tuning(self, threads_per_block=0, blocks_per_sm=0, pairs_per_lane=0,
                   compaction=COMPACT_AUTO, use_graph=1):
        t = Tuning(threads_per_block, blocks_per_sm, pairs_per_lane, compaction, use_graph)
        _check(lib().sphx_set_tuning(self.handle, ctypes.byref(t)), "sphx_set_tuning")

    def reset_tuning(self):
        _check(lib().sphx_set_tuning(self.handle, None), "sphx_set_tuning")

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(lib().sphx_get_tuning(self.handle, ctypes.byref(t)), "sphx_get_tuning")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def sync_status(self, stream=None) -> int:
        return lib().sphx_sync_status(self.handle, _stream(stream))


def _host_tensor(t, dtype, name, shape):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")


def sphx_intersect_gca_constlat_host(ctx: "Context", A, B, z0, out_pts, out_count, mode="wide",
                                     stream=None):
    """Dense call on host tensors (best pinned): copies in, kernels and copies
    out pipelined on the context's streams, ordered after the work already on
    `stream` (default: the current stream). The outputs are complete after
    sphx_host_join(ctx, stream) and a synchronisation of `stream`."""
    n = int(z0.shape[0])
    _host_tensor(A, torch.float64, "A", (n, 3))
    _host_tensor(B, torch.float64, "B", (n, 3))
    _host_tensor(z0, torch.float64, "z0", (n,))
    _host_tensor(out_pts, torch.float64, "out_pts", (n, 2, 3))
    _host_tensor(out_count, torch.int32, "out_count", (n,))
    st = lib().sphx_intersect_gca_constlat_host(ctx.handle, _ptr(A), _ptr(B), _ptr(z0), n,
                                                _ptr(out_pts), _ptr(out_count), _mode(mode),
                                                _stream(stream))
    _check(st, "sphx_intersect_gca_constlat_host")


def sphx_host_join(ctx: "Context", stream=None):
    """Make `stream` wait for every host-buffer call enqueued on ctx so far."""
    _check(lib().sphx_host_join(ctx.handle, _stream(stream)), "sphx_host_join")


def sphx_candidate_ranges(A, B, edge_offsets, lat_z, lat_offsets, lo, hi, stream=None):
    """Per-edge candidate latitude ranges [lo, hi) (global latitude indices)."""
    M = int(edge_offsets.shape[0]) - 1
    E = int(A.shape[0])
    L = int(lat_z.shape[0])
    _check(lib().sphx_candidate_ranges(_ptr(A), _ptr(B), _ptr(edge_offsets), M, E, _ptr(lat_z),
                                       _ptr(lat_offsets), L, _ptr(lo), _ptr(hi), _stream(stream)),
           "sphx_candidate_ranges")


def sphx_intersect_ragged(ctx: Context, A, B, edge_offsets, lat_z, lat_offsets, out, out_total,
                          mode="eft", edge_lat_lo=None, edge_lat_hi=None, stream=None):
    """Ragged call (see include/sphx.h). out: uint8/int8 CUDA tensor of cap*32 bytes
    (or any contiguous tensor whose byte size is a multiple of 32); out_total: (1,) int64."""
    M = int(edge_offsets.shape[0]) - 1
    E = int(A.shape[0])
    L = int(lat_z.shape[0])
    _dev_tensor(A, torch.float64, "A", (E, 3))
    _dev_tensor(B, torch.float64, "B", (E, 3))
    _dev_tensor(edge_offsets, torch.int64, "edge_offsets")
    _dev_tensor(lat_offsets, torch.int64, "lat_offsets", (M + 1,))
    _dev_tensor(out_total, torch.int64, "out_total", (1,))
    cap = out.numel() * out.element_size() // HIT_BYTES
    st = lib().sphx_intersect_ragged(ctx.handle, _ptr(A), _ptr(B), _ptr(edge_offsets), M, E,
                                     _ptr(lat_z), _ptr(lat_offsets), L, _ptr(edge_lat_lo),
                                     _ptr(edge_lat_hi), _mode(mode), _ptr(out), cap,
                                     _ptr(out_total), _stream(stream))
    _check(st, "sphx_intersect_ragged")


NOALLOC_MAX_EDGES = 262144


def sphx_intersect_ragged_noalloc(A, B, edge_offsets, lat_z, lat_offsets, out, out_total,
                                  mode="eft", stream=None):
    """The ragged call on the library's fixed scratch array (no allocation).

    Same arguments and results as sphx_intersect_ragged, without a context or
    caller-given ranges; E may not exceed NOALLOC_MAX_EDGES. A capacity
    overflow shows as out_total > capacity. Calls that overlap on the GPU race
    on the shared scratch and must be serialised by the caller.
    """
    M = int(edge_offsets.shape[0]) - 1
    E = int(A.shape[0])
    L = int(lat_z.shape[0])
    cap = out.numel() * out.element_size() // HIT_BYTES
    st = lib().sphx_intersect_ragged_noalloc(_ptr(A), _ptr(B), _ptr(edge_offsets), M, E,
                                             _ptr(lat_z), _ptr(lat_offsets), L, _mode(mode),
                                             _ptr(out), cap, _ptr(out_total), _stream(stream))
    _check(st, "sphx_intersect_ragged_noalloc")


def sphx_noalloc_sync_status(stream=None) -> int:
    """Status of the latest allocation-free ragged call on the current device
    (synchronises `stream`; clears the word): OK, ERR_CAPACITY or ERR_INVALID_ARG."""
    return lib().sphx_noalloc_sync_status(_stream(stream))


def sphx_autotune_ragged(ctx: Context, A, B, edge_offsets, lat_z, lat_offsets, out, out_total,
                         mode="eft", stream=None) -> float:
    M = int(edge_offsets.shape[0]) - 1
    E = int(A.shape[0])
    L = int(lat_z.shape[0])
    cap = out.numel() * out.element_size() // HIT_BYTES
    ms = ctypes.c_double(0.0)
    st = lib().sphx_autotune_ragged(ctx.handle, _ptr(A), _ptr(B), _ptr(edge_offsets), M, E,
                                    _ptr(lat_z), _ptr(lat_offsets), L, _mode(mode), _ptr(out), cap,
                                    _ptr(out_total), _stream(stream), ctypes.byref(ms))
    _check(st, "sphx_autotune_ragged")
    return ms.value


def sphx_autotune_dense(A, B, z0, out_pts, out_count, mode="wide", stream=None) -> float:
    """Pick the dense call's grid for `mode` on these arrays (or take it from
    the tuning cache); returns the best time in ms. Overwrites the outputs."""
    n = int(z0.shape[0])
    _dev_tensor(A, torch.float64, "A", (n, 3))
    _dev_tensor(B, torch.float64, "B", (n, 3))
    _dev_tensor(z0, torch.float64, "z0", (n,))
    _dev_tensor(out_pts, torch.float64, "out_pts", (n, 2, 3))
    _dev_tensor(out_count, torch.int32, "out_count", (n,))
    ms = ctypes.c_double(0.0)
    st = lib().sphx_autotune_dense(_ptr(A), _ptr(B), _ptr(z0), n, _ptr(out_pts), _ptr(out_count),
                                   _mode(mode), _stream(stream), ctypes.byref(ms))
    _check(st, "sphx_autotune_dense")
    return ms.value


def tuning_cache_stats() -> tuple[int, int]:
    """(hits, sweeps) of the process-wide tuning cache."""
    h, w = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().sphx_tuning_cache_stats(ctypes.byref(h), ctypes.byref(w)),
           "sphx_tuning_cache_stats")
    return h.value, w.value


def tuning_cache_clear():
    _check(lib().sphx_tuning_cache_clear(), "sphx_tuning_cache_clear")


# ------------------------------------------------------------- band areas --
def _mesh_args(nodes, face_offsets, face_nodes, lat_z):
    _dev_tensor(nodes, torch.float64, "nodes")
    if nodes.dim() != 2 or nodes.shape[1] != 3:
        raise ValueError("nodes must have shape (n_nodes, 3)")
    _dev_tensor(face_offsets, torch.int64, "face_offsets")
    _dev_tensor(face_nodes, torch.int32, "face_nodes")
    _dev_tensor(lat_z, torch.float64, "lat_z")
    return (_ptr(nodes), int(nodes.shape[0]), _ptr(face_offsets), _ptr(face_nodes),
            int(face_nodes.numel()), int(face_offsets.numel()) - 1, _ptr(lat_z), int(lat_z.numel()))


def sphx_band_ranges(ctx: Context, nodes, face_offsets, face_nodes, lat_z, band_lo, band_hi,
                     area_offsets, stream=None):
    """Bands [band_lo, band_hi) per cell and the output offsets (see include/sphx.h).

    nodes: (n_nodes, 3) float64; face_offsets: (n_faces + 1,) int64; face_nodes:
    int32; lat_z: ascending float64; band_lo, band_hi: (n_faces,) int32;
    area_offsets: (n_faces + 1,) int64 (all CUDA tensors).
    """
    args = _mesh_args(nodes, face_offsets, face_nodes, lat_z)
    F = args[5]
    _dev_tensor(band_lo, torch.int32, "band_lo", (F,))
    _dev_tensor(band_hi, torch.int32, "band_hi", (F,))
    _dev_tensor(area_offsets, torch.int64, "area_offsets", (F + 1,))
    _check(lib().sphx_band_ranges(ctx.handle, *args, _ptr(band_lo), _ptr(band_hi),
                                  _ptr(area_offsets), _stream(stream)), "sphx_band_ranges")


def sphx_band_areas(ctx: Context, nodes, face_offsets, face_nodes, lat_z, band_lo, band_hi,
                    area_offsets, areas, mode="wide", stream=None):
    """Area of each cell in each band of its range, into areas (float64 CUDA tensor)."""
    args = _mesh_args(nodes, face_offsets, face_nodes, lat_z)
    _dev_tensor(areas, torch.float64, "areas")
    _check(lib().sphx_band_areas(ctx.handle, *args, _ptr(band_lo), _ptr(band_hi),
                                 _ptr(area_offsets), _mode(mode), _ptr(areas), int(areas.numel()),
                                 _stream(stream)), "sphx_band_areas")


def sphx_zonal_sums(ctx: Context, band_lo, band_hi, area_offsets, areas, field, n_lat, out_fa,
                    out_a, stream=None):
    """Per band: sum of field * area (out_fa) and of area (out_a), order-independent."""
    F = int(band_lo.numel())
    _dev_tensor(field, torch.float64, "field", (F,))
    _dev_tensor(out_fa, torch.float64, "out_fa", (int(n_lat) - 1,))
    _dev_tensor(out_a, torch.float64, "out_a", (int(n_lat) - 1,))
    _check(lib().sphx_zonal_sums(ctx.handle, _ptr(band_lo), _ptr(band_hi), _ptr(area_offsets), F,
                                 _ptr(areas), _ptr(field), int(n_lat), _ptr(out_fa), _ptr(out_a),
                                 _stream(stream)), "sphx_zonal_sums")


def band_areas(ctx: Context, nodes, face_offsets, face_nodes, lat_z, mode="wide", stream=None):
    """Both band-area calls with freshly allocated outputs (reads the entry count
    back to the host once). Returns (band_lo, band_hi, area_offsets, areas)."""
    F = int(face_offsets.numel()) - 1
    dev = nodes.device
    band_lo = torch.empty(F, dtype=torch.int32, device=dev)
    band_hi = torch.empty(F, dtype=torch.int32, device=dev)
    off = torch.empty(F + 1, dtype=torch.int64, device=dev)
    sphx_band_ranges(ctx, nodes, face_offsets, face_nodes, lat_z, band_lo, band_hi, off, stream)
    total = int(off[-1].item())
    areas = torch.empty(max(total, 1), dtype=torch.float64, device=dev)
    sphx_band_areas(ctx, nodes, face_offsets, face_nodes, lat_z, band_lo, band_hi, off, areas,
                    mode, stream)
    return band_lo, band_hi, off, areas[:total]


def zonal_sums(ctx: Context, nodes, face_offsets, face_nodes, lat_z, field, mode="wide",
               stream=None):
    """The whole zonal-mean step in one call: band ranges, band areas and the
    per-band sums. Returns (sum of field * area, sum of area) per band as
    float64 CUDA tensors of n_lat - 1 entries; their ratio is the zonal mean."""
    lo, hi, off, areas = band_areas(ctx, nodes, face_offsets, face_nodes, lat_z, mode, stream)
    nb = int(lat_z.numel()) - 1
    fa = torch.empty(nb, dtype=torch.float64, device=nodes.device)
    aa = torch.empty(nb, dtype=torch.float64, device=nodes.device)
    if areas.numel() == 0:  # no cell meets any band
        areas = torch.zeros(1, dtype=torch.float64, device=nodes.device)
    sphx_zonal_sums(ctx, lo, hi, off, areas, field, int(lat_z.numel()), fa, aa, stream)
    return fa, aa


def hits_to_numpy(out, total: int):
    """View the first `total` records of a ragged output buffer as a numpy structured array."""
    import numpy as np
    raw = out.view(torch.uint8)[: int(total) * HIT_BYTES].cpu().numpy()
    return raw.view(np.dtype(HIT_DTYPE))


PIPE_FP32, PIPE_FP64, PIPE_INT32 = 0, 1, 2


def sphx_probe_fma_rate(pipe) -> float:
    """Measured throughput of a pipe: FP32 / FP64 FMA in flop/s (an FMA counts
    2), or 32-bit integer multiply-adds per second (pipe 2). A bool selects
    FP64 (True) or FP32 (False)."""
    v = ctypes.c_double(0.0)
    _check(lib().sphx_probe_fma_rate(int(pipe), ctypes.byref(v)), "sphx_probe_fma_rate")
    return v.value
