"""Python binding of librcfar, the GB300 radar-chain library.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels (see include/rcfar.h for the meaning of every argument). Tensors are
torch CUDA tensors; their device pointers and the current torch stream are
passed to the C ABI. If the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librcfar.so")

RCFAR_OK = 0
RCFAR_ERR_INVALID_ARG = 1
RCFAR_ERR_UNSUPPORTED = 2
RCFAR_ERR_OUT_OF_WORKSPACE = 3
RCFAR_ERR_CUDA = 4
RCFAR_ERR_TIMEOUT = 5
RCFAR_ERR_BAD_STATE = 6
RCFAR_ERR_RANGE = 7

RCFAR_MAP_F32 = 0
RCFAR_MAP_F16 = 1
RCFAR_SAT_TILE_F32 = 0
RCFAR_SAT_I64 = 1
RCFAR_SAT_NAIVE_F32 = 2
RCFAR_SAT_TILE_I64 = 3
RCFAR_SAT_FUSED = 4

RCFAR_DETECT_MAGNITUDE = 0
RCFAR_DETECT_SQUARE_LAW = 1
RCFAR_NORM_GLOBAL_MAX = 0
RCFAR_NORM_ROW_ZSCORE = 1
RCFAR_X_RANGE_MAJOR = 0
RCFAR_X_TRACE_MAJOR = 1
RCFAR_CFAR_CA = 0
RCFAR_CFAR_GO = 1
RCFAR_CFAR_SO = 2
RCFAR_CFAR_OS = 3
RCFAR_MEM_HOST = 0
RCFAR_MEM_DEVICE = 1

SAT_TILE_H = 32
SAT_TILE_W = 128

# Every symbol include/rcfar.h declares.
EXPORTS = (
    "rcfar_create", "rcfar_destroy", "rcfar_alpha", "rcfar_n_ref", "rcfar_band_plan", "rcfar_sat_scale",
    "rcfar_status_string", "rcfar_preprocess", "rcfar_sat", "rcfar_cfar", "rcfar_cfar_direct",
    "rcfar_sat_materialize", "rcfar_run_batch", "rcfar_batch_bytes", "rcfar_prepare", "rcfar_get_error",
    "rcfar_trace_enable", "rcfar_trace_read", "rcfar_sat_cfar_static",
    "rcfar_server_create", "rcfar_server_submit", "rcfar_server_prepare", "rcfar_server_poll", "rcfar_server_get_stats",
    "rcfar_server_now_ns", "rcfar_server_destroy", "rcfar_selftest_wait",
    "rcfar_tune_batch", "rcfar_set_batch_tuning", "rcfar_get_batch_tuning", "rcfar_sat_cfar",
    "rcfar_threshold_factor", "rcfar_server_submit_many",
)


class RcfarError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class rcfar_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_rows", ctypes.c_int32), ("max_cols", ctypes.c_int32),
                ("max_n", ctypes.c_int32), ("max_window", ctypes.c_int32), ("max_frames", ctypes.c_int32),
                ("batch_bytes", ctypes.c_int64), ("cfar_tile_rows", ctypes.c_int32),
                ("cfar_tile_cols", ctypes.c_int32)]


class rcfar_pre_params(ctypes.Structure):
    _fields_ = [("fs_hz", ctypes.c_double), ("f_lo_hz", ctypes.c_double), ("f_hi_hz", ctypes.c_double),
                ("mean_len", ctypes.c_int32), ("halo_c", ctypes.c_int32), ("detector", ctypes.c_int32),
                ("normalise", ctypes.c_int32), ("x_layout", ctypes.c_int32), ("pad", ctypes.c_int32)]


class rcfar_band(ctypes.Structure):
    _fields_ = [("k_lo", ctypes.c_int32), ("k_hi", ctypes.c_int32), ("c0", ctypes.c_int32), ("c1", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("value_bound", ctypes.c_float)]


class rcfar_window(ctypes.Structure):
    _fields_ = [("train_r", ctypes.c_int32), ("train_c", ctypes.c_int32), ("guard_r", ctypes.c_int32),
                ("guard_c", ctypes.c_int32), ("pfa", ctypes.c_double), ("kind", ctypes.c_int32),
                ("os_rank", ctypes.c_int32)]


class rcfar_sat_view(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("scale_log2", ctypes.c_int32),
                ("table", ctypes.c_void_p), ("ld", ctypes.c_int64), ("row_carry", ctypes.c_void_p),
                ("col_carry", ctypes.c_void_p), ("ld_carry", ctypes.c_int64), ("generation", ctypes.c_uint64)]


class rcfar_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class rcfar_frame_desc(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("M", ctypes.c_int32), ("N", ctypes.c_int32), ("ldx", ctypes.c_int64),
                ("window", rcfar_window), ("det", ctypes.c_void_p), ("ld_det", ctypes.c_int64),
                ("thr", ctypes.c_void_p), ("ld_thr", ctypes.c_int64), ("map", ctypes.c_void_p),
                ("ld_map", ctypes.c_int64)]


_lib = None


class rcfar_batch_tuning(ctypes.Structure):
    _fields_ = [("dft_kblocks_per_cta", ctypes.c_int32), ("sat_mode", ctypes.c_int32),
                ("cfar_tile_rows", ctypes.c_int32), ("cfar_tile_cols", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("candidates", ctypes.c_int32), ("dft_operands", ctypes.c_int32)]


class rcfar_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32),
                ("max_batch_frames", ctypes.c_int32), ("max_rows", ctypes.c_int32), ("max_n", ctypes.c_int32),
                ("max_window", ctypes.c_int32), ("params", rcfar_pre_params)]


class rcfar_request(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("M", ctypes.c_int32), ("N", ctypes.c_int32), ("ldx", ctypes.c_int64),
                ("window", rcfar_window), ("det", ctypes.c_void_p), ("ld_det", ctypes.c_int64),
                ("tag", ctypes.c_int64), ("arrival_ns", ctypes.c_int64), ("memory", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class rcfar_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int64), ("status", ctypes.c_int32), ("batch_frames", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("pad", ctypes.c_int32), ("arrival_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class rcfar_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("max_batch_frames_seen", ctypes.c_int64), ("max_inflight_frames", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


def lib() -> ctypes.CDLL:
    """The loaded librcfar.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librcfar.so is not built ({LIB_PATH}); run paper_2012_11077_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, F32, F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        sig = {
            "rcfar_create": [ctypes.POINTER(rcfar_config), ctypes.POINTER(P)],
            "rcfar_destroy": [P],
            "rcfar_alpha": [I32, F64, ctypes.POINTER(F64)],
            "rcfar_n_ref": [ctypes.POINTER(rcfar_window), ctypes.POINTER(I32)],
            "rcfar_threshold_factor": [ctypes.POINTER(rcfar_window), ctypes.POINTER(F64), ctypes.POINTER(I32)],
            "rcfar_band_plan": [I32, ctypes.POINTER(rcfar_pre_params), ctypes.POINTER(rcfar_band)],
            "rcfar_sat_scale": [F32, I64, ctypes.POINTER(I32)],
            "rcfar_status_string": [ctypes.c_int],
            "rcfar_preprocess": [P, P, I32, I32, I64, ctypes.POINTER(rcfar_pre_params), P, I64,
                                 ctypes.POINTER(rcfar_band), P],
            "rcfar_sat": [P, P, I32, I32, I32, I32, I64, F32, I32, ctypes.POINTER(rcfar_sat_view), P],
            "rcfar_cfar": [P, ctypes.POINTER(rcfar_sat_view), P, I32, I32, I64, ctypes.POINTER(rcfar_window), I32,
                           I32, P, I64, P, I64, P],
            "rcfar_cfar_direct": [P, P, I32, I32, I64, ctypes.POINTER(rcfar_window), I32, I32, P, I64, P, I64, P],
            "rcfar_sat_materialize": [P, ctypes.POINTER(rcfar_sat_view), P, I64, P],
            "rcfar_run_batch": [P, ctypes.POINTER(rcfar_frame_desc), I32, ctypes.POINTER(rcfar_pre_params), P],
            "rcfar_batch_bytes": [I32, I32, ctypes.POINTER(rcfar_pre_params), ctypes.POINTER(rcfar_window),
                                  ctypes.POINTER(I64)],
            "rcfar_prepare": [P, ctypes.POINTER(rcfar_frame_desc), I32, ctypes.POINTER(rcfar_pre_params)],
            "rcfar_get_error": [P, P],
            "rcfar_trace_enable": [P, I32],
            "rcfar_trace_read": [P, ctypes.POINTER(rcfar_trace_entry), I32, ctypes.POINTER(I32)],
            "rcfar_sat_cfar_static": [P, I32, I32, I64, F32, ctypes.POINTER(rcfar_window), I32, I32, P, I64, P,
                                      I64, P, P],
            "rcfar_server_create": [ctypes.POINTER(rcfar_server_config), ctypes.POINTER(P)],
            "rcfar_server_submit": [P, ctypes.POINTER(rcfar_request)],
            "rcfar_server_submit_many": [P, ctypes.POINTER(rcfar_request), I32, ctypes.POINTER(I32)],
            "rcfar_server_prepare": [P, ctypes.POINTER(I32), ctypes.POINTER(rcfar_window), I32],
            "rcfar_server_poll": [P, ctypes.POINTER(rcfar_completion), I32, ctypes.POINTER(I32), I32],
            "rcfar_server_get_stats": [P, ctypes.POINTER(rcfar_server_stats)],
            "rcfar_server_now_ns": [],
            "rcfar_server_destroy": [P],
            "rcfar_selftest_wait": [I32, I32],
            "rcfar_tune_batch": [P, ctypes.POINTER(rcfar_frame_desc), I32, ctypes.POINTER(rcfar_pre_params), I32,
                                 ctypes.POINTER(rcfar_batch_tuning), P],
            "rcfar_set_batch_tuning": [P, ctypes.POINTER(rcfar_batch_tuning)],
            "rcfar_get_batch_tuning": [P, ctypes.POINTER(rcfar_batch_tuning)],
            "rcfar_sat_cfar": [P, P, I32, I32, I32, I32, I64, F32, ctypes.POINTER(rcfar_window), I32, I32, I32, P, I64,
                               P, I64, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = {"rcfar_status_string": ctypes.c_char_p,
                          "rcfar_server_now_ns": ctypes.c_int64}.get(name, ctypes.c_int)
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().rcfar_status_string(int(status)).decode()


def _check(st: int, what: str):
    if st != RCFAR_OK:
        raise RcfarError(st, what)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream) or None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None


def _ld(t) -> int:
    """Leading dimension (elements) of a row-major 2D tensor."""
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a row-major 2D tensor")
    return int(t.stride(0))


def _torch():
    import torch
    return torch


def _require(t, name: str, dtypes, rows: int = 0, cols: int = 0, cuda: bool = True):
    """Raise ValueError unless t is a 2D row-major tensor of one of dtypes with at
    least rows x cols elements, on the current CUDA device (cuda=True) or in host
    memory (cuda=False). Runs before any call into the library."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype}, expected one of {tuple(str(d) for d in dtypes)}")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name}: expected a row-major 2D tensor")
    if t.shape[0] < rows or t.shape[1] < cols:
        raise ValueError(f"{name}: shape {tuple(t.shape)} is smaller than {rows} x {cols}")
    if cuda:
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name}: must be on the current CUDA device")
    elif t.device.type != "cpu":
        raise ValueError(f"{name}: must be in host memory")


def _f32():
    return (_torch().float32,)


def _f32_f16():
    return (_torch().float32, _torch().float16)


def _u8():
    return (_torch().uint8,)


def _require_status(t):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or t.numel() < 1 or not t.is_contiguous():
        raise ValueError("status: expected a contiguous int32 tensor with at least one element")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError("status: must be on the current CUDA device")


def make_window(train_r, train_c, guard_r, guard_c, pfa, kind=RCFAR_CFAR_CA, os_rank=0) -> rcfar_window:
    """kind: RCFAR_CFAR_CA (cell averaging), RCFAR_CFAR_GO, RCFAR_CFAR_SO or RCFAR_CFAR_OS;
    os_rank: the OS rank k (0: ceil(3 n_ref / 4))."""
    return rcfar_window(int(train_r), int(train_c), int(guard_r), int(guard_c), float(pfa), int(kind), int(os_rank))


def make_pre_params(fs_hz=20.0, f_lo_hz=0.3, f_hi_hz=0.8, mean_len=5, halo_c=0, detector=0,
                    normalise=0, x_layout=0) -> rcfar_pre_params:
    """detector: RCFAR_DETECT_MAGNITUDE (0) or RCFAR_DETECT_SQUARE_LAW (1);
    normalise: RCFAR_NORM_GLOBAL_MAX (0) or RCFAR_NORM_ROW_ZSCORE (1);
    x_layout: RCFAR_X_RANGE_MAJOR (0, frames [M][N]) or RCFAR_X_TRACE_MAJOR (1, frames [N][M])."""
    return rcfar_pre_params(float(fs_hz), float(f_lo_hz), float(f_hi_hz), int(mean_len), int(halo_c),
                            int(detector), int(normalise), int(x_layout), 0)


def rcfar_alpha(n_ref: int, pfa: float) -> float:
    out = ctypes.c_double()
    _check(lib().rcfar_alpha(int(n_ref), float(pfa), ctypes.byref(out)), "rcfar_alpha")
    return out.value


def rcfar_n_ref(window: rcfar_window) -> int:
    out = ctypes.c_int32()
    _check(lib().rcfar_n_ref(ctypes.byref(window), ctypes.byref(out)), "rcfar_n_ref")
    return out.value


def rcfar_threshold_factor(window: rcfar_window):
    """(factor, cells): alpha / n_ref and n_ref for cell averaging; the
    half-sum factor t and the cells of one half for greatest-of / smallest-of;
    alpha_os and n_ref for the ordered statistic."""
    f = ctypes.c_double()
    n = ctypes.c_int32()
    _check(lib().rcfar_threshold_factor(ctypes.byref(window), ctypes.byref(f), ctypes.byref(n)),
           "rcfar_threshold_factor")
    return f.value, n.value


def rcfar_band_plan(N: int, params: rcfar_pre_params) -> rcfar_band:
    out = rcfar_band()
    _check(lib().rcfar_band_plan(int(N), ctypes.byref(params), ctypes.byref(out)), "rcfar_band_plan")
    return out


def rcfar_sat_scale(bound: float, max_cells: int) -> int:
    out = ctypes.c_int32()
    _check(lib().rcfar_sat_scale(float(bound), int(max_cells), ctypes.byref(out)), "rcfar_sat_scale")
    return out.value


def rcfar_batch_bytes(M: int, N: int, params: rcfar_pre_params, window: Optional[rcfar_window] = None) -> int:
    out = ctypes.c_int64()
    _check(lib().rcfar_batch_bytes(int(M), int(N), ctypes.byref(params),
                                   ctypes.byref(window) if window is not None else None, ctypes.byref(out)),
           "rcfar_batch_bytes")
    return out.value


# ---------------------------------------------------------------- handle
def rcfar_create(device: int = 0, max_rows: int = 1024, max_cols: int = 1024, max_n: int = 4096,
                 max_window: int = 32, max_frames: int = 64, batch_bytes: int = 0, cfar_tile=(0, 0)) -> int:
    cfg = rcfar_config(int(device), int(max_rows), int(max_cols), int(max_n), int(max_window), int(max_frames),
                       int(batch_bytes), int(cfar_tile[0]), int(cfar_tile[1]))
    h = ctypes.c_void_p()
    _check(lib().rcfar_create(ctypes.byref(cfg), ctypes.byref(h)), "rcfar_create")
    return h.value


def rcfar_destroy(h: int):
    _check(lib().rcfar_destroy(h), "rcfar_destroy")


def rcfar_get_error(h: int, stream=None) -> int:
    """Waits for the stream; returns the asynchronous status (does not raise)."""
    return lib().rcfar_get_error(h, _stream(stream))


def rcfar_preprocess(h: int, x, params: rcfar_pre_params, map_out, stream=None) -> rcfar_band:
    """x: float32 CUDA tensor (row-major), [M][N] or, with params.x_layout = RCFAR_X_TRACE_MAJOR,
    [N][M]; map_out: float32 [M][>=cols]."""
    M, N = _frame_dims(x, params.x_layout == RCFAR_X_TRACE_MAJOR)
    _require(x, "x", _f32())
    _require(map_out, "map_out", _f32(), M, rcfar_band_plan(N, params).cols)
    band = rcfar_band()
    _check(lib().rcfar_preprocess(h, _ptr(x), M, N, _ld(x), ctypes.byref(params), _ptr(map_out), _ld(map_out),
                                  ctypes.byref(band), _stream(stream)), "rcfar_preprocess")
    return band


def rcfar_sat(h: int, map_t, value_bound: float = 0.0, mode: int = RCFAR_SAT_TILE_I64, map_exp2: int = 0,
              stream=None) -> rcfar_sat_view:
    import torch
    _require(map_t, "map", _f32_f16())
    dtype = RCFAR_MAP_F16 if map_t.dtype == torch.float16 else RCFAR_MAP_F32
    view = rcfar_sat_view()
    _check(lib().rcfar_sat(h, _ptr(map_t), dtype, int(map_exp2), int(map_t.shape[0]), int(map_t.shape[1]),
                           _ld(map_t), float(value_bound), int(mode), ctypes.byref(view), _stream(stream)),
           "rcfar_sat")
    return view


def rcfar_cfar(h: int, view: rcfar_sat_view, map_t, window: rcfar_window, cut_c_lo: int, cut_c_hi: int, det,
               thr=None, map_exp2: int = 0, stream=None):
    import torch
    if map_t is not None:
        _require(map_t, "map", _f32_f16(), view.rows, view.cols)
    _require(det, "det", _u8(), view.rows, view.cols)
    if thr is not None:
        _require(thr, "thr", _f32(), view.rows, view.cols)
    dtype = RCFAR_MAP_F16 if map_t is not None and map_t.dtype == torch.float16 else RCFAR_MAP_F32
    _check(lib().rcfar_cfar(h, ctypes.byref(view), _ptr(map_t), dtype, int(map_exp2),
                            _ld(map_t) if map_t is not None else 0,
                            ctypes.byref(window), int(cut_c_lo), int(cut_c_hi), _ptr(det), _ld(det), _ptr(thr),
                            _ld(thr) if thr is not None else 0, _stream(stream)), "rcfar_cfar")


def rcfar_cfar_direct(h: int, map_t, window: rcfar_window, cut_c_lo: int, cut_c_hi: int, det, thr=None,
                      stream=None):
    _require(map_t, "map", _f32())
    rows, cols = int(map_t.shape[0]), int(map_t.shape[1])
    _require(det, "det", _u8(), rows, cols)
    if thr is not None:
        _require(thr, "thr", _f32(), rows, cols)
    _check(lib().rcfar_cfar_direct(h, _ptr(map_t), int(map_t.shape[0]), int(map_t.shape[1]), _ld(map_t),
                                   ctypes.byref(window), int(cut_c_lo), int(cut_c_hi), _ptr(det), _ld(det),
                                   _ptr(thr), _ld(thr) if thr is not None else 0, _stream(stream)),
           "rcfar_cfar_direct")


def rcfar_sat_materialize(h: int, view: rcfar_sat_view, out, stream=None):
    _require(out, "out", (_torch().float64,), view.rows, view.cols)
    _check(lib().rcfar_sat_materialize(h, ctypes.byref(view), _ptr(out), _ld(out), _stream(stream)),
           "rcfar_sat_materialize")


def _frame_dims(x, trace_major: bool):
    """(M, N) of a raw frame tensor: [M][N], or [N][M] when trace-major."""
    return (int(x.shape[1]), int(x.shape[0])) if trace_major else (int(x.shape[0]), int(x.shape[1]))


def frame_desc(x, window: rcfar_window, det, thr=None, map_out=None, trace_major: bool = False) -> rcfar_frame_desc:
    M, N = _frame_dims(x, trace_major)
    _require(x, "x", _f32())
    _require(det, "det", _u8(), M)
    if thr is not None:
        _require(thr, "thr", _f32(), M)
    if map_out is not None:
        _require(map_out, "map_out", _f32(), M)
    d = rcfar_frame_desc(_ptr(x), M, N, _ld(x), window, _ptr(det), _ld(det),
                            _ptr(thr), _ld(thr) if thr is not None else 0, _ptr(map_out),
                            _ld(map_out) if map_out is not None else 0)
    d._outputs = (det, thr, map_out)  # checked against the band's columns by rcfar_run_batch
    return d


def _check_batch_outputs(frames, params: rcfar_pre_params):
    """Every frame's det / thr / map must hold the band's columns (known only with the params)."""
    for i, f in enumerate(frames):
        outs = getattr(f, "_outputs", None)
        if outs is None:
            continue
        pf = rcfar_pre_params(params.fs_hz, params.f_lo_hz, params.f_hi_hz, params.mean_len,
                              f.window.guard_c + f.window.train_c if params.halo_c < 0 else params.halo_c,
                              params.detector, params.normalise, params.x_layout, 0)
        cols = rcfar_band_plan(int(f.N), pf).cols
        for name, t in zip(("det", "thr", "map"), outs):
            if t is not None and t.shape[1] < cols:
                raise ValueError(f"frame {i}: {name} has {t.shape[1]} columns, the band needs {cols}")


def rcfar_run_batch(h: int, frames: Sequence[rcfar_frame_desc], params: rcfar_pre_params, stream=None):
    _check_batch_outputs(frames, params)
    arr = (rcfar_frame_desc * len(frames))(*frames)
    _check(lib().rcfar_run_batch(h, arr, len(frames), ctypes.byref(params), _stream(stream)), "rcfar_run_batch")


def rcfar_prepare(h: int, frames: Sequence[rcfar_frame_desc], params: rcfar_pre_params):
    arr = (rcfar_frame_desc * len(frames))(*frames)
    _check(lib().rcfar_prepare(h, arr, len(frames), ctypes.byref(params)), "rcfar_prepare")


def rcfar_trace_enable(h: int, on: bool = True):
    _check(lib().rcfar_trace_enable(h, 1 if on else 0), "rcfar_trace_enable")


def rcfar_trace_read(h: int) -> dict:
    """{kernel family: (launches, total_ms)} of the launches recorded since tracing started."""
    arr = (rcfar_trace_entry * 32)()
    n = ctypes.c_int32()
    _check(lib().rcfar_trace_read(h, arr, 32, ctypes.byref(n)), "rcfar_trace_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def rcfar_sat_cfar_static(map_t, value_bound: float, window: rcfar_window, cut_c_lo: int, cut_c_hi: int, det,
                          thr=None, status=None, stream=None):
    """SAT + CA-CFAR of a float32 map without any device allocation (see rcfar.h)."""
    _require(map_t, "map", _f32())
    rows, cols = int(map_t.shape[0]), int(map_t.shape[1])
    _require(det, "det", _u8(), rows, cols)
    if thr is not None:
        _require(thr, "thr", _f32(), rows, cols)
    if status is not None:
        _require_status(status)
    _check(lib().rcfar_sat_cfar_static(_ptr(map_t), int(map_t.shape[0]), int(map_t.shape[1]), _ld(map_t),
                                       float(value_bound), ctypes.byref(window), int(cut_c_lo), int(cut_c_hi),
                                       _ptr(det), _ld(det), _ptr(thr), _ld(thr) if thr is not None else 0,
                                       _ptr(status), _stream(stream)), "rcfar_sat_cfar_static")


# ---- serving ---------------------------------------------------------------

def rcfar_server_create(device: int = 0, budget_bytes: int = 8 << 30, slots: int = 3, max_batch_frames: int = 64,
                        max_rows: int = 1024, max_n: int = 4096, max_window: int = 32,
                        params: Optional[rcfar_pre_params] = None) -> int:
    cfg = rcfar_server_config(int(device), int(budget_bytes), int(slots), int(max_batch_frames), int(max_rows),
                              int(max_n), int(max_window), params if params is not None else make_pre_params(halo_c=-1))
    out = ctypes.c_void_p()
    _check(lib().rcfar_server_create(ctypes.byref(cfg), ctypes.byref(out)), "rcfar_server_create")
    return out.value


def rcfar_server_submit(srv: int, x, window: rcfar_window, det, tag: int, arrival_ns: int = 0,
                        trace_major: bool = False):
    """x, det: both host (CPU) tensors (pinned memory gives asynchronous copies) or both tensors on the
    current CUDA device (the server's device: read and written in place; the work that wrote x must be
    complete), row-major; they must stay alive until the frame's completion has been polled.
    trace_major: x is [N][M] (the server's params must say so too)."""
    req = server_request(x, window, det, tag, arrival_ns, trace_major)
    _check(lib().rcfar_server_submit(srv, ctypes.byref(req)), "rcfar_server_submit")


def server_request(x, window: rcfar_window, det, tag: int, arrival_ns: int = 0,
                   trace_major: bool = False) -> rcfar_request:
    """One request for rcfar_server_submit_many (same arguments and checks as rcfar_server_submit)."""
    M, N = _frame_dims(x, trace_major)
    device = bool(getattr(x, "is_cuda", False))
    _require(x, "x", _f32(), cuda=device)
    _require(det, "det", _u8(), M, cuda=device)
    return rcfar_request(_ptr(x), M, N, _ld(x), window, _ptr(det), _ld(det), int(tag), int(arrival_ns),
                         RCFAR_MEM_DEVICE if device else RCFAR_MEM_HOST, 0)


def rcfar_server_submit_many(srv: int, reqs: Sequence[rcfar_request]) -> int:
    """Queues the requests in order under one lock; returns how many were queued (raises on a refusal,
    after queueing the ones before it)."""
    n = len(reqs)
    arr = (rcfar_request * n)(*reqs)
    done = ctypes.c_int32()
    _check(lib().rcfar_server_submit_many(srv, arr, n, ctypes.byref(done)), "rcfar_server_submit_many")
    return done.value


def rcfar_server_prepare(srv: int, sizes: Sequence[int], windows: Sequence[rcfar_window]):
    n = len(sizes)
    Ns = (ctypes.c_int32 * n)(*[int(v) for v in sizes])
    ws = (rcfar_window * n)(*windows)
    _check(lib().rcfar_server_prepare(srv, Ns, ws, n), "rcfar_server_prepare")


def rcfar_server_poll(srv: int, max_n: int = 256, wait_ms: int = 0) -> list:
    buf = (rcfar_completion * max_n)()
    n = ctypes.c_int32()
    _check(lib().rcfar_server_poll(srv, buf, int(max_n), ctypes.byref(n), int(wait_ms)), "rcfar_server_poll")
    return [buf[i] for i in range(n.value)]


def rcfar_server_get_stats(srv: int) -> dict:
    st = rcfar_server_stats()
    _check(lib().rcfar_server_get_stats(srv, ctypes.byref(st)), "rcfar_server_get_stats")
    return {f: getattr(st, f) for f, _ in rcfar_server_stats._fields_}


def rcfar_server_now_ns() -> int:
    return int(lib().rcfar_server_now_ns())


def rcfar_server_destroy(srv: int):
    _check(lib().rcfar_server_destroy(srv), "rcfar_server_destroy")


def rcfar_selftest_wait(device: int = 0, polls: int = 2000) -> int:
    """Runs the bounded-wait self-test; returns the status (RCFAR_ERR_TIMEOUT expected)."""
    return int(lib().rcfar_selftest_wait(int(device), int(polls)))


# ---- batch tuning -------------------------------------------------------------

def make_batch_tuning(dft_kblocks_per_cta: int = 0, sat_mode: int = RCFAR_SAT_TILE_I64, cfar_tile=(0, 0),
                      dft_operands: int = 0):
    """dft_operands: 0 = band-DFT operands by the tensor memory accelerator, 1 = by cp.async."""
    return rcfar_batch_tuning(int(dft_kblocks_per_cta), int(sat_mode), int(cfar_tile[0]), int(cfar_tile[1]), 0.0, 0,
                              int(dft_operands))


def rcfar_tune_batch(h: int, frames: Sequence[rcfar_frame_desc], params: rcfar_pre_params, reps: int = 3,
                     stream=None) -> rcfar_batch_tuning:
    arr = (rcfar_frame_desc * len(frames))(*frames)
    out = rcfar_batch_tuning()
    _check(lib().rcfar_tune_batch(h, arr, len(frames), ctypes.byref(params), int(reps), ctypes.byref(out),
                                  _stream(stream)), "rcfar_tune_batch")
    return out


def rcfar_set_batch_tuning(h: int, t: rcfar_batch_tuning):
    _check(lib().rcfar_set_batch_tuning(h, ctypes.byref(t)), "rcfar_set_batch_tuning")


def rcfar_get_batch_tuning(h: int) -> rcfar_batch_tuning:
    out = rcfar_batch_tuning()
    _check(lib().rcfar_get_batch_tuning(h, ctypes.byref(out)), "rcfar_get_batch_tuning")
    return out


def rcfar_sat_cfar(h: int, map_t, value_bound: float, window: rcfar_window, cut_c_lo: int, cut_c_hi: int, det,
                   thr=None, map_cut: bool = True, map_exp2: int = 0, stream=None):
    """Fused SAT + CFAR (no table in device memory); same decisions as rcfar_sat + rcfar_cfar."""
    import torch
    _require(map_t, "map", _f32_f16())
    rows, cols = int(map_t.shape[0]), int(map_t.shape[1])
    _require(det, "det", _u8(), rows, cols)
    if thr is not None:
        _require(thr, "thr", _f32(), rows, cols)
    dtype = RCFAR_MAP_F16 if map_t.dtype == torch.float16 else RCFAR_MAP_F32
    _check(lib().rcfar_sat_cfar(h, _ptr(map_t), dtype, int(map_exp2), rows, cols, _ld(map_t), float(value_bound),
                                ctypes.byref(window), int(cut_c_lo), int(cut_c_hi), 1 if map_cut else 0, _ptr(det),
                                _ld(det), _ptr(thr), _ld(thr) if thr is not None else 0, _stream(stream)),
           "rcfar_sat_cfar")
