"""Python binding of libpardtw (C-ABI in include/pardtw.h).

Argument marshalling only: every step of the alignment (normalisation, cost,
DP, backtrace) runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  If the shared library is missing or cannot be loaded
the calls raise -- there is no CPU fallback.

Low-level names follow the C-ABI (``dtw_cost``, ``dtw_align``,
``dtw_align_many``); ``Aligner`` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libpardtw.so")

DTW_OK = 0
DTW_ERR_INVALID = 1
DTW_ERR_UNREACHABLE = 2
DTW_ERR_OOM = 3
DTW_ERR_CUDA = 4
DTW_ERR_TIMEOUT = 5
DTW_ERR_UNSUPPORTED = 6
DTW_ERR_SCRATCH_LIMIT = 7
DTW_COST_FP32 = 0
DTW_COST_BF16 = 1

# every entry point include/pardtw.h declares
EXPORTS = ("dtw_default_options", "dtw_status_string", "dtw_create", "dtw_destroy",
           "dtw_set_stream", "dtw_workspace_size", "dtw_cost", "dtw_align", "dtw_align_many",
           "dtw_enable_timing", "dtw_stage_times", "dtw_align_static",
           "dtw_static_scratch_bytes", "dtw_align_banded", "dtw_encoder_param_count",
           "dtw_encode", "dtw_encoder_grad", "dtw_encoder_adam", "dtw_align_learned",
           "dtw_band_cells", "dtw_wsdtw", "dtw_wsdtw_cseg", "dtw_batch_create",
           "dtw_batch_run", "dtw_batch_info", "dtw_batch_destroy", "dtw_fp32_peak")
DTW_BATCH_AUTOTUNE = 1
TRANSPOSE_AUTO, TRANSPOSE_NEVER, TRANSPOSE_ALWAYS = 0, 1, 2

# learned band (include/pardtw.h)
DTW_BAND_WMIN = 256
DTW_BAND_WMAX = 2048
ENC_CHANNELS = 64
ENC_EMBED = 16
ENC_KERNEL = 5


class PardtwError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


class Options(ctypes.Structure):
    _fields_ = [("cost_precision", ctypes.c_int), ("cost_shift", ctypes.c_float),
                ("wait_limit", ctypes.c_int), ("debug_skip_publish", ctypes.c_int),
                ("rows_per_lane", ctypes.c_int), ("dp_schedule", ctypes.c_int),
                ("strips_per_cta", ctypes.c_int), ("transpose", ctypes.c_int),
                ("clusters", ctypes.c_int)]

SCHEDULE_AUTO, SCHEDULE_FUSED, SCHEDULE_SPLIT = 0, 1, 2
CLUSTERS_AUTO, CLUSTERS_NEVER = 0, 1


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpardtw.so (built by ``paper_2607_15478_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libpardtw.so not built at {path}; run "
                      "`python -m paper_2607_15478_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    ip = ctypes.POINTER(ci)
    lib.dtw_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.dtw_default_options.restype = None
    lib.dtw_status_string.argtypes = [ci]
    lib.dtw_status_string.restype = ctypes.c_char_p
    lib.dtw_create.argtypes = [ctypes.POINTER(vp), ci, vp]
    lib.dtw_destroy.argtypes = [vp]
    lib.dtw_set_stream.argtypes = [vp, vp]
    lib.dtw_workspace_size.argtypes = [ci, ci, ci, ctypes.POINTER(Options),
                                       ctypes.POINTER(ctypes.c_size_t)]
    lib.dtw_cost.argtypes = [vp, vp, ci, vp, ci, ci, vp]
    lib.dtw_align.argtypes = [vp, vp, ci, vp, ci, ci, ctypes.POINTER(Options), vp, ci, vp, vp]
    lib.dtw_align_banded.argtypes = [vp, vp, ci, vp, ci, ci, ctypes.POINTER(Options), ci, ci, vp,
                                     ci, vp, vp, ctypes.POINTER(ci)]
    lib.dtw_align_many.argtypes = [vp, ci, vp, vp, vp, vp, ci, ctypes.POINTER(Options), vp, vp,
                                   vp, vp, vp]
    lib.dtw_enable_timing.argtypes = [vp, ci]
    lib.dtw_stage_times.argtypes = [vp, ctypes.POINTER(cf), ci]
    lib.dtw_align_static.argtypes = [vp, ci, vp, ci, ci, ctypes.POINTER(Options), vp, vp, ci, vp,
                                     vp]
    lib.dtw_static_scratch_bytes.argtypes = []
    lib.dtw_static_scratch_bytes.restype = ctypes.c_size_t
    lib.dtw_encoder_param_count.argtypes = [ci]
    lib.dtw_encoder_param_count.restype = ctypes.c_size_t
    lib.dtw_encode.argtypes = [vp, vp, ci, vp, ci, ci, ci, vp, vp]
    lib.dtw_encoder_grad.argtypes = [vp, vp, ci, ci, vp, ci, vp, ci, vp, vp, ci, vp, vp]
    lib.dtw_encoder_adam.argtypes = [vp, ci, vp, vp, vp, vp, ci, cf]
    lib.dtw_align_learned.argtypes = [vp, vp, ci, vp, ci, ci, ctypes.POINTER(Options), vp, ci,
                                      ci, vp, ci, vp, vp, ctypes.POINTER(ci)]
    lib.dtw_band_cells.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.dtw_wsdtw.argtypes = [vp, vp, ci, vp, ci, ci, ci, vp, ci, vp, vp, vp]
    lib.dtw_wsdtw_cseg.argtypes = [vp, ci, ci, vp]
    lib.dtw_batch_create.argtypes = [vp, ci, vp, vp, vp, vp, ci, vp, vp, vp, vp, ci,
                                     ctypes.POINTER(vp)]
    lib.dtw_batch_run.argtypes = [vp]
    lib.dtw_batch_info.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(cf)]
    lib.dtw_batch_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name not in ("dtw_default_options", "dtw_status_string", "dtw_static_scratch_bytes",
                        "dtw_encoder_param_count"):
            getattr(lib, name).restype = ci
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load_library().dtw_status_string(int(status)).decode()


def make_options(cost_shift: float = 0.0, wait_limit_us: int = 0,
                 debug_skip_publish: int = -1, rows_per_lane: int = 0,
                 dp_schedule: int = SCHEDULE_AUTO, cost_precision: int = DTW_COST_FP32,
                 strips_per_cta: int = 0, transpose: int = 0, clusters: int = 0) -> Options:
    o = Options()
    load_library().dtw_default_options(ctypes.byref(o))
    o.cost_precision = int(cost_precision)
    o.cost_shift = float(cost_shift)
    o.wait_limit = int(wait_limit_us)
    o.debug_skip_publish = int(debug_skip_publish)
    o.rows_per_lane = int(rows_per_lane)
    o.dp_schedule = int(dp_schedule)
    o.strips_per_cta = int(strips_per_cta)
    o.transpose = int(transpose)
    o.clusters = int(clusters)
    return o


def workspace_size(La: int, Lb: int, D: int, options: Options | None = None) -> int:
    n = ctypes.c_size_t(0)
    rc = load_library().dtw_workspace_size(La, Lb, D, ctypes.byref(options) if options else None,
                                           ctypes.byref(n))
    if rc != DTW_OK:
        raise PardtwError(rc, "dtw_workspace_size")
    return n.value


def _check(rc: int, what: str):
    if rc != DTW_OK:
        raise PardtwError(rc, what)


def _features(X):
    import torch
    if not isinstance(X, torch.Tensor):
        X = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32))
    if X.dtype != torch.float32 or X.dim() != 2:
        raise ValueError("features must be a 2-D float32 tensor (L x D)")
    return X.contiguous()


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C-ABI mirrors ------------------------------------------------------------------

def dtw_create(device: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load_library().dtw_create(ctypes.byref(h), int(device), _stream_ptr(stream)),
           "dtw_create")
    return h.value


def dtw_destroy(h: int) -> None:
    _check(load_library().dtw_destroy(h), "dtw_destroy")


def dtw_cost(h: int, A, B, C) -> None:
    """C[i, j] = 1 - cos(a_i, b_j) into the La x Lb float32 tensor C."""
    A, B = _features(A), _features(B)
    _check(load_library().dtw_cost(h, A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0],
                                   A.shape[1], C.data_ptr()), "dtw_cost")


def dtw_align(h: int, A, B, path, path_len, total=None, options: Options | None = None) -> None:
    """Exact DTW of A and B into caller buffers (path: cap x 2 int32; path_len: int32[1];
    total: float32[1] or None).  Asynchronous when every buffer is on the device."""
    A, B = _features(A), _features(B)
    cap = path.shape[0]
    _check(load_library().dtw_align(h, A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0],
                                    A.shape[1], ctypes.byref(options) if options else None,
                                    path.data_ptr(), cap, path_len.data_ptr(),
                                    total.data_ptr() if total is not None else None),
           "dtw_align")


def dtw_align_many(h: int, As: Sequence, Bs: Sequence, paths, path_off, path_len, cost, status,
                   options: Options | None = None) -> None:
    """Batched exact DTW; per-pair outputs as in include/pardtw.h."""
    n = len(As)
    As = [_features(a) for a in As]
    Bs = [_features(b) for b in Bs]
    D = As[0].shape[1] if n else 1
    Ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in As])
    Bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in Bs])
    La = (ctypes.c_int * n)(*[a.shape[0] for a in As])
    Lb = (ctypes.c_int * n)(*[b.shape[0] for b in Bs])
    off = (ctypes.c_int64 * n)(*[int(x) for x in path_off])
    _check(load_library().dtw_align_many(
        h, n, ctypes.cast(Ap, ctypes.c_void_p), ctypes.cast(La, ctypes.c_void_p),
        ctypes.cast(Bp, ctypes.c_void_p), ctypes.cast(Lb, ctypes.c_void_p), D,
        ctypes.byref(options) if options else None, paths.data_ptr(),
        ctypes.cast(off, ctypes.c_void_p), path_len.data_ptr(),
        cost.data_ptr() if cost is not None else None, status.data_ptr()), "dtw_align_many")


def dtw_align_banded(h: int, A, B, path, path_len, total=None, downsample: int = 8,
                     halfwidth: int = 256, options: Options | None = None) -> bool:
    """Exact DTW inside the band of the coarse alignment (include/pardtw.h);
    returns True when the band was given up for the full exact DTW."""
    A, B = _features(A), _features(B)
    fb = ctypes.c_int(0)
    _check(load_library().dtw_align_banded(
        h, A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1],
        ctypes.byref(options) if options else None, int(downsample), int(halfwidth),
        path.data_ptr(), path.shape[0], path_len.data_ptr(),
        total.data_ptr() if total is not None else None, ctypes.byref(fb)), "dtw_align_banded")
    return bool(fb.value)


def dtw_encoder_param_count(D: int) -> int:
    return int(load_library().dtw_encoder_param_count(int(D)))


def dtw_encode(h: int, params, X, emb, halfwidth=None, downsample: int = 8,
               bf16: bool = False) -> None:
    """Band encoder forward of one sequence (include/pardtw.h)."""
    X = _features(X)
    _check(load_library().dtw_encode(
        h, params.data_ptr(), X.shape[1], X.data_ptr(), X.shape[0], int(downsample), int(bf16),
        emb.data_ptr(), halfwidth.data_ptr() if halfwidth is not None else None), "dtw_encode")


def dtw_encoder_grad(h: int, params, A, B, path, path_len, mode: int, grad, loss,
                     downsample: int = 8) -> None:
    """Adds one pair's loss gradient (mode 0: embedding, 1: half-width) to grad."""
    A, B = _features(A), _features(B)
    _check(load_library().dtw_encoder_grad(
        h, params.data_ptr(), A.shape[1], int(downsample), A.data_ptr(), A.shape[0],
        B.data_ptr(), B.shape[0], path.data_ptr(), path_len.data_ptr(), int(mode),
        grad.data_ptr(), loss.data_ptr()), "dtw_encoder_grad")


def dtw_encoder_adam(h: int, params, grad, m, v, step: int, lr: float) -> None:
    _check(load_library().dtw_encoder_adam(
        h, params.numel(), params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(),
        int(step), float(lr)), "dtw_encoder_adam")


def dtw_align_learned(h: int, A, B, params, path, path_len, total=None, downsample: int = 8,
                      bf16: bool = True, options: Options | None = None) -> bool:
    """Exact DTW inside the learned band; returns True when it fell back to
    the full exact DTW."""
    A, B = _features(A), _features(B)
    fb = ctypes.c_int(0)
    _check(load_library().dtw_align_learned(
        h, A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1],
        ctypes.byref(options) if options else None, params.data_ptr(), int(downsample),
        int(bf16), path.data_ptr(), path.shape[0], path_len.data_ptr(),
        total.data_ptr() if total is not None else None, ctypes.byref(fb)), "dtw_align_learned")
    return bool(fb.value)


def dtw_wsdtw(h: int, A, B, nfrag: int, path, path_len, ends=None, total=None) -> None:
    """Weakly-ordered Segmental DTW of query A against reference B (include/pardtw.h)."""
    A, B = _features(A), _features(B)
    _check(load_library().dtw_wsdtw(
        h, A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1], int(nfrag),
        path.data_ptr(), path.shape[0], path_len.data_ptr(),
        ends.data_ptr() if ends is not None else None,
        total.data_ptr() if total is not None else None), "dtw_wsdtw")


def dtw_wsdtw_cseg(h: int, nfrag: int, Lb: int, cseg) -> None:
    _check(load_library().dtw_wsdtw_cseg(h, int(nfrag), int(Lb), cseg.data_ptr()),
           "dtw_wsdtw_cseg")


def dtw_band_cells(h: int) -> int:
    c = ctypes.c_longlong(0)
    _check(load_library().dtw_band_cells(h, ctypes.byref(c)), "dtw_band_cells")
    return int(c.value)


def dtw_align_static(A, B, path, path_len, total=None, options: Options | None = None,
                     stream=None) -> None:
    """Exact DTW into caller device buffers without any device allocation.

    For callers that cannot allocate device memory while they align (a
    real-time loop that must not block in the allocator, or a process whose
    device memory is reserved by another allocator).  The library keeps all
    scratch in one fixed device array (``dtw_static_scratch_bytes()``); too
    large a problem raises ``PardtwError`` with ``DTW_ERR_SCRATCH_LIMIT``.
    All tensors must be on the device; calls overlapping on the GPU race.
    """
    A, B = _features(A), _features(B)
    _check(load_library().dtw_align_static(
        A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1],
        ctypes.byref(options) if options else None, _stream_ptr(stream), path.data_ptr(),
        path.shape[0], path_len.data_ptr(), total.data_ptr() if total is not None else None),
        "dtw_align_static")


def dtw_static_scratch_bytes() -> int:
    return int(load_library().dtw_static_scratch_bytes())


def fp32_peak(device: int = 0, iters: int = 4096) -> float:
    """Measured FP32 FMA throughput of the device (FFMA per second)."""
    v = ctypes.c_double(0.0)
    _check(load_library().dtw_fp32_peak(int(device), int(iters), ctypes.byref(v)),
           "dtw_fp32_peak")
    return float(v.value)


class BatchPlan:
    """A planned batch (dtw_batch_create): fixed device inputs, outputs owned
    here, the DP schedule chosen by the autotuner, one CUDA graph per run."""

    def __init__(self, h: int, As: Sequence, Bs: Sequence, autotune: bool = True):
        import torch
        n = len(As)
        self.As = [_features(a) for a in As]
        self.Bs = [_features(b) for b in Bs]
        dev = self.As[0].device
        D = self.As[0].shape[1]
        caps = [min(a.shape[0], b.shape[0]) for a, b in zip(self.As, self.Bs)]
        self.off = np.concatenate([[0], np.cumsum(caps)[:-1]]).astype(np.int64)
        self.paths = torch.empty((int(sum(caps)), 2), dtype=torch.int32, device=dev)
        self.path_len = torch.zeros(n, dtype=torch.int32, device=dev)
        self.cost = torch.zeros(n, dtype=torch.float32, device=dev)
        Ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in self.As])
        Bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in self.Bs])
        La = (ctypes.c_int * n)(*[a.shape[0] for a in self.As])
        Lb = (ctypes.c_int * n)(*[b.shape[0] for b in self.Bs])
        off = (ctypes.c_int64 * n)(*[int(x) for x in self.off])
        b = ctypes.c_void_p(0)
        _check(load_library().dtw_batch_create(
            h, n, ctypes.cast(Ap, ctypes.c_void_p), ctypes.cast(La, ctypes.c_void_p),
            ctypes.cast(Bp, ctypes.c_void_p), ctypes.cast(Lb, ctypes.c_void_p), D,
            self.paths.data_ptr(), ctypes.cast(off, ctypes.c_void_p), self.path_len.data_ptr(),
            self.cost.data_ptr(), DTW_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(b)),
            "dtw_batch_create")
        self.b = b.value

    def run(self) -> None:
        _check(load_library().dtw_batch_run(self.b), "dtw_batch_run")

    def info(self):
        """(rows per lane, strips per CTA, autotuner times in ms: 2, 3, 4 rows per
        lane with two strips per CTA, then with four; -1 where not tried)."""
        R, NS = ctypes.c_int(0), ctypes.c_int(0)
        t = (ctypes.c_float * 6)()
        _check(load_library().dtw_batch_info(self.b, ctypes.byref(R), ctypes.byref(NS), t),
               "dtw_batch_info")
        return R.value, NS.value, [float(x) for x in t]

    def results(self):
        """(list of paths, costs, path lengths) of the last run (synchronises)."""
        lens = self.path_len.cpu().numpy()
        out = [self.paths[self.off[k]:self.off[k] + lens[k]] if lens[k] > 0 else None
               for k in range(len(lens))]
        return out, self.cost.cpu().numpy(), lens

    def close(self) -> None:
        if getattr(self, "b", None):
            load_library().dtw_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper --------------------------------------------------------------

class Aligner:
    """A library handle bound to a device and a stream, with tensor-level calls."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = torch.device("cuda", device)
        self._stream = stream
        self.h = dtw_create(device, stream)

    def close(self):
        for plan in list(getattr(self, "_plans", ())):
            plan.close()
        if getattr(self, "h", None):
            dtw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _enter(self):
        """The handle's stream waits for the work queued so far on torch's current
        stream (the inputs), so that a handle with its own stream sees them."""
        if self._stream is not None:
            import torch
            self._stream.wait_stream(torch.cuda.current_stream(self.device))

    def _leave(self):
        """torch's current stream waits for the handle's work (the outputs)."""
        if self._stream is not None:
            import torch
            torch.cuda.current_stream(self.device).wait_stream(self._stream)

    def enable_timing(self, on: bool = True):
        _check(load_library().dtw_enable_timing(self.h, int(on)), "dtw_enable_timing")

    def stage_times(self) -> Tuple[float, float, float]:
        ms = (ctypes.c_float * 3)()
        _check(load_library().dtw_stage_times(self.h, ms, 3), "dtw_stage_times")
        return tuple(ms)

    def cost(self, A, B):
        import torch
        A, B = _features(A), _features(B)
        C = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float32,
                        device=A.device if A.is_cuda else self.device)
        self._enter()
        dtw_cost(self.h, A, B, C)
        self._leave()
        return C

    def align_into(self, A, B, path, path_len, total, **opts):
        """Asynchronous form: all outputs are caller-owned device tensors."""
        self._enter()
        dtw_align(self.h, A, B, path, path_len, total, make_options(**opts) if opts else None)
        self._leave()

    def align(self, A, B, **opts):
        """Return (path as an (n, 2) int32 tensor on the device, total cost as float)."""
        import torch
        A, B = _features(A), _features(B)
        cap = min(A.shape[0], B.shape[0])
        dev = A.device if A.is_cuda else self.device
        path = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        plen = torch.zeros(1, dtype=torch.int32, device=dev)
        tot = torch.zeros(1, dtype=torch.float32, device=dev)
        self._enter()
        dtw_align(self.h, A, B, path, plen, tot, make_options(**opts) if opts else None)
        self._leave()
        n = int(plen.item())
        if n < 0:
            raise PardtwError(-n, "dtw_align (device)")
        return path[:n], float(tot.item())

    def align_banded(self, A, B, downsample: int = 8, halfwidth: int = 256, **opts):
        """Banded exact DTW; returns (path, total, fell_back)."""
        import torch
        A, B = _features(A), _features(B)
        cap = min(A.shape[0], B.shape[0])
        path = torch.empty((cap, 2), dtype=torch.int32, device=A.device)
        plen = torch.zeros(1, dtype=torch.int32, device=A.device)
        tot = torch.zeros(1, dtype=torch.float32, device=A.device)
        self._enter()
        fb = dtw_align_banded(self.h, A, B, path, plen, tot, downsample, halfwidth,
                              make_options(**opts) if opts else None)
        self._leave()
        n = int(plen.item())
        if n < 0:
            raise PardtwError(-n, "dtw_align_banded (device)")
        return path[:n], float(tot.item()), fb

    def align_learned(self, A, B, params, downsample: int = 8, bf16: bool = True, **opts):
        """Exact DTW in the learned band; returns (path, total, fell_back)."""
        import torch
        A, B = _features(A), _features(B)
        cap = min(A.shape[0], B.shape[0])
        path = torch.empty((cap, 2), dtype=torch.int32, device=A.device)
        plen = torch.zeros(1, dtype=torch.int32, device=A.device)
        tot = torch.zeros(1, dtype=torch.float32, device=A.device)
        self._enter()
        fb = dtw_align_learned(self.h, A, B, params, path, plen, tot, downsample, bf16,
                               make_options(**opts) if opts else None)
        self._leave()
        n = int(plen.item())
        if n < 0:
            raise PardtwError(-n, "dtw_align_learned (device)")
        return path[:n], float(tot.item()), fb

    def encode(self, X, params, downsample: int = 8, bf16: bool = False):
        """Band encoder forward: (embeddings, half-widths) of one sequence."""
        import torch
        X = _features(X)
        Lc = (X.shape[0] + downsample - 1) // downsample
        emb = torch.empty((Lc, ENC_EMBED), dtype=torch.float32, device=X.device)
        hw = torch.empty(Lc, dtype=torch.float32, device=X.device)
        self._enter()
        dtw_encode(self.h, params, X, emb, hw, downsample, bf16)
        self._leave()
        return emb, hw

    def band_cells(self) -> int:
        return dtw_band_cells(self.h)

    def wsdtw(self, A, B, nfrag: int):
        """WSDTW; returns (path, ends, total)."""
        import torch
        A, B = _features(A), _features(B)
        path = torch.empty((A.shape[0], 2), dtype=torch.int32, device=A.device)
        plen = torch.zeros(1, dtype=torch.int32, device=A.device)
        ends = torch.empty(nfrag, dtype=torch.int32, device=A.device)
        tot = torch.zeros(1, dtype=torch.float32, device=A.device)
        self._enter()
        dtw_wsdtw(self.h, A, B, nfrag, path, plen, ends, tot)
        self._leave()
        n = int(plen.item())
        if n < 0:
            raise PardtwError(-n, "dtw_wsdtw (device)")
        return path[:n], ends, float(tot.item())

    def wsdtw_cseg(self, nfrag: int, Lb: int):
        import torch
        c = torch.empty((nfrag, Lb), dtype=torch.float32, device=self.device)
        self._enter()
        dtw_wsdtw_cseg(self.h, nfrag, Lb, c)
        self._leave()
        return c

    def plan_batch(self, As: List, Bs: List, autotune: bool = True) -> "BatchPlan":
        """A graph-captured, autotuned plan of this batch (runs on this handle's
        stream; closed with this Aligner at the latest)."""
        import weakref
        self._enter()
        plan = BatchPlan(self.h, As, Bs, autotune)
        self._leave()
        if not hasattr(self, "_plans"):
            self._plans = weakref.WeakSet()
        self._plans.add(plan)
        return plan

    def align_many(self, As: List, Bs: List, **opts):
        """Align independent pairs; returns (list of paths or None, costs, statuses)."""
        import torch
        n = len(As)
        caps = [min(a.shape[0], b.shape[0]) for a, b in zip(As, Bs)]
        off = np.concatenate([[0], np.cumsum(caps)[:-1]]).astype(np.int64) if n else []
        paths = torch.empty((int(sum(caps)), 2), dtype=torch.int32, device=self.device)
        plen = torch.zeros(n, dtype=torch.int32, device=self.device)
        cost = torch.zeros(n, dtype=torch.float32, device=self.device)
        status = torch.zeros(n, dtype=torch.int32, device=self.device)
        self._enter()
        dtw_align_many(self.h, As, Bs, paths, off, plen, cost, status,
                       make_options(**opts) if opts else None)
        self._leave()
        plen_h = plen.cpu().numpy()
        st = status.cpu().numpy()
        out = []
        for k in range(n):
            out.append(paths[off[k]:off[k] + plen_h[k]] if st[k] == 0 else None)
        return out, cost.cpu().numpy(), st
