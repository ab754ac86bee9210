"""Python binding of the NTF C ABI (include/ntf.h): argument marshalling only.

Every computation runs in ``libntf.so``; this module checks tensor devices, dtypes, shapes
and contiguity, passes raw device pointers and the current CUDA stream, and turns status
codes into exceptions.  There is no fallback: if the library is missing or cannot be
loaded, importing the entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libntf.so")

NTF_F32, NTF_BF16 = 0, 1
NTF_KR_PRIMAL, NTF_KR_AUX = 0, 1
NTF_RHO_ADAPTIVE, NTF_RHO_TRACE, NTF_RHO_FIXED = 0, 1, 2
NTF_CONTRACT_AUTO, NTF_CONTRACT_TENSOR, NTF_CONTRACT_SIMT = 0, 1, 2
NTF_CONSTRAINT_NONNEG, NTF_CONSTRAINT_BOX, NTF_CONSTRAINT_SPARSE = 0, 1, 2

STATUS = {
    0: "NTF_OK", 1: "NTF_ERR_INVALID_ARG", 2: "NTF_ERR_CUDA", 3: "NTF_ERR_OOM",
    4: "NTF_ERR_NOT_SPD", 5: "NTF_ERR_NONFINITE", 6: "NTF_ERR_NOT_CONVERGED",
    7: "NTF_ERR_TIMEOUT", 8: "NTF_ERR_UNSUPPORTED",
}


class NTFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("inner_iters", ctypes.c_int), ("kr_source", ctypes.c_int),
                ("rho_policy", ctypes.c_int), ("rho0", ctypes.c_double),
                ("mu", ctypes.c_double), ("tau_incr", ctypes.c_double),
                ("tau_decr", ctypes.c_double), ("eps_abs", ctypes.c_double),
                ("eps_rel", ctypes.c_double), ("contraction", ctypes.c_int),
                ("kkt_dual_tol", ctypes.c_double), ("kkt_comp_tol", ctypes.c_double),
                ("fuse_level", ctypes.c_int), ("tensor_copy", ctypes.c_int)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("stream", ctypes.c_int), ("mode", ctypes.c_int),
                ("start_us", ctypes.c_double), ("end_us", ctypes.c_double)]


class UpdateStats(ctypes.Structure):
    _fields_ = [("primal_res", ctypes.c_double), ("dual_res", ctypes.c_double),
                ("norm_A", ctypes.c_double), ("norm_At", ctypes.c_double),
                ("norm_Y", ctypes.c_double), ("rho", ctypes.c_double),
                ("kkt_neg_x", ctypes.c_double), ("kkt_dual", ctypes.c_double),
                ("kkt_comp", ctypes.c_double)]


class RunStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("reached_target", ctypes.c_int), ("kkt_met", ctypes.c_int),
                ("rel_err", ctypes.c_double), ("kkt_dual", ctypes.c_double),
                ("kkt_comp", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("contractions", ctypes.c_int64 * 2), ("contraction_ms", ctypes.c_double * 2),
                ("contraction_bytes", ctypes.c_double * 2),
                ("ws_rows_considered", ctypes.c_int64), ("ws_rows_accepted", ctypes.c_int64),
                ("tensor_copy_bytes", ctypes.c_int64)]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "ntf_default_params": (None, [ctypes.POINTER(Params), ctypes.c_int]),
    "ntf_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_I64),
                                  ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(Params), _P]),
    "ntf_destroy": (ctypes.c_int, [_P]),
    "ntf_tensor_norm2": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ntf_mttkrp": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), _P]),
    "ntf_gram": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "ntf_system": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ntf_admm_update": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P,
                                       ctypes.POINTER(UpdateStats)]),
    "ntf_set_rho": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "ntf_set_constraint": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, _I64]),
    "ntf_get_rho": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ntf_fit": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double)]),
    "ntf_fit_from_mttkrp": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ntf_fit_explicit": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double)]),
    "ntf_run": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                               ctypes.c_int, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(RunStats)]),
    "ntf_sync": (ctypes.c_int, [_P]),
    "ntf_watchdog_check": (ctypes.c_int, [_P, ctypes.c_double]),
    "ntf_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ntf_profile_get": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "ntf_to_bf16": (ctypes.c_int, [_P, _P, _I64, _P]),
    "ntf_mlp_param_count": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int]),
    "ntf_mlp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, _P,
                                      ctypes.c_int, ctypes.c_int, _P]),
    "ntf_mlp_destroy": (ctypes.c_int, [_P]),
    "ntf_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "ntf_mlp_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P]),
    "ntf_mlp_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_int,
                                          ctypes.c_float, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "ntf_mlp_last_error": (ctypes.c_char_p, []),
    "ntf_attach_warmstart": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "ntf_warmstart_rows": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P,
                                          ctypes.POINTER(ctypes.c_double)]),
    "ntf_trace_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ntf_trace_get": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]),
    "ntf_mttkrp_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_I64), ctypes.c_int,
                                          ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(_P), _P,
                                          _P]),
    "ntf_sptensor_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int,
                                           ctypes.POINTER(_I64), _I64, _P, _P, _P]),
    "ntf_sptensor_destroy": (ctypes.c_int, [_P]),
    "ntf_sptensor_mttkrp": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P),
                                           _P]),
    "ntf_sptensor_nnz": (_I64, [_P]),
    "ntf_sptensor_last_error": (ctypes.c_char_p, []),
    "ntf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ntf_last_error": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libntf.so (built in-tree by ``paper_1409_2383_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1409_2383_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        raise NTFError(status, lib().ntf_last_error().decode())


def default_params(paper_mode: bool = False, **overrides) -> Params:
    p = Params()
    lib().ntf_default_params(ctypes.byref(p), 1 if paper_mode else 0)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _ptr_array(ts: Sequence[Optional[torch.Tensor]]):
    arr = (_P * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t)
    return arr


def _mat(t: torch.Tensor, rows: int, R: int, name: str, dtype=torch.float32,
         device: Optional[torch.device] = None) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the tensor on {device}")
    if t.dtype != dtype or tuple(t.shape) != (rows, R) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape ({rows}, {R}); "
                         f"got {t.dtype} {tuple(t.shape)}")


def to_bf16(x: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """FP32 -> BF16 (round to nearest even) with the library's conversion kernel.  x: a CUDA
    tensor, or a page-locked (pinned) host tensor, which the kernel reads directly over the
    host link (copy and conversion in one pass; the result is on the current CUDA device)."""
    pinned = not x.is_cuda and x.is_pinned()
    if x.dtype != torch.float32 or not (x.is_cuda or pinned) or not x.is_contiguous():
        raise ValueError("to_bf16 needs a contiguous float32 tensor on the GPU or pinned")
    dev = x.device if x.is_cuda else torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(x.shape, dtype=torch.bfloat16, device=dev)
    _check(lib().ntf_to_bf16(_ptr(x), _ptr(out), x.numel(), _stream_ptr(stream)))
    return out


def mttkrp_noalloc(X: torch.Tensor, mode: int, F: Sequence[Optional[torch.Tensor]],
                   out: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """MTTKRP without a context and without any device allocation inside the library (its
    scratch is a static device array shared by all calls on a GPU; calls that overlap on the
    GPU race on it).  For callers that cannot allocate device memory on their call path;
    ``out`` may be preallocated for the same reason."""
    if not isinstance(X, torch.Tensor) or not X.is_cuda or not X.is_contiguous():
        raise ValueError("X must be a contiguous CUDA tensor")
    if X.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("X must be float32 or bfloat16")
    dims = tuple(int(d) for d in X.shape)
    R = next(int(t.shape[1]) for m, t in enumerate(F) if m != mode)
    for m, t in enumerate(F):
        if m != mode:
            _mat(t, dims[m], R, f"factor {m}", device=X.device)
    if out is None:
        out = torch.empty(dims[mode], R, device=X.device)
    _mat(out, dims[mode], R, "out", device=X.device)
    cdims = (_I64 * len(dims))(*dims)
    dtype = NTF_F32 if X.dtype == torch.float32 else NTF_BF16
    with torch.cuda.device(X.device):      # the entry point works on the current device
        _check(lib().ntf_mttkrp_noalloc(len(dims), cdims, R, dtype, _ptr(X), mode,
                                        _ptr_array(F), _ptr(out), _stream_ptr(stream)))
    return out


class Context:
    """One tensor + rank + parameters; wraps ``ntf_ctx``.  Method names follow the ABI."""

    def __init__(self, X: torch.Tensor, rank: int, params: Optional[Params] = None,
                 stream: Optional[torch.cuda.Stream] = None):
        if not isinstance(X, torch.Tensor) or not X.is_cuda or not X.is_contiguous():
            raise ValueError("X must be a contiguous CUDA tensor")
        if X.dtype == torch.float32:
            dtype = NTF_F32
        elif X.dtype == torch.bfloat16:
            dtype = NTF_BF16
        else:
            raise ValueError("X must be float32 or bfloat16")
        self.X = X  # keeps the borrowed tensor alive
        self.dims = tuple(int(d) for d in X.shape)
        self.N = X.dim()
        self.R = int(rank)
        self.params = params if params is not None else default_params()
        self.stream = stream
        self._h = _P()
        dims = (_I64 * self.N)(*self.dims)
        with torch.cuda.device(X.device):
            _check(lib().ntf_create(ctypes.byref(self._h), self.N, dims, self.R, dtype,
                                    _ptr(X), ctypes.byref(self.params), _stream_ptr(stream)))

    def close(self) -> None:
        if self._h:
            lib().ntf_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- entry points -------------------------------------------------------------
    def tensor_norm2(self) -> float:
        v = ctypes.c_double()
        _check(lib().ntf_tensor_norm2(self._h, ctypes.byref(v)))
        return v.value

    def _factors(self, F: Sequence[Optional[torch.Tensor]], skip: int = -1):
        if len(F) != self.N:
            raise ValueError(f"need {self.N} factors")
        for m, t in enumerate(F):
            if m != skip:
                _mat(t, self.dims[m], self.R, f"factor {m}", device=self.X.device)
        return _ptr_array(F)

    def mttkrp(self, mode: int, F: Sequence[Optional[torch.Tensor]],
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.dims[mode], self.R, device=self.X.device)
        _mat(out, self.dims[mode], self.R, "out", device=self.X.device)
        _check(lib().ntf_mttkrp(self._h, mode, self._factors(F, skip=mode), _ptr(out)))
        return out

    def gram(self, mode: int, F: torch.Tensor, out: Optional[torch.Tensor] = None):
        _mat(F, self.dims[mode], self.R, "F", device=self.X.device)
        if out is not None:
            _mat(out, self.R, self.R, "out", torch.float64, self.X.device)
        _check(lib().ntf_gram(self._h, mode, _ptr(F), _ptr(out)))
        return out

    def system(self, mode: int, H: Optional[torch.Tensor] = None,
               L: Optional[torch.Tensor] = None) -> float:
        for t, n in ((H, "H"), (L, "L")):
            if t is not None:
                _mat(t, self.R, self.R, n, torch.float64, self.X.device)
        rho = ctypes.c_double()
        _check(lib().ntf_system(self._h, mode, _ptr(H), _ptr(L), ctypes.byref(rho)))
        return rho.value

    def admm_update(self, mode: int, M: torch.Tensor, A: torch.Tensor, At: torch.Tensor,
                    Y: torch.Tensor, stats: bool = True):
        for t, n in ((M, "M"), (A, "A"), (At, "At"), (Y, "Y")):
            _mat(t, self.dims[mode], self.R, n, device=self.X.device)
        st = UpdateStats() if stats else None
        _check(lib().ntf_admm_update(self._h, mode, _ptr(M), _ptr(A), _ptr(At), _ptr(Y),
                                     ctypes.byref(st) if st is not None else None))
        if st is None:
            return None
        return {k: getattr(st, k) for k, _ in UpdateStats._fields_}

    def set_constraint(self, mode: int, kind: int, lo: float = 0.0, hi: float = float("inf"),
                       max_nonzeros: int = 0) -> None:
        """Constraint set of factor `mode`'s auxiliary (NTF_CONSTRAINT_NONNEG / _BOX with
        [lo, hi] / _SPARSE with at most `max_nonzeros` nonzeros)."""
        _check(lib().ntf_set_constraint(self._h, mode, int(kind), float(lo), float(hi),
                                        int(max_nonzeros)))

    def set_rho(self, mode: int, rho: float) -> None:
        _check(lib().ntf_set_rho(self._h, mode, float(rho)))

    def get_rho(self, mode: int) -> float:
        v = ctypes.c_double()
        _check(lib().ntf_get_rho(self._h, mode, ctypes.byref(v)))
        return v.value

    def fit(self, F: Sequence[torch.Tensor]) -> float:
        v = ctypes.c_double()
        _check(lib().ntf_fit(self._h, self._factors(F), ctypes.byref(v)))
        return v.value

    def fit_explicit(self, F: Sequence[torch.Tensor]) -> float:
        """Relative error by explicit reconstruction (accurate at low noise)."""
        v = ctypes.c_double()
        _check(lib().ntf_fit_explicit(self._h, self._factors(F), ctypes.byref(v)))
        return v.value

    def fit_from_mttkrp(self, M_last: torch.Tensor, F_last: torch.Tensor) -> float:
        _mat(M_last, self.dims[-1], self.R, "M_last", device=self.X.device)
        _mat(F_last, self.dims[-1], self.R, "F_last", device=self.X.device)
        v = ctypes.c_double()
        _check(lib().ntf_fit_from_mttkrp(self._h, _ptr(M_last), _ptr(F_last), ctypes.byref(v)))
        return v.value

    def run(self, A: Sequence[torch.Tensor], At: Sequence[torch.Tensor],
            Y: Sequence[torch.Tensor], max_outer: int, target_rfe: float = 0.0,
            check_every: int = 1, history: bool = False, raise_not_converged: bool = False):
        """Outer iterations in place on (A, At, Y); returns a dict of run statistics."""
        pa, pt, py = self._factors(A), self._factors(At), self._factors(Y)
        hist = (ctypes.c_double * max_outer)() if history else None
        rs = RunStats()
        st = lib().ntf_run(self._h, pa, pt, py, int(max_outer), float(target_rfe),
                           int(check_every), hist, ctypes.byref(rs))
        if st != 0 and (st != 6 or raise_not_converged):
            _check(st)
        out = {k: getattr(rs, k) for k, _ in RunStats._fields_}
        if history:
            out["history"] = [hist[i] for i in range(max_outer)]
        return out

    def sync(self) -> None:
        _check(lib().ntf_sync(self._h))

    def watchdog_check(self, limit_ms: float) -> None:
        """Runs the bounded device-side wait on a barrier that nothing completes; raises
        NTFError (NTF_ERR_TIMEOUT) when it gave up, as it must."""
        _check(lib().ntf_watchdog_check(self._h, float(limit_ms)))

    def profile_enable(self, enable: bool = True) -> None:
        _check(lib().ntf_profile_enable(self._h, 1 if enable else 0))

    def profile_get(self) -> dict:
        p = Profile()
        _check(lib().ntf_profile_get(self._h, ctypes.byref(p)))
        return {"sweeps": p.sweeps, "kernel_launches": p.kernel_launches,
                "contractions": list(p.contractions), "contraction_ms": list(p.contraction_ms),
                "contraction_bytes": list(p.contraction_bytes),
                "ws_rows_considered": p.ws_rows_considered,
                "ws_rows_accepted": p.ws_rows_accepted,
                "tensor_copy_bytes": p.tensor_copy_bytes}

    def trace_enable(self, enable: bool = True) -> None:
        _check(lib().ntf_trace_enable(self._h, 1 if enable else 0))

    def trace_get(self) -> list:
        """Steps of the last traced outer iteration: dicts with name, stream, mode and
        start/end in microseconds from the iteration's start."""
        buf = (TraceEntry * 64)()
        n = ctypes.c_int(0)
        _check(lib().ntf_trace_get(self._h, ctypes.cast(buf, ctypes.c_void_p), 64,
                                   ctypes.byref(n)))
        return [{"name": buf[i].name.decode(), "stream": buf[i].stream, "mode": buf[i].mode,
                 "start_us": buf[i].start_us, "end_us": buf[i].end_us}
                for i in range(min(n.value, 64))]

    def warmstart_rows(self, mode: int, M: torch.Tensor, At: Optional[torch.Tensor] = None,
                       Y: Optional[torch.Tensor] = None):
        """Network inputs of factor `mode`'s rows (and targets [At ; Y/s] if At, Y are given)
        with the update's own coefficient system: (Gn [R, R], rows [I, 2R], targets or None,
        s)."""
        I, R = self.dims[mode], self.R
        _mat(M, I, R, "M", device=self.X.device)
        if (At is None) != (Y is None):
            raise ValueError("give both At and Y, or neither")
        if At is not None:
            _mat(At, I, R, "At", device=self.X.device)
            _mat(Y, I, R, "Y", device=self.X.device)
        Gn = torch.empty(R, R, device=self.X.device)
        rows = torch.empty(I, 2 * R, device=self.X.device)
        tg = torch.empty(I, 2 * R, device=self.X.device) if At is not None else None
        s = ctypes.c_double()
        _check(lib().ntf_warmstart_rows(self._h, mode, _ptr(M), _ptr(At), _ptr(Y), _ptr(Gn),
                                        _ptr(rows), _ptr(tg), ctypes.byref(s)))
        return Gn, rows, tg, s.value

    def attach_warmstart(self, net: Optional["Mlp"], sweeps: int = 0) -> None:
        """sweeps >= 1: consult the network in the first `sweeps` outer iterations of each
        run; 0: in every iteration."""
        _check(lib().ntf_attach_warmstart(self._h, net._h if net is not None else None,
                                          int(sweeps)))
        self._ws = net  # keep the network alive while attached


def _mcheck(status: int) -> None:
    if status != 0:
        raise NTFError(status, lib().ntf_mlp_last_error().decode())


class Mlp:
    """Warm-start network (wraps ``ntf_mlp``); parameters in the flat layout of the ABI."""

    def __init__(self, rank: int, hidden: int, params: torch.Tensor, max_rows: int,
                 max_groups: int, stream: Optional[torch.cuda.Stream] = None):
        n = int(lib().ntf_mlp_param_count(int(rank), int(hidden)))
        if n < 0:
            raise ValueError("bad rank or hidden width")
        p = params.detach().to("cpu", torch.float32).contiguous()
        if p.numel() != n:
            raise ValueError(f"expected {n} parameters, got {p.numel()}")
        self.R, self.H, self.count = int(rank), int(hidden), n
        self.stream = stream
        self._h = _P()
        _mcheck(lib().ntf_mlp_create(ctypes.byref(self._h), self.R, self.H, _ptr(p),
                                     int(max_rows), int(max_groups), _stream_ptr(stream)))

    def close(self) -> None:
        if self._h:
            lib().ntf_mlp_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> torch.Tensor:
        out = torch.empty(self.count, dtype=torch.float32)
        _mcheck(lib().ntf_mlp_get_params(self._h, _ptr(out)))
        return out

    def forward(self, Gn: torch.Tensor, offsets: torch.Tensor, mrows: torch.Tensor) -> torch.Tensor:
        groups, rows = int(offsets.numel()) - 1, int(mrows.shape[0])
        out = torch.empty(rows, 2 * self.R, device=mrows.device)
        _mcheck(lib().ntf_mlp_forward(self._h, _ptr(Gn), _ptr(offsets), groups, _ptr(mrows),
                                      rows, _ptr(out)))
        return out

    def train_step(self, Gn, offsets, mrows, targets, lr: float, apply: bool = True,
                   want_loss: bool = True, grad_out: Optional[torch.Tensor] = None):
        groups, rows = int(offsets.numel()) - 1, int(mrows.shape[0])
        loss = ctypes.c_double()
        _mcheck(lib().ntf_mlp_train_step(self._h, _ptr(Gn), _ptr(offsets), groups, _ptr(mrows),
                                         _ptr(targets), rows, float(lr), 1 if apply else 0,
                                         ctypes.byref(loss) if want_loss else None,
                                         _ptr(grad_out)))
        return loss.value if want_loss else None


def _scheck(status: int) -> None:
    if status != 0:
        raise NTFError(status, lib().ntf_sptensor_last_error().decode())


class SparseTensor:
    """A sparse tensor in coordinate form laid out for MTTKRP (wraps ``ntf_sptensor``):
    indices int32 [nnz, N] and values float32 [nnz] on the GPU."""

    def __init__(self, indices: torch.Tensor, values: torch.Tensor, dims: Sequence[int],
                 stream: Optional[torch.cuda.Stream] = None):
        if (not isinstance(indices, torch.Tensor) or not indices.is_cuda
                or indices.dtype != torch.int32 or indices.dim() != 2
                or not indices.is_contiguous()):
            raise ValueError("indices must be a contiguous int32 CUDA tensor [nnz, N]")
        if (not isinstance(values, torch.Tensor) or not values.is_cuda
                or values.dtype != torch.float32 or values.shape != (indices.shape[0],)
                or not values.is_contiguous() or values.device != indices.device):
            raise ValueError("values must be a contiguous float32 CUDA tensor [nnz]")
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        if indices.shape[1] != self.N:
            raise ValueError("indices must have one column per mode")
        self.device = indices.device
        self.stream = stream
        self._h = _P()
        cd = (_I64 * self.N)(*self.dims)
        with torch.cuda.device(self.device):
            _scheck(lib().ntf_sptensor_create(ctypes.byref(self._h), self.N, cd,
                                              int(indices.shape[0]), _ptr(indices),
                                              _ptr(values), _stream_ptr(stream)))

    @property
    def nnz(self) -> int:
        return int(lib().ntf_sptensor_nnz(self._h))

    def mttkrp(self, mode: int, F: Sequence[Optional[torch.Tensor]],
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
        R = next(int(t.shape[1]) for m, t in enumerate(F) if m != mode)
        for m, t in enumerate(F):
            if m != mode:
                _mat(t, self.dims[m], R, f"factor {m}", device=self.device)
        if out is None:
            out = torch.empty(self.dims[mode], R, device=self.device)
        _mat(out, self.dims[mode], R, "out", device=self.device)
        with torch.cuda.device(self.device):
            _scheck(lib().ntf_sptensor_mttkrp(self._h, mode, R, _ptr_array(F), _ptr(out)))
        return out

    def close(self) -> None:
        if self._h:
            lib().ntf_sptensor_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def zeros_state(dims: Sequence[int], R: int, device="cuda") -> List[torch.Tensor]:
    return [torch.zeros(d, R, device=device) for d in dims]


__all__ = ["Context", "Params", "NTFError", "default_params", "to_bf16", "lib", "zeros_state",
           "mttkrp_noalloc", "Mlp", "SparseTensor",
           "NTF_F32", "NTF_BF16", "NTF_KR_PRIMAL", "NTF_KR_AUX", "NTF_RHO_ADAPTIVE",
           "NTF_RHO_TRACE", "NTF_RHO_FIXED", "NTF_CONTRACT_AUTO", "NTF_CONTRACT_TENSOR",
           "NTF_CONTRACT_SIMT", "NTF_CONSTRAINT_NONNEG", "NTF_CONSTRAINT_BOX",
           "NTF_CONSTRAINT_SPARSE", "LIB_PATH"]
