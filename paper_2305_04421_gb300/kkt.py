"""Thin ctypes binding of the C ABI in include/kkt.h (argument marshalling only).

Every function here forwards to ``libkkt.so``; all arithmetic of the method runs in the
library's CUDA kernels. Device vectors are torch CUDA float64 tensors (contiguous, layout
[u | z | w] x [n][j][i] as in the header); the stream defaults to torch's current stream.
If the library is missing, loading raises: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkkt.so")

KKT_OK = 0
KKT_NOT_CONVERGED = 1
KKT_ERR_INVALID_ARG = -1
KKT_ERR_OOM = -2
KKT_ERR_CUDA = -3
KKT_ERR_NONFINITE = -4
KKT_ERR_TIMEOUT = -5
KKT_ERR_BREAKDOWN = -6
KKT_ERR_UNSUPPORTED = -7

PREC = {"fp64": 0, "bf16": 1, "tf32": 2}
COARSE = {"exact": 0, "none": 1, "learned": 2}
VARIANT = {"multiplicative": 0, "additive": 1}
POU = {"left": 0, "right": 1}
NORM = {"l2": 0, "euclidean": 1}
ORTH = {"mgs": 0, "cgs2": 1, "mgs2": 2, "mgs4": 3, "mgs8": 4}
BASIS = {"physical": 0, "spectral": 1}
LOCAL = {"rasq": 0, "ras": 1}
COARSE_SOLVE = {"auto": 0, "thomas": 1, "cyclic": 2}
STAGING = {"auto": 0, "copy_engine": 1}
DST_METHOD = {"auto": 0, "tiles": 1, "lane": 2, "tensor": 3}
MLP_MODE = {"learned": 0, "none": 1, "network": 2}
HISTORY_MAX = 1024


class KKTOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("coarse", ctypes.c_int), ("variant", ctypes.c_int),
                ("pou", ctypes.c_int), ("restart", ctypes.c_int), ("jhat_sign", ctypes.c_int),
                ("residual_norm", ctypes.c_int), ("tc_split", ctypes.c_int), ("orth", ctypes.c_int),
                ("basis", ctypes.c_int), ("local", ctypes.c_int),
                ("Lx", ctypes.c_double),
                ("Ly", ctypes.c_double), ("coarse_solve", ctypes.c_int)]


class KKTInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Nt", ctypes.c_int), ("n_sub", ctypes.c_int),
                ("N", ctypes.c_longlong), ("V", ctypes.c_longlong), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dt", ctypes.c_double), ("h", ctypes.c_double),
                ("workspace_bytes", ctypes.c_longlong)]


class KKTStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("precond_applies", ctypes.c_int),
                ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_euclid", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("history_len", ctypes.c_int), ("history", ctypes.c_double * HISTORY_MAX)]


# "graph" is a replayed CUDA graph of the batched form: its kernels are counted in their own
# classes, its device time, flops and bytes under "graph"; it is not itself a kernel launch.
KERNEL_CLASSES = ["dst", "coarse", "sweep", "matvec", "multidot", "update", "axpy", "reduce", "graph", "pack"]
_NK = len(KERNEL_CLASSES)


class KKTKernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * _NK), ("ms", ctypes.c_double * _NK),
                ("timed", ctypes.c_longlong * _NK), ("flops", ctypes.c_double * _NK),
                ("bytes", ctypes.c_double * _NK)]


BATCH_MAX = 256


class KKTInstance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Nt", ctypes.c_int), ("n_sub", ctypes.c_int),
                ("T", ctypes.c_double), ("nu", ctypes.c_double), ("omega", ctypes.c_double)]


class KKTBatchStats(ctypes.Structure):
    _fields_ = [("solo", ctypes.c_int), ("waves", ctypes.c_int), ("graphs", ctypes.c_int),
                ("graph_launches", ctypes.c_longlong),
                ("tile_lines", ctypes.c_int), ("sweep_block", ctypes.c_int),
                ("tune_ms_dst", ctypes.c_double * 3), ("tune_ms_sweep", ctypes.c_double * 3),
                ("time_ms", ctypes.c_double), ("iterations", ctypes.c_int * BATCH_MAX),
                ("status", ctypes.c_int * BATCH_MAX), ("rel_residual", ctypes.c_double * BATCH_MAX)]


class KKTMlpConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("Nt", ctypes.c_int), ("n_sub", ctypes.c_int), ("modes", ctypes.c_int),
                ("width", ctypes.c_int), ("seed", ctypes.c_int), ("samples", ctypes.c_int), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("T", ctypes.c_double), ("nu_lo", ctypes.c_double), ("nu_hi", ctypes.c_double),
                ("omega_lo", ctypes.c_double), ("omega_hi", ctypes.c_double), ("lr", ctypes.c_double),
                ("resid_epochs", ctypes.c_int)]


class KKTMlpTrainStats(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int), ("steps", ctypes.c_int), ("final_train_loss", ctypes.c_double),
                ("val_loss", ctypes.c_double), ("val_cosine", ctypes.c_double), ("val_resid", ctypes.c_double),
                ("val_within_guard", ctypes.c_double)]


class KKTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"kkt status {status}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("kkt_last_error", ctypes.c_char_p, []),
    ("kkt_status_string", ctypes.c_char_p, [_I]),
    ("kkt_default_options", _I, [ctypes.POINTER(KKTOptions)]),
    ("kkt_create", _P, [_I, _I, _I, _D, _D, _D, _I]),
    ("kkt_destroy", None, [_P]),
    ("kkt_set_options", _I, [_P, ctypes.POINTER(KKTOptions)]),
    ("kkt_get_options", _I, [_P, ctypes.POINTER(KKTOptions)]),
    ("kkt_get_info", _I, [_P, ctypes.POINTER(KKTInfo)]),
    ("kkt_build_rhs", _I, [_P, _P, _P, _P, _P]),
    ("kkt_matvec", _I, [_P, _P, _P, _P]),
    ("kkt_precond_apply", _I, [_P, _P, _P, _P]),
    ("kkt_solve", _I, [_P, _P, _P, _D, _I, ctypes.POINTER(KKTStats), _P]),
    ("kkt_solve_zero_guess", _I, [_P, _P, _P, _D, _I, ctypes.POINTER(KKTStats), _P]),
    ("kkt_set_staging", _I, [_P, _I]),
    ("kkt_set_dst_method", _I, [_P, _I]),
    ("kkt_get_dst_method", _I, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("kkt_dst2d", _I, [_P, _P, _P, _P]),
    ("kkt_schur_apply", _I, [_P, _P, _P, _P]),
    ("kkt_schur_precond_apply", _I, [_P, _P, _P, _P]),
    ("kkt_coarse_apply", _I, [_P, _P, _P, _P]),
    ("kkt_multidot", _I, [_P, _P, ctypes.c_longlong, _I, _P, ctypes.c_longlong, _P, _P]),
    ("kkt_multidot_noalloc", _I, [_P, ctypes.c_longlong, _I, _P, ctypes.c_longlong, _P, _P]),
    ("kkt_mlp_default_config", _I, [ctypes.POINTER(KKTMlpConfig)]),
    ("kkt_mlp_create", _P, [ctypes.POINTER(KKTMlpConfig)]),
    ("kkt_mlp_destroy", None, [_P]),
    ("kkt_mlp_param_count", _I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    ("kkt_mlp_get_config", _I, [_P, ctypes.POINTER(KKTMlpConfig)]),
    ("kkt_mlp_set_params", _I, [_P, _P, ctypes.c_longlong]),
    ("kkt_mlp_get_params", _I, [_P, _P, ctypes.c_longlong]),
    ("kkt_mlp_forward", _I, [_P, _P, _P, _I, _I, _P]),
    ("kkt_mlp_loss_grad", _I, [_P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("kkt_mlp_resid_loss_grad", _I, [_P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("kkt_mlp_coarse_data", _I, [_P, _P, _P, ctypes.c_longlong, _P, _P, _P]),
    ("kkt_mlp_adam_step", _I, [_P, _P, _P, _I, _D, ctypes.POINTER(ctypes.c_double), _P]),
    ("kkt_mlp_train", _I, [_P, ctypes.POINTER(KKTMlpTrainStats), _P]),
    ("kkt_mlp_save", _I, [_P, ctypes.c_char_p]),
    ("kkt_mlp_load", _P, [ctypes.c_char_p]),
    ("kkt_attach_mlp", _I, [_P, _P, _I]),
    ("kkt_inject_tc_timeout", _I, [_P]),
    ("kkt_learned_stats", _I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _I]),
    ("kkt_batch_create", _P, [_I, ctypes.POINTER(KKTInstance), ctypes.POINTER(KKTOptions)]),
    ("kkt_batch_destroy", None, [_P]),
    ("kkt_batch_get_info", _I, [_P, _I, ctypes.POINTER(KKTInfo)]),
    ("kkt_batch_set_memory_limit", _I, [_P, ctypes.c_longlong]),
    ("kkt_batch_set_graphs", _I, [_P, _I]),
    ("kkt_batch_set_single_threshold", _I, [_P, ctypes.c_longlong]),
    ("kkt_batch_set_dst_method", _I, [_P, _I]),
    ("kkt_batch_solve", _I, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), _D, _I,
                             ctypes.POINTER(KKTBatchStats), _P]),
    ("kkt_profile_enable", _I, [_I]),
    ("kkt_profile_read", _I, [ctypes.POINTER(KKTKernelStats), _I]),
    ("kkt_probe_fma_rate", _I, [_I, ctypes.POINTER(ctypes.c_double), _P]),
]

_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libkkt.so (built by paper_2305_04421_gb300.build). Raises if it is absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int) -> int:
    if status < 0:
        lib = load_library()
        raise KKTError(status, lib.kkt_last_error().decode())
    return status


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("vectors must be contiguous float64 tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---- same-named wrappers of the C entry points ----------------------------------------------

def kkt_create(nx, ny, Nt, T, nu, omega, n_sub) -> int:
    lib = load_library()
    h = lib.kkt_create(nx, ny, Nt, T, nu, omega, n_sub)
    if not h:
        raise KKTError(KKT_ERR_INVALID_ARG, lib.kkt_last_error().decode())
    return h


def kkt_destroy(h) -> None:
    load_library().kkt_destroy(h)


def kkt_set_options(h, opt: KKTOptions) -> int:
    return _check(load_library().kkt_set_options(h, ctypes.byref(opt)))


def kkt_get_options(h) -> KKTOptions:
    opt = KKTOptions()
    _check(load_library().kkt_get_options(h, ctypes.byref(opt)))
    return opt


def kkt_get_info(h) -> KKTInfo:
    info = KKTInfo()
    _check(load_library().kkt_get_info(h, ctypes.byref(info)))
    return info


def kkt_build_rhs(h, u_target, u0, f, stream=None) -> int:
    return _check(load_library().kkt_build_rhs(h, _ptr(u_target), _ptr(u0), _ptr(f), _stream(stream)))


def kkt_matvec(h, x, y, stream=None) -> int:
    return _check(load_library().kkt_matvec(h, _ptr(x), _ptr(y), _stream(stream)))


def kkt_precond_apply(h, r, y, stream=None) -> int:
    return _check(load_library().kkt_precond_apply(h, _ptr(r), _ptr(y), _stream(stream)))


def kkt_solve(h, f, x, tol, maxit, stats: KKTStats | None = None, stream=None) -> int:
    st = stats if stats is not None else KKTStats()
    return _check(load_library().kkt_solve(h, _ptr(f), _ptr(x), tol, maxit, ctypes.byref(st), _stream(stream)))


def kkt_solve_zero_guess(h, f, x, tol, maxit, stats: KKTStats | None = None, stream=None) -> int:
    st = stats if stats is not None else KKTStats()
    return _check(load_library().kkt_solve_zero_guess(h, _ptr(f), _ptr(x), tol, maxit, ctypes.byref(st),
                                                      _stream(stream)))


def kkt_set_staging(h, mode: int) -> int:
    return _check(load_library().kkt_set_staging(h, mode))


def kkt_dst2d(h, x, y, stream=None) -> int:
    return _check(load_library().kkt_dst2d(h, _ptr(x), _ptr(y), _stream(stream)))


def kkt_schur_apply(h, x, y, stream=None) -> int:
    return _check(load_library().kkt_schur_apply(h, _ptr(x), _ptr(y), _stream(stream)))


def kkt_schur_precond_apply(h, r, y, stream=None) -> int:
    return _check(load_library().kkt_schur_precond_apply(h, _ptr(r), _ptr(y), _stream(stream)))


def kkt_coarse_apply(h, r, y, stream=None) -> int:
    return _check(load_library().kkt_coarse_apply(h, _ptr(r), _ptr(y), _stream(stream)))


def kkt_multidot(h, V, stride, count, w, n, out, stream=None) -> int:
    """out[k] = <V_k, w> (k < count), out[count] = <w, w>; V a contiguous float64 device tensor."""
    return _check(load_library().kkt_multidot(h, _ptr(V), stride, count, _ptr(w), n, _ptr(out), _stream(stream)))


def kkt_multidot_noalloc(V, stride, count, w, n, out, stream=None) -> int:
    """kkt_multidot without a handle or any device allocation (scratch in a static device array);
    for callers that cannot allocate device memory. Calls must not overlap on the GPU."""
    return _check(load_library().kkt_multidot_noalloc(_ptr(V), stride, count, _ptr(w), n, _ptr(out),
                                                      _stream(stream)))


def kkt_batch_create(instances, opt: KKTOptions | None = None) -> int:
    """instances: a sequence of KKTInstance (or (nx, ny, Nt, n_sub, T, nu, omega) tuples)."""
    lib = load_library()
    arr = (KKTInstance * len(instances))(*[i if isinstance(i, KKTInstance) else KKTInstance(*i) for i in instances])
    b = lib.kkt_batch_create(len(instances), arr, ctypes.byref(opt) if opt is not None else None)
    if not b:
        raise KKTError(KKT_ERR_INVALID_ARG, lib.kkt_last_error().decode())
    return b


def kkt_batch_destroy(b) -> None:
    load_library().kkt_batch_destroy(b)


def kkt_batch_get_info(b, i) -> KKTInfo:
    info = KKTInfo()
    _check(load_library().kkt_batch_get_info(b, i, ctypes.byref(info)))
    return info


def kkt_batch_set_memory_limit(b, nbytes: int) -> int:
    return _check(load_library().kkt_batch_set_memory_limit(b, int(nbytes)))


def kkt_batch_solve(b, fs, xs, tol, maxit, stats: KKTBatchStats | None = None, stream=None) -> int:
    n = len(fs)
    fp = (ctypes.c_void_p * n)(*[_ptr(t).value for t in fs])
    xp = (ctypes.c_void_p * n)(*[_ptr(t).value for t in xs])
    st = stats if stats is not None else KKTBatchStats()
    return _check(load_library().kkt_batch_solve(b, fp, xp, tol, maxit, ctypes.byref(st), _stream(stream)))


def kkt_profile_enable(on: bool) -> int:
    return _check(load_library().kkt_profile_enable(1 if on else 0))


def kkt_profile_read(reset: bool = False) -> dict:
    """Per kernel class: launches, timed launches and summed device milliseconds."""
    st = KKTKernelStats()
    _check(load_library().kkt_profile_read(ctypes.byref(st), 1 if reset else 0))
    return {name: {"launches": st.launches[i], "timed": st.timed[i], "ms": st.ms[i], "flops": st.flops[i],
                   "bytes": st.bytes[i]} for i, name in enumerate(KERNEL_CLASSES)}


def kkt_probe_fma_rate(precision: str, stream=None) -> float:
    """Measured FMA throughput of this GPU in FLOP/s ('fp64' or 'fp32'; 2 FLOPs per FMA)."""
    r = ctypes.c_double()
    _check(load_library().kkt_probe_fma_rate({"fp64": 0, "fp32": 1}[precision], ctypes.byref(r), _stream(stream)))
    return r.value


def _fptr(t):
    if t is None:
        return None
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("network tensors must be contiguous float32")
    return ctypes.c_void_p(t.data_ptr())


def kkt_mlp_default_config() -> KKTMlpConfig:
    c = KKTMlpConfig()
    _check(load_library().kkt_mlp_default_config(ctypes.byref(c)))
    return c


class Mlp:
    """The learned coarse correction's network (owns a kkt_mlp)."""

    def __init__(self, cfg: KKTMlpConfig | None = None, *, handle=None, **overrides):
        lib = load_library()
        if handle is not None:
            self.m = handle
        else:
            c = cfg if cfg is not None else kkt_mlp_default_config()
            for k, v in overrides.items():
                setattr(c, k, v)
            self.m = lib.kkt_mlp_create(ctypes.byref(c))
            if not self.m:
                raise KKTError(KKT_ERR_INVALID_ARG, lib.kkt_last_error().decode())
        self.cfg = KKTMlpConfig()
        _check(lib.kkt_mlp_get_config(self.m, ctypes.byref(self.cfg)))
        n = ctypes.c_longlong()
        _check(lib.kkt_mlp_param_count(self.m, ctypes.byref(n)))
        self.nparam = n.value

    @classmethod
    def load(cls, path: str) -> "Mlp":
        lib = load_library()
        m = lib.kkt_mlp_load(path.encode())
        if not m:
            raise KKTError(KKT_ERR_INVALID_ARG, lib.kkt_last_error().decode())
        return cls(handle=m)

    def save(self, path: str) -> None:
        _check(load_library().kkt_mlp_save(self.m, path.encode()))

    def get_params(self):
        import numpy as np
        out = np.empty(self.nparam, dtype=np.float32)
        _check(load_library().kkt_mlp_get_params(self.m, out.ctypes.data_as(ctypes.c_void_p), self.nparam))
        return out

    def set_params(self, arr) -> None:
        import numpy as np
        a = np.ascontiguousarray(arr, dtype=np.float32)
        _check(load_library().kkt_mlp_set_params(self.m, a.ctypes.data_as(ctypes.c_void_p), a.size))

    def forward(self, X, use_bf16=False, stream=None):
        B = X.shape[0]
        Y = torch.empty((B, self._d_out()), dtype=torch.float32, device=X.device)
        _check(load_library().kkt_mlp_forward(self.m, _fptr(X), _fptr(Y), B, 1 if use_bf16 else 0, _stream(stream)))
        return Y

    def loss_grad(self, X, T, stream=None):
        g = torch.empty(self.nparam, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        _check(load_library().kkt_mlp_loss_grad(self.m, _fptr(X), _fptr(T), X.shape[0], _fptr(g), ctypes.byref(loss),
                                                _stream(stream)))
        return loss.value, g

    def resid_loss_grad(self, X, mu, stream=None):
        """Coarse-residual loss of net(X) and its parameter gradient; mu: float64 [batch]."""
        g = torch.empty(self.nparam, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        _check(load_library().kkt_mlp_resid_loss_grad(self.m, _fptr(X), _ptr(mu), X.shape[0], _fptr(g),
                                                      ctypes.byref(loss), _stream(stream)))
        return loss.value, g

    def coarse_data(self, r, mu, stream=None):
        """Training pairs: r float64 [Nt][count] time series, mu float64 [count] ->
        (c = R_0 r, x = G(mu)^-1 c), each float64 [count][2 n_sub]."""
        count = mu.shape[0]
        c = torch.empty((count, self._d_out()), dtype=torch.float64, device=r.device)
        x = torch.empty_like(c)
        _check(load_library().kkt_mlp_coarse_data(self.m, _ptr(r), _ptr(mu), count, _ptr(c), _ptr(x),
                                                  _stream(stream)))
        return c, x

    def adam_step(self, X, T, lr, stream=None):
        loss = ctypes.c_double()
        _check(load_library().kkt_mlp_adam_step(self.m, _fptr(X), _fptr(T), X.shape[0], lr, ctypes.byref(loss),
                                                _stream(stream)))
        return loss.value

    def train(self, stream=None) -> KKTMlpTrainStats:
        st = KKTMlpTrainStats()
        _check(load_library().kkt_mlp_train(self.m, ctypes.byref(st), _stream(stream)))
        return st

    def _d_out(self):
        return 2 * self.cfg.n_sub

    def close(self):
        if getattr(self, "m", None):
            load_library().kkt_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience object ---------------------------------------------------------------------

@dataclass
class SolveResult:
    x: torch.Tensor
    status: int
    iterations: int
    restarts: int
    rel_residual: float
    rel_residual_euclid: float
    time_ms: float
    history: list


class Solver:
    """One KKT instance on the current CUDA device (owns a kkt_handle)."""

    def __init__(self, nx, ny, Nt, T=1.0, nu=1.0, omega=1e-4, n_sub=1, *, precision="fp64",
                 coarse="exact", variant="multiplicative", pou="left", restart=30, jhat_sign=-1,
                 residual_norm="l2", tc_split=True, orth="mgs2", basis="physical", local="rasq", Lx=1.0,
                 Ly=1.0, coarse_solve="auto"):
        self.h = kkt_create(nx, ny, Nt, T, nu, omega, n_sub)
        self.set_options(precision=precision, coarse=coarse, variant=variant, pou=pou, restart=restart,
                         jhat_sign=jhat_sign, residual_norm=residual_norm, tc_split=tc_split, orth=orth,
                         basis=basis, local=local, Lx=Lx, Ly=Ly, coarse_solve=coarse_solve)
        self.info = kkt_get_info(self.h)

    def set_options(self, *, precision="fp64", coarse="exact", variant="multiplicative", pou="left",
                    restart=30, jhat_sign=-1, residual_norm="l2", tc_split=True, orth="mgs2", basis="physical",
                    local="rasq", Lx=1.0, Ly=1.0, coarse_solve="auto"):
        opt = KKTOptions(PREC[precision], COARSE[coarse], VARIANT[variant], POU[pou], restart, jhat_sign,
                         NORM[residual_norm], 1 if tc_split else 0, ORTH[orth], BASIS[basis], LOCAL[local],
                         Lx, Ly, COARSE_SOLVE[coarse_solve])
        kkt_set_options(self.h, opt)
        self.info = kkt_get_info(self.h)

    def set_dst_method(self, method="auto"):
        """FP64 sine transforms: 'auto' (timed at create), 'tiles' (warp per line), 'lane'
        (thread per line; lines of at most 31 points) or 'tensor' (FP64-accurate digit-plane
        GEMMs on the tensor cores; square grids of at most 256 intervals)."""
        _check(load_library().kkt_set_dst_method(self.h, DST_METHOD[method]))

    def dst_method(self) -> str:
        """The FP64 transform method in use: 'tiles', 'lane' or 'tensor'."""
        m = ctypes.c_int()
        _check(load_library().kkt_get_dst_method(self.h, ctypes.byref(m)))
        return {v: k for k, v in DST_METHOD.items()}[m.value]

    def set_staging(self, mode="auto"):
        """How solve() moves host vectors: 'auto' (pinned buffers by a copy kernel, pageable by
        cudaMemcpyAsync) or 'copy_engine' (always cudaMemcpyAsync)."""
        kkt_set_staging(self.h, STAGING[mode])

    def close(self):
        if getattr(self, "h", None):
            kkt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def V(self) -> int:
        return int(self.info.V)

    def _out(self, like: torch.Tensor, n: int) -> torch.Tensor:
        return torch.empty(n, dtype=torch.float64, device=like.device)

    def build_rhs(self, u_target, u0=None, out=None, stream=None):
        f = out if out is not None else torch.empty(3 * self.V, dtype=torch.float64, device=u_target.device)
        kkt_build_rhs(self.h, u_target, u0, f, stream)
        return f

    def matvec(self, x, out=None, stream=None):
        y = out if out is not None else self._out(x, 3 * self.V)
        kkt_matvec(self.h, x, y, stream)
        return y

    def precond_apply(self, r, out=None, stream=None):
        y = out if out is not None else self._out(r, 3 * self.V)
        kkt_precond_apply(self.h, r, y, stream)
        return y

    def dst2d(self, x, out=None, stream=None):
        y = out if out is not None else self._out(x, self.V)
        kkt_dst2d(self.h, x, y, stream)
        return y

    def schur_apply(self, x, out=None, stream=None):
        y = out if out is not None else self._out(x, self.V)
        kkt_schur_apply(self.h, x, y, stream)
        return y

    def schur_precond_apply(self, r, out=None, stream=None):
        y = out if out is not None else self._out(r, self.V)
        kkt_schur_precond_apply(self.h, r, y, stream)
        return y

    def coarse_apply(self, r, out=None, stream=None):
        y = out if out is not None else self._out(r, self.V)
        kkt_coarse_apply(self.h, r, y, stream)
        return y

    def attach_mlp(self, mlp: "Mlp", mode: str = "learned"):
        """Use `mlp` for coarse='learned': mode 'learned' (the network's corrections, guarded,
        exact solve where the guard rejects), 'none' (no coarse correction on the learned modes,
        the ablation) or 'network' (the network's corrections always, no guard or fallback);
        then switch the options to coarse='learned'."""
        _check(load_library().kkt_attach_mlp(self.h, mlp.m, MLP_MODE[mode]))
        self._mlp = mlp

    def learned_stats(self, reset=False):
        kept, fb = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load_library().kkt_learned_stats(self.h, ctypes.byref(kept), ctypes.byref(fb), 1 if reset else 0))
        return kept.value, fb.value

    def solve(self, f, x=None, tol=1e-8, maxit=420, stream=None, zero_guess=False) -> SolveResult:
        """x: the initial guess, overwritten by the solution (zeros when None). zero_guess=True
        starts from 0 whatever x holds and never reads it (a host x is not uploaded)."""
        if x is None:
            x = torch.empty_like(f)
            zero_guess = True
        st = KKTStats()
        status = (kkt_solve_zero_guess if zero_guess else kkt_solve)(self.h, f, x, tol, maxit, st, stream)
        return SolveResult(x, status, st.iterations, st.restarts, st.rel_residual, st.rel_residual_euclid, st.time_ms,
                           list(st.history[: st.history_len]))


@dataclass
class BatchResult:
    xs: list
    status: int
    solo: int
    statuses: list
    iterations: list
    rel_residual: list
    waves: int
    graphs: int
    graph_launches: int
    tile_lines: int
    sweep_block: int
    tune_ms_dst: list
    tune_ms_sweep: list
    time_ms: float


class Batch:
    """Many independent KKT instances solved together (owns a kkt_batch). instances: objects
    with nx, ny, Nt, n_sub, T, nu, omega attributes (e.g. workloads.Workload) or tuples."""

    def __init__(self, instances, *, coarse="exact", variant="multiplicative", pou="left", restart=30,
                 jhat_sign=-1, residual_norm="l2", orth="mgs2", basis="physical", Lx=1.0, Ly=1.0,
                 coarse_solve="auto"):
        descs = []
        for w in instances:
            if isinstance(w, tuple):
                descs.append(KKTInstance(*w))
            else:
                descs.append(KKTInstance(w.nx, w.ny, w.Nt, w.n_sub, w.T, w.nu, w.omega))
        opt = KKTOptions(PREC["fp64"], COARSE[coarse], VARIANT[variant], POU[pou], restart, jhat_sign,
                         NORM[residual_norm], 1, ORTH[orth], BASIS[basis], LOCAL["rasq"], Lx, Ly,
                         COARSE_SOLVE[coarse_solve])
        self.b = kkt_batch_create(descs, opt)
        self.infos = [kkt_batch_get_info(self.b, i) for i in range(len(descs))]

    def __len__(self):
        return len(self.infos)

    def set_single_threshold(self, points: int) -> None:
        """Instances with at least `points` unknowns per block are solved one by one (0: none)."""
        _check(load_library().kkt_batch_set_single_threshold(self.b, int(points)))

    def set_dst_method(self, method="auto") -> None:
        """Every instance's FP64 transform method ('auto', 'tiles', 'lane' or 'tensor')."""
        _check(load_library().kkt_batch_set_dst_method(self.b, DST_METHOD[method]))

    def set_graphs(self, on: bool) -> None:
        """Replay the per-step preconditioner + matvec phase as CUDA graphs (default) or not."""
        _check(load_library().kkt_batch_set_graphs(self.b, 1 if on else 0))

    def set_memory_limit(self, nbytes: int) -> None:
        """Krylov storage per wave in bytes (0: 85% of free device memory)."""
        kkt_batch_set_memory_limit(self.b, nbytes)

    def close(self):
        if getattr(self, "b", None):
            kkt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, fs, xs=None, tol=1e-8, maxit=420, stream=None) -> BatchResult:
        if xs is None:
            xs = [torch.zeros_like(f) for f in fs]
        st = KKTBatchStats()
        status = kkt_batch_solve(self.b, fs, xs, tol, maxit, st, stream)
        n = len(fs)
        return BatchResult(xs, status, st.solo, list(st.status[:n]), list(st.iterations[:n]), list(st.rel_residual[:n]),
                           st.waves, st.graphs, st.graph_launches, st.tile_lines, st.sweep_block,
                           list(st.tune_ms_dst), list(st.tune_ms_sweep), st.time_ms)
