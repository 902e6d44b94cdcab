"""ctypes binding of libheat (include/heat.h): the same entry points, argument marshalling only.

Pointers may be given as torch tensors (their data_ptr), numpy arrays (host memory),
plain integers (raw addresses) or None.  Streams are cudaStream_t handles as integers
(e.g. ``torch.cuda.current_stream().cuda_stream``) or None for the legacy stream.
The library must have been built (``paper_1311_4627_gb300.build.build_lib``); there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libheat.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "heat.h")

HEAT_OK, HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA, HEAT_ENUMERIC, HEAT_ETIMEOUT, HEAT_ESTATE = range(7)
HEAT_F64, HEAT_F32 = 0, 1
HEAT_BUILD_F64, HEAT_BUILD_F32 = 0, 1
HEAT_HEATING_INTEGRAL, HEAT_HEATING_POINT = 0, 1
HEAT_COOLING_CONTINUOUS, HEAT_COOLING_DISCRETE = 0, 1
HEAT_EMIS_NONE, HEAT_EMIS_F64, HEAT_EMIS_BF16X3, HEAT_EMIS_TF32X3, HEAT_EMIS_BF16, HEAT_EMIS_TF32 = -1, 0, 1, 2, 3, 4
EMIS_NAMES = {HEAT_EMIS_F64: "f64", HEAT_EMIS_BF16X3: "bf16x3", HEAT_EMIS_TF32X3: "tf32x3", HEAT_EMIS_BF16: "bf16",
              HEAT_EMIS_TF32: "tf32"}
HEAT_T_FIELD, HEAT_T_BUILD, HEAT_T_RECUR, HEAT_T_EMIS, HEAT_T_COUNT = range(5)
TIMING_NAMES = ("field", "build", "recur", "emis")

_STATUS = {0: "HEAT_OK", 1: "HEAT_EINVAL", 2: "HEAT_ENOMEM", 3: "HEAT_ECUDA", 4: "HEAT_ENUMERIC",
           5: "HEAT_ETIMEOUT", 6: "HEAT_ESTATE"}


class HeatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class heat_opts(ctypes.Structure):
    _fields_ = [("build", ctypes.c_int), ("emis", ctypes.c_int), ("j_dtype", ctypes.c_int),
                ("size_integrate", ctypes.c_int), ("cell_begin", ctypes.c_int), ("cell_count", ctypes.c_int),
                ("chunk_cells", ctypes.c_int), ("host_io", ctypes.c_int), ("timing", ctypes.c_int),
                ("ledger_out", ctypes.c_void_p), ("streams", ctypes.c_int), ("heating", ctypes.c_int),
                ("prune_eps", ctypes.c_double), ("fused_build", ctypes.c_int),
                ("recur_blocks_per_sm", ctypes.c_int), ("emis_n_tile", ctypes.c_int),
                ("cooling", ctypes.c_int), ("build_prefetch", ctypes.c_int)]


class heat_tuning(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int), ("chunk_cells", ctypes.c_int), ("row_weight", ctypes.c_int),
                ("recur_blocks_per_sm", ctypes.c_int), ("emis_n_tile", ctypes.c_int), ("fused_build", ctypes.c_int),
                ("build_prefetch", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p


def declared_symbols():
    """Names of the functions include/heat.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*[a-z_ ]+\*?\s*\*?(heat_[a-z0-9_]+)\s*\(", text, flags=re.M)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1311_4627_gb300.build.build_lib()")
        L = ctypes.CDLL(LIB_PATH)
        L.heat_default_opts.restype = None
        L.heat_default_opts.argtypes = [ctypes.POINTER(heat_opts)]
        L.heat_create_grid.restype = ctypes.c_int
        L.heat_create_grid.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _vp]
        L.heat_set_grains.restype = ctypes.c_int
        L.heat_set_grains.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp]
        L.heat_set_fields.restype = ctypes.c_int
        L.heat_set_fields.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp]
        L.heat_solve.restype = ctypes.c_int
        L.heat_solve.argtypes = [_vp, ctypes.POINTER(heat_opts), _vp, _vp, _vp]
        L.heat_sync.restype = ctypes.c_int
        L.heat_sync.argtypes = [_vp]
        L.heat_last_error.restype = ctypes.c_char_p
        L.heat_last_error.argtypes = [_vp]
        L.heat_get_cooling.restype = ctypes.c_int
        L.heat_get_cooling.argtypes = [_vp, _vp]
        L.heat_band_elements.restype = ctypes.c_int
        L.heat_band_elements.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
        L.heat_graph_create.restype = ctypes.c_int
        L.heat_graph_create.argtypes = [_vp, ctypes.POINTER(heat_opts), _vp, _vp, _vp, ctypes.POINTER(_vp)]
        L.heat_graph_launch.restype = ctypes.c_int
        L.heat_graph_launch.argtypes = [_vp, _vp]
        L.heat_graph_nodes.restype = ctypes.c_int
        L.heat_graph_nodes.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
        L.heat_graph_destroy.restype = None
        L.heat_graph_destroy.argtypes = [_vp]
        L.heat_autotune.restype = ctypes.c_int
        L.heat_autotune.argtypes = [_vp, ctypes.POINTER(heat_opts), _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
        L.heat_get_timing.restype = ctypes.c_int
        L.heat_get_timing.argtypes = [_vp, _vp, _vp, ctypes.c_int]
        L.heat_get_cooling_discrete.restype = ctypes.c_int
        L.heat_get_cooling_discrete.argtypes = [_vp, _vp]
        L.heat_get_tuning.restype = ctypes.c_int
        L.heat_get_tuning.argtypes = [_vp, ctypes.POINTER(heat_tuning)]
        L.heat_set_wait_limit.restype = ctypes.c_int
        L.heat_set_wait_limit.argtypes = [_vp, ctypes.c_longlong]
        L.heat_debye_enthalpy.restype = ctypes.c_double
        L.heat_debye_enthalpy.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.heat_measure_fma_peak.restype = ctypes.c_int
        L.heat_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.heat_solve_noalloc.restype = ctypes.c_int
        L.heat_solve_noalloc.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]
        for name, args in [
            ("heat_surrogate_init", [_vp, ctypes.c_int, _vp, ctypes.c_ulonglong]),
            ("heat_surrogate_samples", [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
            ("heat_surrogate_fit_norm", [_vp, _vp, _vp, ctypes.c_longlong, _vp]),
            ("heat_surrogate_train", [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_ulonglong, _vp, _vp]),
            ("heat_surrogate_predict", [_vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp]),
            ("heat_solve_surrogate", [_vp, ctypes.POINTER(heat_opts), ctypes.c_float, _vp,
                                      ctypes.POINTER(ctypes.c_int), _vp]),
            ("heat_surrogate_grads", [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double),
                                      _vp]),
            ("heat_surrogate_params", [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
            ("heat_surrogate_save", [_vp, ctypes.c_char_p]),
            ("heat_surrogate_load", [_vp, ctypes.c_char_p]),
        ]:
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        L.heat_destroy.restype = None
        L.heat_destroy.argtypes = [_vp]
        _lib = L
    return _lib


def _ptr(x):
    """Raw address of a torch tensor, numpy array, integer or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays passed to libheat must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libheat must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(ctx, st):
    if st != HEAT_OK:
        msg = heat_last_error(ctx) if ctx else ""
        raise HeatError(st, msg)


def heat_default_opts(**kw) -> heat_opts:
    """Defaults of the library; keyword overrides (ledger_out takes a pointer-like)."""
    o = heat_opts()
    lib().heat_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, _ptr(v) if k == "ledger_out" else (float(v) if k == "prune_eps" else int(v)))
    return o


def heat_create_grid(device: int, lam_cm) -> int:
    lam = np.ascontiguousarray(lam_cm, dtype=np.float64)
    h = _vp()
    st = lib().heat_create_grid(ctypes.byref(h), int(device), lam.size, lam.ctypes.data)
    if st != HEAT_OK:
        raise HeatError(st, "heat_create_grid failed")
    return h.value


def heat_set_grains(ctx, radius_cm, c_abs_cm2, bin_offset, T_bins_K, H_bins_erg, size_weight=None):
    r = np.ascontiguousarray(radius_cm, dtype=np.float64)
    c = np.ascontiguousarray(c_abs_cm2, dtype=np.float64)
    o = np.ascontiguousarray(bin_offset, dtype=np.int32)
    t = np.ascontiguousarray(T_bins_K, dtype=np.float64)
    e = np.ascontiguousarray(H_bins_erg, dtype=np.float64)
    w = None if size_weight is None else np.ascontiguousarray(size_weight, dtype=np.float64)
    st = lib().heat_set_grains(ctx, r.size, r.ctypes.data, c.ctypes.data, o.ctypes.data, t.ctypes.data,
                               e.ctypes.data, None if w is None else w.ctypes.data)
    _check(ctx, st)


def heat_get_cooling_discrete(ctx, bins) -> list:
    """The thermal-discrete downward rates, one nb x nb array (row l, column u) per grain;
    bins: the bins of each grain."""
    n = int(sum(int(b) * int(b) for b in bins))
    D = np.zeros(n)
    _check(ctx, lib().heat_get_cooling_discrete(ctx, D.ctypes.data))
    out, k = [], 0
    for b in bins:
        b = int(b)
        out.append(D[k:k + b * b].reshape(b, b))
        k += b * b
    return out


def heat_get_tuning(ctx) -> dict:
    t = heat_tuning()
    _check(ctx, lib().heat_get_tuning(ctx, ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in heat_tuning._fields_}


WAIT_POLLS_DEFAULT = 1 << 22


def heat_set_wait_limit(ctx, polls):
    _check(ctx, lib().heat_set_wait_limit(ctx, int(polls)))


def heat_measure_fma_peak(device: int = 0, fp64: bool = True) -> float:
    """Measured FMA throughput of the device in TFLOP/s (FP64 or FP32)."""
    v = ctypes.c_double(0.0)
    st = lib().heat_measure_fma_peak(int(device), int(bool(fp64)), ctypes.byref(v))
    if st != HEAT_OK:
        raise HeatError(st, "heat_measure_fma_peak failed")
    return v.value


def heat_debye_enthalpy(theta_D: float, n_atoms: float, T) -> np.ndarray:
    """H(T) in erg for each temperature in T (host; one call per value)."""
    L = lib()
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    return np.array([L.heat_debye_enthalpy(float(theta_D), float(n_atoms), float(t)) for t in T.ravel()]).reshape(T.shape)


def heat_set_fields(ctx, n_cells, u, dtype, on_device, stream=None):
    _check(ctx, lib().heat_set_fields(ctx, int(n_cells), _ptr(u), int(dtype), int(on_device), stream))


def heat_solve(ctx, opts: heat_opts, P_out=None, j_out=None, stream=None):
    _check(ctx, lib().heat_solve(ctx, ctypes.byref(opts), _ptr(P_out), _ptr(j_out), stream))


class Graph:
    """A heat_solve captured into a CUDA graph (heat_graph_create); launch() replays it."""

    def __init__(self, ctx, opts: heat_opts, P_out=None, j_out=None, stream=None):
        h = _vp()
        _check(ctx, lib().heat_graph_create(ctx, ctypes.byref(opts), _ptr(P_out), _ptr(j_out), stream,
                                            ctypes.byref(h)))
        self.ctx, self.handle = ctx, h

    def launch(self, stream=None):
        _check(self.ctx, lib().heat_graph_launch(self.handle, stream))

    def kernel_nodes(self) -> int:
        v = ctypes.c_longlong()
        _check(self.ctx, lib().heat_graph_nodes(self.handle, ctypes.byref(v)))
        return v.value

    def close(self):
        if self.handle:
            lib().heat_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def heat_autotune(ctx, opts: heat_opts, P_out=None, j_out=None, stream=None):
    """Time (streams, chunk_cells) candidates on the current fields, keep the fastest for
    later solves that leave both at 0; returns (streams, chunk_cells)."""
    s, c = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().heat_autotune(ctx, ctypes.byref(opts), _ptr(P_out), _ptr(j_out), stream, ctypes.byref(s),
                                    ctypes.byref(c)))
    return s.value, c.value


def heat_sync(ctx):
    _check(ctx, lib().heat_sync(ctx))


def heat_last_error(ctx) -> str:
    m = lib().heat_last_error(ctx)
    return m.decode() if m else ""


def heat_get_cooling(ctx, nbt: int) -> np.ndarray:
    out = np.zeros(int(nbt))
    _check(ctx, lib().heat_get_cooling(ctx, out.ctypes.data))
    return out


def heat_band_elements(ctx) -> int:
    v = ctypes.c_longlong()
    _check(ctx, lib().heat_band_elements(ctx, ctypes.byref(v)))
    return v.value


def heat_get_timing(ctx, reset=True):
    """{kernel class: (ms, launches)} recorded by solves with timing=1."""
    ms = np.zeros(HEAT_T_COUNT)
    n = np.zeros(HEAT_T_COUNT, dtype=np.int64)
    _check(ctx, lib().heat_get_timing(ctx, ms.ctypes.data, n.ctypes.data, int(reset)))
    return {TIMING_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(HEAT_T_COUNT)}


def heat_solve_noalloc(ctx, build, u_dev, n_cells, P_out, stream=None):
    _check(ctx, lib().heat_solve_noalloc(ctx, int(build), _ptr(u_dev), int(n_cells), _ptr(P_out), stream))


HEAT_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
SURROGATE_INPUTS = 128


def heat_surrogate_init(ctx, members, grain_flag=None, seed=0):
    gf = None if grain_flag is None else np.ascontiguousarray(grain_flag, dtype=np.float32)
    _check(ctx, lib().heat_surrogate_init(ctx, int(members), None if gf is None else gf.ctypes.data, int(seed)))


def heat_surrogate_samples(ctx, cell_begin, cell_count, j, X, Y=None, lnp=None, stream=None):
    _check(ctx, lib().heat_surrogate_samples(ctx, int(cell_begin), int(cell_count), _ptr(j), _ptr(X), _ptr(Y),
                                             _ptr(lnp), stream))


def heat_surrogate_fit_norm(ctx, X, Y, n, stream=None):
    _check(ctx, lib().heat_surrogate_fit_norm(ctx, _ptr(X), _ptr(Y), int(n), stream))


def heat_surrogate_train(ctx, X, Y, n, batch, epochs, lr, seed=0, stream=None):
    hist = np.zeros(int(epochs))
    _check(ctx, lib().heat_surrogate_train(ctx, _ptr(X), _ptr(Y), int(n), int(batch), int(epochs), float(lr),
                                           int(seed), hist.ctypes.data, stream))
    return hist


def heat_surrogate_predict(ctx, X, lnp, n, lnj, spread, stream=None):
    _check(ctx, lib().heat_surrogate_predict(ctx, _ptr(X), _ptr(lnp), int(n), _ptr(lnj), _ptr(spread), stream))


def heat_solve_surrogate(ctx, fallback_opts, tol, j_out, stream=None):
    nfb = ctypes.c_int(0)
    _check(ctx, lib().heat_solve_surrogate(ctx, ctypes.byref(fallback_opts), float(tol), _ptr(j_out),
                                           ctypes.byref(nfb), stream))
    return nfb.value


def heat_surrogate_grads(ctx, member, Xn, Tn, n, grad_out, stream=None):
    loss = ctypes.c_double(0.0)
    _check(ctx, lib().heat_surrogate_grads(ctx, int(member), _ptr(Xn), _ptr(Tn), int(n), _ptr(grad_out),
                                           ctypes.byref(loss), stream))
    return loss.value


def heat_surrogate_params(ctx, member, values=None):
    """Get (values None) or set the flat FP32 parameters of one member."""
    n = ctypes.c_longlong(0)
    _check(ctx, lib().heat_surrogate_params(ctx, int(member), None, 0, ctypes.byref(n)))
    if values is None:
        out = np.zeros(n.value, dtype=np.float32)
        _check(ctx, lib().heat_surrogate_params(ctx, int(member), out.ctypes.data, 0, ctypes.byref(n)))
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(ctx, lib().heat_surrogate_params(ctx, int(member), v.ctypes.data, 1, ctypes.byref(n)))
    return v


def heat_surrogate_save(ctx, path):
    _check(ctx, lib().heat_surrogate_save(ctx, str(path).encode()))


def heat_surrogate_load(ctx, path):
    _check(ctx, lib().heat_surrogate_load(ctx, str(path).encode()))


def heat_destroy(ctx):
    if ctx:
        lib().heat_destroy(ctx)
