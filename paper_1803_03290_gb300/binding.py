"""ctypes binding of libgpcg (include/gpcg.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  The library must
be built for the GPU in use; there is no CPU fallback, and importing this
module without the compiled library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GPCG_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "BASE_NOT_CONVERGED", 4: "BASE_ISLANDED",
          5: "TIMEOUT", 6: "OOM", 7: "NOT_READY"}
PLAIN_FP64, BATCHED_FP32, BATCHED_FP64, BATCHED_FP32_F16 = 0, 1, 2, 3
PRECOND_IC0, PRECOND_JACOBI, PRECOND_EXACT = 0, 1, 2
SCEN_OK, SCEN_MAXITER, SCEN_DIVERGED, SCEN_ISLAND_NO_GEN, SCEN_QLIM_OVERFLOW = 0, 1, 2, 3, 4
MAX_TAIL_ROWS = 248  # GPCG_MAX_TAIL_ROWS: largest dense tail of a factor (rows)
MAX_EXT_ROWS = 8  # GPCG_MAX_EXT_ROWS: B'' rows a scenario can add (held buses, tripped one)


class GPCGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32),
                ("bus_type", C.c_void_p), ("P_sched", C.c_void_p), ("Q_sched", C.c_void_p),
                ("P_gen", C.c_void_p), ("V_set", C.c_void_p), ("from_", C.c_void_p),
                ("to", C.c_void_p), ("r", C.c_void_p), ("x", C.c_void_p),
                ("b_sh", C.c_void_p), ("rating", C.c_void_p), ("tap", C.c_void_p),
                ("Q_min", C.c_void_p), ("Q_max", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("base_tol", C.c_double), ("inner_rtol", C.c_double),
                ("max_outer", C.c_int32), ("max_inner", C.c_int32), ("precision", C.c_int32),
                ("precond", C.c_int32), ("tile", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("tail_rows", C.c_int32), ("wait_limit", C.c_int32)]


class Info(C.Structure):
    _fields_ = [(k, C.c_int32) for k in (
        "n_bus", "n_branch", "slack", "n_p", "n_q", "nnz_p", "nnz_q", "nnz_lp", "nnz_lq",
        "levels_p", "levels_q", "blevels_p", "blevels_q", "n_bridges", "tile", "num_sms",
        "base_outer", "ctas_per_sm", "tail_rows_p", "tail_rows_q", "tuned")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("gpcg_default_options", "gpcg_create", "gpcg_destroy", "gpcg_set_options",
           "gpcg_get_info", "gpcg_base_solve", "gpcg_n1_screen", "gpcg_apply",
           "gpcg_export_matrix", "gpcg_last_timings", "gpcg_n1_screen_noalloc",
           "gpcg_n1_adjoint", "gpcg_n1_dc_screen", "gpcg_n1_gen_screen", "gpcg_analyze",
           "gpcg_last_error")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgpcg.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libgpcg.so not found at {_build.LIB}: build it with "
                          "__graft_entry__.build()")
    lib = C.CDLL(_build.LIB)
    vp, i32, f64p = C.c_void_p, C.c_int32, C.c_void_p
    lib.gpcg_default_options.argtypes = [C.POINTER(Options)]
    lib.gpcg_create.argtypes = [C.POINTER(_Grid), C.POINTER(Options), C.POINTER(vp)]
    lib.gpcg_destroy.argtypes = [vp]
    lib.gpcg_destroy.restype = None
    lib.gpcg_set_options.argtypes = [vp, C.POINTER(Options)]
    lib.gpcg_get_info.argtypes = [vp, C.POINTER(Info)]
    lib.gpcg_base_solve.argtypes = [vp, f64p, f64p, f64p, vp]
    lib.gpcg_n1_screen.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_n1_gen_screen.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_apply.argtypes = [vp, i32, i32, vp, i32, i32, vp, vp]
    lib.gpcg_export_matrix.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_last_timings.argtypes = [vp, vp]
    lib.gpcg_n1_adjoint.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.gpcg_n1_dc_screen.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_analyze.argtypes = [C.POINTER(_Grid), i32, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_n1_screen_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gpcg_last_error.argtypes = []
    lib.gpcg_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("gpcg_destroy", "gpcg_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(lib, st):
    if st != GPCG_OK:
        raise GPCGError(st, lib.gpcg_last_error().decode())


def mask_words(n_branch: int) -> int:
    """32-bit words per scenario of the overload bit mask (GPCG_MASK_WORDS)."""
    return (int(n_branch) + 31) // 32


def unpack_mask(words, n_branch: int):
    """Bool array [..., n_branch] from overload mask words [..., mask_words]."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    bits = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :n_branch].astype(bool)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class PlanInfo(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("n_rows", "nnz_a", "nnz_l", "levels", "blevels",
                                          "n_bridges")]


def _grid_struct(grid):
    keep = dict(
        bus_type=np.ascontiguousarray(grid.bus_type, dtype=np.int8),
        P_sched=np.ascontiguousarray(grid.P_sched, dtype=np.float64),
        Q_sched=np.ascontiguousarray(grid.Q_sched, dtype=np.float64),
        P_gen=np.ascontiguousarray(grid.P_gen, dtype=np.float64),
        V_set=np.ascontiguousarray(grid.V_set, dtype=np.float64),
        from_=np.ascontiguousarray(grid.f, dtype=np.int32),
        to=np.ascontiguousarray(grid.t, dtype=np.int32),
        r=np.ascontiguousarray(grid.r, dtype=np.float64),
        x=np.ascontiguousarray(grid.x, dtype=np.float64),
        b_sh=np.ascontiguousarray(grid.b_sh, dtype=np.float64),
        rating=np.ascontiguousarray(grid.rating, dtype=np.float64))
    for k in ("tap", "Q_min", "Q_max"):
        v = getattr(grid, k, None)
        if v is not None:
            keep[k] = np.ascontiguousarray(v, dtype=np.float64)
    g = _Grid(n_bus=int(grid.n_bus), n_branch=int(grid.n_branch),
              **{k: v.ctypes.data for k, v in keep.items()})
    return g, keep


def analyze(grid, precond=PRECOND_EXACT, which=0):
    """Host-only structural plan (gpcg_analyze): numpy arrays."""
    lib = load()
    g, keep = _grid_struct(grid)
    info = PlanInfo()
    _check(lib, lib.gpcg_analyze(C.byref(g), precond, which, C.byref(info), None, None, None,
                                 None, None, None))
    d = dict(bus_order=np.empty(grid.n_bus, np.int32), bus_of_row=np.empty(info.n_rows, np.int32),
             lrowptr=np.empty(info.n_rows + 1, np.int32), lcol=np.empty(info.nnz_l, np.int32),
             level=np.empty(info.n_rows, np.int32), bridge=np.empty(grid.n_branch, np.uint8))
    _check(lib, lib.gpcg_analyze(C.byref(g), precond, which, C.byref(info),
                                 *[_ptr(d[k]) for k in ("bus_order", "bus_of_row", "lrowptr",
                                                         "lcol", "level", "bridge")]))
    d["info"] = {k: getattr(info, k) for k, _ in info._fields_}
    return d


def default_options(**kw) -> Options:
    lib = load()
    o = Options()
    _check(lib, lib.gpcg_default_options(C.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class GPCG:
    """One grid on the current CUDA device (gpcg_create ... gpcg_destroy)."""

    def __init__(self, grid, **options):
        lib = load()
        self._lib = lib
        self.n_bus = int(grid.n_bus)
        self.n_branch = int(grid.n_branch)
        g, keep = _grid_struct(grid)  # keep: the arrays g points into
        self.options = default_options(**options)
        h = C.c_void_p()
        _check(lib, lib.gpcg_create(C.byref(g), C.byref(self.options), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gpcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_options(self, **kw):
        for k, v in kw.items():
            if not hasattr(self.options, k):
                raise TypeError(f"unknown option {k}")
            setattr(self.options, k, v)
        _check(self._lib, self._lib.gpcg_set_options(self._h, C.byref(self.options)))

    def info(self) -> dict:
        i = Info()
        _check(self._lib, self._lib.gpcg_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def base_solve(self):
        th = np.empty(self.n_bus)
        vm = np.empty(self.n_bus)
        fl = np.empty(self.n_branch)
        it = np.empty(3, np.int32)
        _check(self._lib, self._lib.gpcg_base_solve(self._h, _ptr(th), _ptr(vm), _ptr(fl), _ptr(it)))
        return dict(theta=th, V=vm, flow=fl, iters=it)

    def n1_gen_screen(self, gen_buses, outputs=("theta", "V", "flow", "label", "iters",
                                                "status", "max_loading")):
        """gpcg_n1_gen_screen: generator outages of the given PV buses
        (host memory; outputs as n1_screen)."""
        return self.n1_screen(gen_buses, outputs, _fn="gpcg_n1_gen_screen")

    def n1_gen_screen_device(self, gen_buses, out: dict, stream=None):
        """Device-memory gpcg_n1_gen_screen (arguments as n1_screen_device)."""
        return self.n1_screen_device(gen_buses, out, stream, _fn="gpcg_n1_gen_screen")

    def n1_screen(self, outages, outputs=("theta", "V", "flow", "label", "iters", "status",
                                          "max_loading"), _fn="gpcg_n1_screen", out=None):
        """Host-memory screen: returns numpy arrays.  `out` (optional) maps
        output names to caller-allocated host arrays of the right shape and
        type -- numpy arrays or CPU torch tensors, pinned or not -- which are
        filled instead of new arrays; `outputs` is then ignored."""
        hold = out
        out = np.ascontiguousarray(outages, dtype=np.int32)
        S = out.shape[0]
        n, m = self.n_bus, self.n_branch
        if hold is not None:
            g = lambda k: _ptr(hold.get(k))
            _check(self._lib, getattr(self._lib, _fn)(
                self._h, _ptr(out), S, 0, None, g("theta"), g("V"), g("flow"), g("label"),
                g("iters"), g("status"), g("max_loading"), g("n_overload"), g("overload")))
            return hold
        res = {}
        spec = dict(theta=((S, n), np.float64), V=((S, n), np.float64),
                    flow=((S, m), np.float64), label=((S, n), np.int32),
                    iters=((S, 3), np.int32), status=((S,), np.int32),
                    max_loading=((S,), np.float64), n_overload=((S,), np.int32),
                    overload=((S, mask_words(m)), np.uint32))
        for k in outputs:
            shp, dt = spec[k]
            res[k] = np.empty(shp, dt)
        g = lambda k: _ptr(res.get(k))
        _check(self._lib, getattr(self._lib, _fn)(
            self._h, _ptr(out), S, 0, None, g("theta"), g("V"), g("flow"), g("label"),
            g("iters"), g("status"), g("max_loading"), g("n_overload"), g("overload")))
        return res

    def n1_screen_device(self, outages, out: dict, stream=None, _fn="gpcg_n1_screen"):
        """Device-memory screen: `outages` and every tensor in `out` are CUDA
        tensors (keys as in n1_screen); work is ordered on `stream`
        (a torch.cuda.Stream, default the current stream)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        g = lambda k: _ptr(out.get(k))
        _check(self._lib, getattr(self._lib, _fn)(
            self._h, _ptr(outages), int(outages.shape[0]), 1, C.c_void_p(s.cuda_stream),
            g("theta"), g("V"), g("flow"), g("label"), g("iters"), g("status"),
            g("max_loading"), g("n_overload"), g("overload")))

    def last_timings(self):
        """(islanding kernel ms, N-1 solve kernel ms) of the last screen."""
        ms = np.zeros(2, np.float32)
        _check(self._lib, self._lib.gpcg_last_timings(self._h, _ptr(ms)))
        return float(ms[0]), float(ms[1])

    def n1_screen_noalloc_device(self, outages, out: dict, stream=None):
        """gpcg_n1_screen_noalloc: like n1_screen_device, but the library
        takes all scratch from its fixed device array instead of allocating."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        g = lambda k: _ptr(out.get(k))
        _check(self._lib, self._lib.gpcg_n1_screen_noalloc(
            self._h, _ptr(outages), int(outages.shape[0]), C.c_void_p(s.cuda_stream),
            g("theta"), g("V"), g("flow"), g("label"), g("iters"), g("status"),
            g("max_loading"), g("n_overload"), g("overload")))

    def n1_dc_screen(self, outages, P=None,
                     outputs=("theta", "flow", "iters", "status", "max_loading")):
        """DC (P-theta) quick screen with host arrays (gpcg_n1_dc_screen)."""
        out = np.ascontiguousarray(outages, dtype=np.int32)
        S = out.shape[0]
        n, m = self.n_bus, self.n_branch
        Pa = None if P is None else np.ascontiguousarray(P, dtype=np.float64)
        spec = dict(theta=((S, n), np.float64), flow=((S, m), np.float64),
                    iters=((S,), np.int32), status=((S,), np.int32),
                    max_loading=((S,), np.float64), n_overload=((S,), np.int32),
                    overload=((S, mask_words(m)), np.uint32))
        res = {k: np.empty(*spec[k]) for k in outputs}
        g = lambda k: _ptr(res.get(k))
        _check(self._lib, self._lib.gpcg_n1_dc_screen(
            self._h, _ptr(out), S, 0, None, _ptr(Pa), g("theta"), g("flow"), g("iters"),
            g("status"), g("max_loading"), g("n_overload"), g("overload")))
        return res

    def n1_dc_screen_device(self, outages, out: dict, P=None, stream=None):
        """Device tensors in and out (see gpcg_n1_dc_screen)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        g = lambda k: _ptr(out.get(k))
        _check(self._lib, self._lib.gpcg_n1_dc_screen(
            self._h, _ptr(outages), int(outages.shape[0]), 1, C.c_void_p(s.cuda_stream),
            _ptr(P), g("theta"), g("flow"), g("iters"), g("status"), g("max_loading"),
            g("n_overload"), g("overload")))

    def n1_adjoint(self, outages, P=None, b=None, grads=True):
        """Host arrays: (loss, dL/dP, dL/db) of the N-1 overload penalty."""
        out = np.ascontiguousarray(outages, dtype=np.int32)
        Pa = None if P is None else np.ascontiguousarray(P, dtype=np.float64)
        ba = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        loss = np.zeros(1)
        gP = np.zeros(self.n_bus) if grads else None
        gb = np.zeros(self.n_branch) if grads else None
        _check(self._lib, self._lib.gpcg_n1_adjoint(
            self._h, _ptr(out), out.shape[0], 0, None, _ptr(Pa), _ptr(ba), _ptr(loss),
            _ptr(gP), _ptr(gb)))
        return float(loss[0]), gP, gb

    def n1_adjoint_device(self, outages, P, b, loss, gP, gb, stream=None):
        """Device tensors in and out (see gpcg_n1_adjoint)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(self._lib, self._lib.gpcg_n1_adjoint(
            self._h, _ptr(outages), int(outages.shape[0]), 1, C.c_void_p(s.cuda_stream),
            _ptr(P), _ptr(b), _ptr(loss), _ptr(gP), _ptr(gb)))

    def apply(self, which, op, outages, X, precision=BATCHED_FP64):
        out = np.ascontiguousarray(outages, dtype=np.int32)
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.empty_like(X)
        _check(self._lib, self._lib.gpcg_apply(self._h, which, op, _ptr(out), out.shape[0],
                                               precision, _ptr(X), _ptr(Y)))
        return Y

    def export_matrix(self, which):
        inf = self.info()
        n = inf["n_p"] if which == 0 else inf["n_q"]
        nnz = inf["nnz_p"] if which == 0 else inf["nnz_q"]
        nl = inf["nnz_lp"] if which == 0 else inf["nnz_lq"]
        d = dict(bus_of_row=np.empty(n, np.int32), rowptr=np.empty(n + 1, np.int32),
                 col=np.empty(nnz, np.int32), val=np.empty(nnz), lrowptr=np.empty(n + 1, np.int32),
                 lcol=np.empty(nl, np.int32), lval=np.empty(nl), level=np.empty(n, np.int32))
        _check(self._lib, self._lib.gpcg_export_matrix(
            self._h, which, *[_ptr(d[k]) for k in ("bus_of_row", "rowptr", "col", "val",
                                                    "lrowptr", "lcol", "lval", "level")]))
        return d
