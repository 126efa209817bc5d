"""Python binding of libhg, the GB300 FFT-Galerkin homogenization library.

Argument marshalling only: every step of the solve runs in the CUDA kernels
of libhg.so (built in-tree by `paper_1311_0089_gb300.build`).  There is no
CPU fallback: if the library cannot be loaded, every call raises.

Arrays may be numpy arrays (host) or torch tensors; CUDA tensors are passed
as device pointers (no copy through the host), and the context can run on a
torch stream.  Names follow include/hg.h.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhg.so")

HG_OK = 0
HG_PENDING = 1
HG_FP64 = 0
HG_MIXED = 1
HG_CG = 0
HG_MS = 1
HG_PRIMAL = 0
HG_DUAL = 1
HG_COEFF_FULL = 0
HG_COEFF_PACKED = 1
STATUS = {
    0: "HG_OK", 1: "HG_PENDING", -1: "HG_ERR_ARG", -2: "HG_ERR_UNSUPPORTED_SIZE",
    -3: "HG_ERR_NOT_SPD", -4: "HG_ERR_NO_MEMORY", -5: "HG_ERR_NOT_CONVERGED",
    -6: "HG_ERR_DEVICE_TIMEOUT", -7: "HG_ERR_BUSY", -8: "HG_ERR_CUDA",
    -9: "HG_ERR_CANCELLED", -10: "HG_ERR_BREAKDOWN", -11: "HG_ERR_NO_COEFFS",
    -12: "HG_ERR_TOO_LARGE",
}
globals().update({name: code for code, name in STATUS.items()})


class HGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.hg_strerror(status).decode() if _lib is not None else ""
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int),
                ("lambda_ref", ctypes.c_double), ("loads_mask", ctypes.c_uint),
                ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("time_pass", ctypes.c_int),
                ("method", ctypes.c_int), ("formulation", ctypes.c_int),
                ("A0", ctypes.c_double * 9), ("batch_tiles", ctypes.c_int), ("resident", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("d", ctypes.c_int), ("AH", ctypes.c_double * 9),
                ("AH_flux", ctypes.c_double * 9), ("iters", ctypes.c_int * 3),
                ("outer", ctypes.c_int * 3), ("rel_res", ctypes.c_double * 3),
                ("device_ms", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("launches", ctypes.c_longlong), ("pass_ms_total", ctypes.c_double),
                ("pass_launches", ctypes.c_int), ("lambda_ref", ctypes.c_double),
                ("c_A", ctypes.c_double), ("C_A", ctypes.c_double), ("CH", ctypes.c_double * 9),
                ("true_rel_res", ctypes.c_double * 3), ("resident_ctas", ctypes.c_int)]

    def to_dict(self) -> dict:
        d = self.d
        return {
            "status": self.status,
            "AH": np.array(self.AH[: d * d]).reshape(d, d),
            "AH_flux": np.array(self.AH_flux[: d * d]).reshape(d, d),
            "iters": list(self.iters[:d]),
            "outer": list(self.outer[:d]),
            "rel_res": list(self.rel_res[:d]),
            "device_ms": self.device_ms,
            "wall_ms": self.wall_ms,
            "launches": self.launches,
            "pass_ms_total": self.pass_ms_total,
            "pass_launches": self.pass_launches,
            "lambda_ref": self.lambda_ref,
            "c_A": self.c_A,
            "C_A": self.C_A,
            "CH": np.array(self.CH[: d * d]).reshape(d, d),
            "true_rel_res": list(self.true_rel_res[:d]),
            "resident_ctas": self.resident_ctas,
        }


class LaunchCfg(ctypes.Structure):
    _fields_ = [("row_rb", ctypes.c_int), ("row_lb", ctypes.c_int), ("lanes", ctypes.c_int * 2),
                ("radix", (ctypes.c_int * 8) * 3)]

    def to_dict(self) -> dict:
        return {"row_rb": self.row_rb, "row_lb": self.row_lb, "lanes": list(self.lanes),
                "radix": [[r for r in self.radix[a] if r] for a in range(3)]}


class TuneResult(ctypes.Structure):
    _fields_ = [("chosen", LaunchCfg), ("heuristic", LaunchCfg), ("ms_chosen", ctypes.c_double),
                ("ms_heuristic", ctypes.c_double), ("candidates", ctypes.c_int), ("from_cache", ctypes.c_int)]

    def to_dict(self) -> dict:
        return {"chosen": self.chosen.to_dict(), "heuristic": self.heuristic.to_dict(),
                "ms_chosen": self.ms_chosen, "ms_heuristic": self.ms_heuristic,
                "candidates": self.candidates, "from_cache": bool(self.from_cache)}


_lib = None

# (name, restype, argtypes) of every entry point declared in include/hg.h
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = [
    ("hg_default_opts", None, [ctypes.POINTER(SolveOpts)]),
    ("hg_create", _I, [ctypes.POINTER(_VP), _I, ctypes.c_size_t, _VP]),
    ("hg_destroy", _I, [_VP]),
    ("hg_create_grid", _I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_VP)]),
    ("hg_destroy_grid", _I, [_VP]),
    ("hg_set_coeffs", _I, [_VP, _VP, _I, _I]),
    ("hg_set_coeffs_phase", _I, [_VP, _VP, _I, _VP, _I]),
    ("hg_set_coeffs_exact", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), _VP, _I, _VP]),
    ("hg_solve_AH", _I, [_VP, ctypes.POINTER(SolveOpts), _VP, ctypes.POINTER(Result)]),
    ("hg_test_resident_timeout", _I, [_VP, ctypes.POINTER(SolveOpts), _I, ctypes.POINTER(Result)]),
    ("hg_get_field", _I, [_VP, _I, _VP, _I]),
    ("hg_submit", _I, [_VP, _VP, ctypes.POINTER(SolveOpts), ctypes.POINTER(ctypes.c_uint64)]),
    ("hg_poll", _I, [_VP, ctypes.c_uint64, ctypes.POINTER(Result), _I]),
    ("hg_cancel", _I, [_VP, ctypes.c_uint64]),
    ("hg_apply", _I, [_VP, _VP, _VP, _I, _VP, _I, _I]),
    ("hg_spectrum", _I, [_VP, _VP, _VP, _I, _I]),
    ("hg_apply_noalloc", _I, [_I, ctypes.POINTER(_I), _VP, _I, _VP, _VP, _VP, _VP]),
    ("hg_launch_count", ctypes.c_longlong, [_VP]),
    ("hg_time_pass", _I, [_VP, _I, _I, _I, ctypes.POINTER(_D), ctypes.c_char_p]),
    ("hg_num_passes", _I, [_VP]),
    ("hg_num_iter_passes", _I, [_VP, ctypes.POINTER(SolveOpts)]),
    ("hg_solve_batch", _I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(SolveOpts), ctypes.POINTER(Result)]),
    ("hg_get_launch_cfg", _I, [_VP, _I, ctypes.POINTER(LaunchCfg)]),
    ("hg_set_launch_cfg", _I, [_VP, _I, ctypes.POINTER(LaunchCfg)]),
    ("hg_tune", _I, [_VP, _I, _I, ctypes.c_char_p, ctypes.POINTER(TuneResult)]),
    ("hg_tune_cache_find", _I, [ctypes.c_char_p, ctypes.c_char_p, _I, _I, _I, ctypes.POINTER(_I),
                                ctypes.POINTER(LaunchCfg), ctypes.POINTER(_D)]),
    ("hg_strerror", ctypes.c_char_p, [_I]),
]


def load(path: Optional[str] = None):
    """Load libhg.so (raises if it is missing or does not export the ABI)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libhg.so not built at {path}: run __graft_entry__.build() "
                           f"or python -m paper_1311_0089_gb300.build")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != HG_OK:
        raise HGError(st, where)


def tune_cache_find(path: str, device_name: str, sm_count: int, prec: int, N: Sequence[int]):
    """hg_tune_cache_find: (launch geometry dict, recorded ms) or None."""
    d = len(N)
    Narr = (_I * 3)(*(list(N) + [0] * (3 - d)))
    c = LaunchCfg()
    ms = ctypes.c_double()
    st = load().hg_tune_cache_find(path.encode(), device_name.encode(), sm_count, prec, d, Narr,
                                   ctypes.byref(c), ctypes.byref(ms))
    return (c.to_dict(), ms.value) if st == HG_OK else None


def default_opts(**kw) -> SolveOpts:
    lib = load()
    o = SolveOpts()
    lib.hg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        if k == "A0":   # d x d reference medium, row-major
            flat = [float(x) for x in np.asarray(v, dtype=np.float64).ravel()]
            v = (ctypes.c_double * 9)(*(flat + [0.0] * (9 - len(flat))))
        setattr(o, k, v)
    return o


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
            if a.dtype != want or not a.is_contiguous():
                a = a.to(want).contiguous()
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


class Context:
    """hg_ctx: one device and one stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream=None, use_torch_stream=True):
        lib = load()
        h = ctypes.c_void_p()
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        elif use_torch_stream:
            try:
                import torch
                if torch.cuda.is_available():
                    sptr = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
            except ImportError:  # pragma: no cover
                pass
        _check(lib.hg_create(ctypes.byref(h), device, mem_budget, sptr), "hg_create")
        self.h = h
        self.device = device
        self._grids = weakref.WeakSet()

    def close(self):
        """Destroys the context; grids still open on it are closed first."""
        if self.h:
            for g in list(self._grids):
                g.close()
            load().hg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launches(self) -> int:
        return int(load().hg_launch_count(self.h))

    def grid(self, N: Sequence[int], Y: Optional[Sequence[float]] = None) -> "Grid":
        return Grid(self, N, Y)

    def submit(self, grid: "Grid", opts: Optional[SolveOpts] = None) -> int:
        t = ctypes.c_uint64()
        o = opts if opts is not None else default_opts()
        _check(load().hg_submit(self.h, grid.h, ctypes.byref(o), ctypes.byref(t)), "hg_submit")
        return t.value

    def solve_batch(self, grids: Sequence["Grid"], opts: Optional[SolveOpts] = None,
                    raise_on_error: bool = True) -> list:
        """hg_solve_batch: grids solved together (one launch per pass for each
        shape, one CUDA graph for all shapes); one result dict each."""
        n = len(grids)
        hs = (_VP * n)(*[g.h for g in grids])
        res = (Result * n)()
        o = opts if opts is not None else default_opts()
        st = load().hg_solve_batch(hs, n, ctypes.byref(o), res)
        if st != HG_OK and raise_on_error:
            raise HGError(st, "hg_solve_batch")
        return [r.to_dict() for r in res]

    def poll(self, ticket: int, timeout_us: int = 0):
        """Returns None while pending, else the result dict (raises on error)."""
        r = Result()
        st = load().hg_poll(self.h, ticket, ctypes.byref(r), timeout_us)
        if st == HG_PENDING:
            return None
        out = r.to_dict()
        out["status"] = st
        return out

    def cancel(self, ticket: int):
        _check(load().hg_cancel(self.h, ticket), "hg_cancel")


class Grid:
    """hg_grid: an odd periodic grid N on the cell prod [-Y_a, Y_a]."""

    def __init__(self, ctx: Context, N: Sequence[int], Y: Optional[Sequence[float]] = None):
        lib = load()
        self.ctx = ctx
        self.N = tuple(int(n) for n in N)
        self.d = len(self.N)
        Narr = (ctypes.c_int * self.d)(*self.N)
        Yarr = (ctypes.c_double * self.d)(*Y) if Y is not None else None
        h = ctypes.c_void_p()
        _check(lib.hg_create_grid(ctx.h, self.d, Narr, Yarr, ctypes.byref(h)), "hg_create_grid")
        self.h = h
        self.M = int(np.prod(self.N))
        ctx._grids.add(self)

    def close(self):
        if self.h and self.ctx.h:
            load().hg_destroy_grid(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_coeffs_phase(self, phase, table):
        p, dev_p, k1 = _ptr(phase, np.uint8)
        t, dev_t, k2 = _ptr(table, np.float64)
        n_ph = int(np.asarray(table.shape[0] if hasattr(table, "shape") else len(table)))
        if dev_p != dev_t:
            raise ValueError("phase map and table must both be on the host or both on the device")
        _check(load().hg_set_coeffs_phase(self.h, p, n_ph, t, dev_p), "hg_set_coeffs_phase")

    def set_coeffs_exact(self, N_trial, phase, table):
        """Ga coefficients: pixels of the grid phase.shape with the given table,
        trial space N_trial; this grid is the quadrature grid (>= 2 N_trial - 1)."""
        ph = np.ascontiguousarray(np.asarray(phase, np.uint8))
        tb = np.ascontiguousarray(np.asarray(table, np.float64))
        if ph.ndim != self.d or len(N_trial) != self.d:
            raise ValueError("phase map and trial grid must have the grid's dimension")
        nt = (_I * 3)(*[int(v) for v in N_trial])
        P = (_I * 3)(*ph.shape)
        _check(load().hg_set_coeffs_exact(self.h, nt, P, ph.ctypes.data, int(tb.shape[0]), tb.ctypes.data),
               "hg_set_coeffs_exact")

    def set_coeffs(self, A, layout: int = HG_COEFF_FULL):
        """A: full (|N|, d, d) voxel-major, or packed (d(d+1)/2, |N|)."""
        p, dev, k = _ptr(A, np.float64)
        _check(load().hg_set_coeffs(self.h, p, layout, dev), "hg_set_coeffs")

    def set_coeffs_field(self, A_field: np.ndarray):
        """A as a (d, d, *N) array (the oracle's layout), passed as FULL voxel-major."""
        A = np.ascontiguousarray(np.moveaxis(np.asarray(A_field, np.float64).reshape(self.d, self.d, -1), 2, 0))
        self.set_coeffs(A, HG_COEFF_FULL)

    def solve(self, opts: Optional[SolveOpts] = None, raise_on_error: bool = True) -> dict:
        r = Result()
        o = opts if opts is not None else default_opts()
        st = load().hg_solve_AH(self.h, ctypes.byref(o), None, ctypes.byref(r))
        if st != HG_OK and raise_on_error:
            raise HGError(st, "hg_solve_AH")
        out = r.to_dict()
        out["status"] = st
        return out

    def test_resident_timeout(self, drop_cta: int, opts: Optional[SolveOpts] = None) -> int:
        """hg_test_resident_timeout: a mixed solve in which CTA drop_cta of the
        resident launch leaves at once; returns the status code."""
        r = Result()
        o = opts if opts is not None else default_opts(prec=HG_MIXED)
        return int(load().hg_test_resident_timeout(self.h, ctypes.byref(o), drop_cta, ctypes.byref(r)))

    def field(self, load_idx: int, out=None) -> np.ndarray:
        """e~ of load `load_idx` from the last solve, shape (d, *N)."""
        if out is None:
            out = np.empty((self.d,) + self.N)
        p, dev, k = _ptr(out, np.float64)
        _check(load().hg_get_field(self.h, load_idx, p, dev), "hg_get_field")
        return out

    def apply(self, u, with_A: bool = True, A0=None, prec: int = HG_FP64, out=None):
        """G_N A_N u (with_A) or G_N u; u of shape (d, *N)."""
        if out is None:
            out = np.empty((self.d,) + self.N)
        pu, dev_u, k1 = _ptr(u, np.float64)
        po, dev_o, k2 = _ptr(out, np.float64)
        if dev_u != dev_o:
            raise ValueError("u and out must both be host or both device arrays")
        a0 = None
        if A0 is not None:
            a0arr = np.ascontiguousarray(A0, dtype=np.float64)
            a0 = a0arr.ctypes.data_as(ctypes.c_void_p)
        _check(load().hg_apply(self.h, pu, po, int(with_A), a0, prec, dev_u), "hg_apply")
        return out

    def spectrum(self, u, prec: int = HG_FP64) -> np.ndarray:
        """Forward DFT (1/|N|) of a real (d, *N) field: half spectrum (d, *N[:-1], (N_d+1)/2)."""
        H = (self.N[-1] + 1) // 2
        out = np.empty((self.d,) + self.N[:-1] + (H, 2))
        pu, dev_u, k1 = _ptr(u, np.float64)
        if dev_u:
            raise ValueError("spectrum() takes a host array")
        _check(load().hg_spectrum(self.h, pu, out.ctypes.data_as(ctypes.c_void_p), prec, 0), "hg_spectrum")
        return out[..., 0] + 1j * out[..., 1]

    def launch_cfg(self, prec: int = HG_FP64) -> dict:
        """hg_get_launch_cfg: the passes' tiling for precision prec."""
        c = LaunchCfg()
        _check(load().hg_get_launch_cfg(self.h, prec, ctypes.byref(c)), "hg_get_launch_cfg")
        return c.to_dict()

    def set_launch_cfg(self, prec: int, row_rb: int, row_lb: int, lanes: Sequence[int], radix=None):
        """hg_set_launch_cfg (raises HGError HG_ERR_ARG for a geometry the kernels
        cannot run).  radix: per axis the radix order ([] = the default order);
        None keeps the grid's current orders."""
        if radix is None:
            radix = self.launch_cfg(prec)["radix"]
        ln = list(lanes) + [0] * (2 - len(lanes))
        c = LaunchCfg()
        c.row_rb, c.row_lb = row_rb, row_lb
        c.lanes[0], c.lanes[1] = ln[0], ln[1]
        for a, order in enumerate(list(radix)[:3]):
            for k, r in enumerate(order):
                c.radix[a][k] = int(r)
        _check(load().hg_set_launch_cfg(self.h, prec, ctypes.byref(c)), "hg_set_launch_cfg")

    def tune(self, prec: int = HG_MIXED, reps: int = 10, cache_path: Optional[str] = None) -> dict:
        """hg_tune: time every admissible geometry and keep the fastest."""
        r = TuneResult()
        _check(load().hg_tune(self.h, prec, reps, cache_path.encode() if cache_path else None, ctypes.byref(r)),
               "hg_tune")
        return r.to_dict()

    def num_passes(self) -> int:
        return int(load().hg_num_passes(self.h))

    def num_iter_passes(self, opts: Optional["SolveOpts"] = None) -> int:
        o = opts if opts is not None else default_opts()
        n = int(load().hg_num_iter_passes(self.h, ctypes.byref(o)))
        if n < 0:
            raise HGError(n, "hg_num_iter_passes")
        return n

    def time_pass(self, pass_idx: int, prec: int = HG_FP64, reps: int = 20):
        ms = ctypes.c_double()
        name = ctypes.create_string_buffer(64)
        _check(load().hg_time_pass(self.h, prec, pass_idx, reps, ctypes.byref(ms), name), "hg_time_pass")
        return ms.value, name.value.decode()
