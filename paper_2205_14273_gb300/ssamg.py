"""Python binding of the SSAMG C ABI (include/ssamg.h).

Argument marshalling only: every step of setup and solve runs in the CUDA
library libssamg.so.  Device vectors are torch CUDA tensors (float64,
contiguous); streams are torch.cuda.Stream objects or raw cudaStream_t
integers.  If the library is missing this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import json
import os
import re
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssamg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ssamg.h")

OK = 0
NOT_CONVERGED = 1
ERR_ARG = -1
ERR_STATE = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_BREAKDOWN = -5
ERR_TIMEOUT = -6
ERR_UNSUPPORTED = -7

TILE_CLASSES = 32   # entries of a tile table (level size classes floor(log2 n))
TILE_BRICKS = 8     # tile table bit: bricks allowed on the level


class SsamgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code}) {last_error()}")


class Params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("relax", ctypes.c_int),
                ("relax_factor", ctypes.c_double), ("skip", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("s_max", ctypes.c_longlong),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("coarse_direct", ctypes.c_int), ("flexible", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("use_tail", ctypes.c_int),
                ("use_pdl", ctypes.c_int), ("tail_cells", ctypes.c_int),
                ("use_bricks", ctypes.c_int), ("rhs_together", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("num_levels", ctypes.c_int), ("coarse_size", ctypes.c_longlong),
                ("operator_complexity", ctypes.c_double),
                ("setup_kernel_launches", ctypes.c_longlong),
                ("solve_kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong
_d = ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "ssamg_status_string": (ctypes.c_char_p, [_i]),
    "ssamg_last_error": (ctypes.c_char_p, []),
    "ssamg_release_device_cache": (ctypes.c_longlong, []),
    "ssamg_grid_create": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "ssamg_grid_set_box": (_i, [_vp, _i, _ip, _ip]),
    "ssamg_grid_add_box": (_i, [_vp, _i, _ip, _ip]),
    "ssamg_grid_assemble": (_i, [_vp]),
    "ssamg_grid_num_cells": (_ll, [_vp]),
    "ssamg_grid_destroy": (None, [_vp]),
    "ssamg_matrix_create": (_i, [_vp, _i, _ip, ctypes.POINTER(_vp)]),
    "ssamg_matrix_set_constant": (_i, [_vp, _i, _i, _d]),
    "ssamg_matrix_set_box_values": (_i, [_vp, _i, _i, _vp, _i]),
    "ssamg_matrix_add_couplings": (_i, [_vp, _ll, _ip, _ip, _ip, _ip, _ip, _dp]),
    "ssamg_matrix_assemble": (_i, [_vp, _vp]),
    "ssamg_matrix_destroy": (None, [_vp]),
    "ssamg_params_default": (None, [ctypes.POINTER(Params)]),
    "ssamg_solver_create": (_i, [ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "ssamg_solver_destroy": (None, [_vp]),
    "ssamg_setup": (_i, [_vp, _vp, _vp]),
    "ssamg_solve": (_i, [_vp, _vp, _vp, _i, _i, _vp, ctypes.POINTER(Stats)]),
    "ssamg_solve_host": (_i, [_vp, _dp, _dp, _i, _vp, ctypes.POINTER(Stats)]),
    "ssamg_adjoint_solve": (_i, [_vp, _vp, _vp, _i, _vp, ctypes.POINTER(Stats)]),
    "ssamg_coef_gradient": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "ssamg_diffusion_exp_gradient": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "ssamg_precondition": (_i, [_vp, _vp, _vp, _vp]),
    "ssamg_level_matvec": (_i, [_vp, _i, _vp, _vp, _vp]),
    "ssamg_num_levels": (_i, [_vp]),
    "ssamg_num_parts": (_i, [_vp]),
    "ssamg_tail_levels": (_i, [_vp, _ip, _ip, ctypes.POINTER(_ll)]),
    "ssamg_level_part_info": (_i, [_vp, _i, _i, _ip, _ip, _ip, _dp, _ip, _ip,
                                   ctypes.POINTER(_ll)]),
    "ssamg_level_sizes": (_i, [_vp, _i, ctypes.POINTER(_ll), ctypes.POINTER(_ll),
                               ctypes.POINTER(_ll)]),
    "ssamg_level_copy": (_i, [_vp, _i, _i, _i, _i, _vp, _ll]),
    "ssamg_spacings": (_i, [_vp, _dp, _dp]),
    "ssamg_coupling_sums_noalloc": (_i, [_vp, _i, _vp, _vp]),
    "ssamg_batch_create": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(Params), _vp,
                                ctypes.POINTER(_vp)]),
    "ssamg_batch_setup": (_i, [_vp, _vp]),
    "ssamg_batch_num_cells": (_ll, [_vp]),
    "ssamg_batch_offsets": (_i, [_vp, ctypes.POINTER(_ll)]),
    "ssamg_batch_solve": (_i, [_vp, _vp, _vp, _i, _vp, ctypes.POINTER(Stats)]),
    "ssamg_batch_destroy": (None, [_vp]),
    "ssamg_batch_solver": (_vp, [_vp]),
    "ssamg_level_stored_coefficients": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "ssamg_selftest_fastdiv": (_i, [ctypes.c_ulonglong, _i]),
    "ssamg_set_spacings": (_i, [_vp, _i, _dp]),
    "ssamg_residual_history": (_i, [_vp, _i, _dp, _i]),
    "ssamg_selftest_barrier": (_i, [_i, _i, ctypes.c_uint, _vp]),
    "ssamg_time_kernel": (_i, [_vp, _i, _i, _i, _dp, _vp]),
    "ssamg_set_tile_table": (_i, [_vp, _ip]),
    "ssamg_get_tile_table": (_i, [_vp, _ip]),
    "ssamg_level_tile": (_i, [_vp, _i, _ip, _ip]),
    "ssamg_autotune": (_i, [_vp, _i, _vp, _ip]),
}


def header_functions() -> list:
    """Names of the functions include/ssamg.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ssamg_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().ssamg_status_string(code).decode()


def last_error() -> str:
    return lib().ssamg_last_error().decode()


def _check(code, what, allow=(OK,)):
    if code not in allow:
        raise SsamgError(code, what)
    return code


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _dptr(t, n: Optional[int] = None, what: str = "vector") -> int:
    """Device pointer of a contiguous float64 CUDA tensor holding at least n
    elements (the library reads or writes n doubles there)."""
    if not (getattr(t, "is_cuda", False) and t.is_contiguous()):
        raise ValueError(f"{what}: expected a contiguous CUDA tensor")
    if str(t.dtype) != "torch.float64":
        raise ValueError(f"{what}: expected float64, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call uses {n}")
    return t.data_ptr()


class _IntBuf:
    """A contiguous int32 array kept alive while its pointer is in use."""

    def __init__(self, a):
        self.a = np.ascontiguousarray(a, dtype=np.int32).ravel()
        if self.a.size == 0:
            self.a = np.zeros(1, np.int32)
        self._as_parameter_ = self.a.ctypes.data_as(_ip)


def _ints(a) -> _IntBuf:
    return _IntBuf(a)


def default_params(**kw) -> Params:
    p = Params()
    lib().ssamg_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Grid:
    """Section 2: parts of cell-centred indices, each one box, or a group of
    boxes (part_boxes[p], held over their bounding box)."""

    def __init__(self, ndim: int, boxes: Sequence, part_boxes=None):
        self.h = _vp()
        _check(lib().ssamg_grid_create(ndim, len(boxes), ctypes.byref(self.h)), "grid_create")
        for p, (lo, hi) in enumerate(boxes):
            group = part_boxes[p] if part_boxes is not None else None
            if group:
                (blo, bhi), rest = group[0], group[1:]
                _check(lib().ssamg_grid_set_box(self.h, p, _ints(blo), _ints(bhi)), "grid_set_box")
                for blo, bhi in rest:
                    _check(lib().ssamg_grid_add_box(self.h, p, _ints(blo), _ints(bhi)),
                           "grid_add_box")
            else:
                _check(lib().ssamg_grid_set_box(self.h, p, _ints(lo), _ints(hi)), "grid_set_box")
        _check(lib().ssamg_grid_assemble(self.h), "grid_assemble")
        self.ndim = ndim
        self.boxes = [(tuple(lo), tuple(hi)) for lo, hi in boxes]
        self.n = lib().ssamg_grid_num_cells(self.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ssamg_grid_destroy(self.h)
            self.h = None


class Matrix:
    """Section 2: A = S + U with a stencil shared by the parts."""

    def __init__(self, grid: Grid, offsets):
        self.grid = grid
        offs = np.asarray(offsets, np.int32).reshape(-1, 3)
        self.offsets = offs
        self.h = _vp()
        _check(lib().ssamg_matrix_create(grid.h, len(offs), _ints(offs), ctypes.byref(self.h)),
               "matrix_create")

    def set_constant(self, part: int, entry: int, value: float):
        _check(lib().ssamg_matrix_set_constant(self.h, part, entry, float(value)), "set_constant")

    def set_box_values(self, part: int, entry: int, vals):
        if hasattr(vals, "is_cuda") and vals.is_cuda:
            lo, hi = self.grid.boxes[part]
            n = int(np.prod([hi[d] - lo[d] + 1 for d in range(3)]))
            _check(lib().ssamg_matrix_set_box_values(self.h, part, entry,
                                                     _dptr(vals, n, "vals"), 1),
                   "set_box_values")
        else:
            a = np.ascontiguousarray(vals, dtype=np.float64).ravel()
            _check(lib().ssamg_matrix_set_box_values(
                self.h, part, entry, a.ctypes.data_as(_vp), 0), "set_box_values")

    def add_couplings(self, part, idx, direction, nbor_part, nbor_idx, vals):
        n = len(vals)
        if n == 0:
            return
        v = np.ascontiguousarray(vals, np.float64)
        _check(lib().ssamg_matrix_add_couplings(
            self.h, n, _ints(part), _ints(idx), _ints(direction), _ints(nbor_part),
            _ints(nbor_idx), v.ctypes.data_as(_dp)), "add_couplings")

    def assemble(self, stream=None):
        _check(lib().ssamg_matrix_assemble(self.h, _stream(stream)), "matrix_assemble")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ssamg_matrix_destroy(self.h)
            self.h = None


def matrix_from_problem(prob, stream=None, device_values=False):
    """Grid and assembled matrix from a problem description with the fields
    ndim, boxes, offsets, coef, u_* (see the problems package)."""
    grid = Grid(prob.ndim, prob.boxes, getattr(prob, "part_boxes", None))
    A = Matrix(grid, prob.offsets)
    for p in range(len(prob.boxes)):
        for e in range(len(prob.offsets)):
            c = prob.coef[p][e]
            if np.isscalar(c):
                A.set_constant(p, e, float(c))
            elif device_values:
                import torch
                A.set_box_values(p, e, torch.as_tensor(np.ascontiguousarray(c).ravel(),
                                                       device="cuda"))
            else:
                A.set_box_values(p, e, c)
    if len(prob.u_val):
        A.add_couplings(prob.u_part, prob.u_idx, prob.u_dir, prob.u_nbor_part,
                        prob.u_nbor_idx, prob.u_val)
    A.assemble(stream)
    return grid, A


class Solver:
    """SSAMG-preconditioned CG (Sections 3 and 4)."""

    def __init__(self, params: Optional[Params] = None, **kw):
        self.params = params if params is not None else default_params(**kw)
        self.h = _vp()
        _check(lib().ssamg_solver_create(ctypes.byref(self.params), ctypes.byref(self.h)),
               "solver_create")
        self.matrix = None

    def setup(self, A: Matrix, stream=None):
        self.matrix = A
        _check(lib().ssamg_setup(self.h, A.h, _stream(stream)), "setup")

    def _n(self, level: int = 0) -> int:
        """Cells of a level of the set-up hierarchy (raises before setup)."""
        return self.level_sizes(level)[0]

    def _nparts(self) -> int:
        n = lib().ssamg_num_parts(self.h)
        if n < 0:
            raise SsamgError(n, "num_parts")
        return n

    def solve(self, b, x, nrhs: int = 1, zero_guess: bool = True, stream=None,
              allow_not_converged=False) -> Stats:
        st = Stats()
        n = nrhs * self._n()
        rc = lib().ssamg_solve(self.h, _dptr(b, n, "b"), _dptr(x, n, "x"), nrhs,
                               int(zero_guess), _stream(stream), ctypes.byref(st))
        _check(rc, "solve", (OK, NOT_CONVERGED) if allow_not_converged else (OK,))
        return st

    def solve_nostats(self, b, x, nrhs: int = 1, stream=None) -> int:
        n = nrhs * self._n()
        return _check(lib().ssamg_solve(self.h, _dptr(b, n, "b"), _dptr(x, n, "x"), nrhs, 1,
                                         _stream(stream), None), "solve", (OK, NOT_CONVERGED))

    def solve_host(self, b: np.ndarray, x: np.ndarray, nrhs: int = 1, stream=None,
                   stats=True) -> Stats:
        st = Stats()
        n = nrhs * self._n()
        if not (b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous
                and x.flags.c_contiguous and b.size >= n and x.size >= n):
            raise ValueError(f"b, x: expected contiguous float64 arrays of {n} elements")
        rc = lib().ssamg_solve_host(self.h, b.ctypes.data_as(_dp), x.ctypes.data_as(_dp), nrhs,
                                    _stream(stream), ctypes.byref(st) if stats else None)
        _check(rc, "solve_host", (OK, NOT_CONVERGED))
        return st

    def adjoint_solve(self, g, lam, nrhs: int = 1, stream=None,
                      allow_not_converged=False) -> Stats:
        st = Stats()
        n = nrhs * self._n()
        rc = lib().ssamg_adjoint_solve(self.h, _dptr(g, n, "g"), _dptr(lam, n, "lambda"), nrhs,
                                       _stream(stream), ctypes.byref(st))
        _check(rc, "adjoint_solve", (OK, NOT_CONVERGED) if allow_not_converged else (OK,))
        return st

    def coef_gradient(self, lam, x, dcoef, stream=None):
        n = self._n()
        ne = len(self.part_info(0, 0)["offsets"])
        _check(lib().ssamg_coef_gradient(self.h, _dptr(lam, n, "lambda"), _dptr(x, n, "x"),
                                         _dptr(dcoef, ne * n, "dcoef"), _stream(stream)),
               "coef_gradient")

    def diffusion_exp_gradient(self, g, lam, x, dg, stream=None):
        n = self._n()
        _check(lib().ssamg_diffusion_exp_gradient(self.h, _dptr(g, n, "g"), _dptr(lam, n, "lambda"),
                                                  _dptr(x, n, "x"), _dptr(dg, n, "dg"),
                                                  _stream(stream)),
               "diffusion_exp_gradient")

    def precondition(self, r, z, stream=None):
        n = self._n()
        _check(lib().ssamg_precondition(self.h, _dptr(r, n, "r"), _dptr(z, n, "z"),
                                        _stream(stream)), "precondition")

    def level_matvec(self, level: int, x, y, stream=None):
        n = self._n(level)
        _check(lib().ssamg_level_matvec(self.h, level, _dptr(x, n, "x"), _dptr(y, n, "y"),
                                        _stream(stream)), "level_matvec")

    # ---- introspection (host copies)
    def num_levels(self) -> int:
        n = lib().ssamg_num_levels(self.h)
        if n < 0:
            raise SsamgError(n, "num_levels")
        return n

    def level_sizes(self, level: int):
        n, r, z = _ll(), _ll(), _ll()
        _check(lib().ssamg_level_sizes(self.h, level, ctypes.byref(n), ctypes.byref(r),
                                       ctypes.byref(z)), "level_sizes")
        return n.value, r.value, z.value

    def part_info(self, level: int, part: int) -> dict:
        lo = (ctypes.c_int * 3)()
        hi = (ctypes.c_int * 3)()
        ds = ctypes.c_int()
        om = ctypes.c_double()
        ne = ctypes.c_int()
        offs = (ctypes.c_int * 81)()
        off = _ll()
        _check(lib().ssamg_level_part_info(self.h, level, part, lo, hi, ctypes.byref(ds),
                                           ctypes.byref(om), ctypes.byref(ne), offs,
                                           ctypes.byref(off)), "level_part_info")
        n = ne.value
        return {"lo": tuple(lo), "hi": tuple(hi), "dstar": ds.value, "omega": om.value,
                "offsets": [tuple(offs[3 * e:3 * e + 3]) for e in range(n)],
                "cell_offset": off.value}

    def tail_levels(self):
        """(first level, number of levels) of the coarse-level transition run
        in one cluster (use_tail = 3); (-1, 0) when there is none."""
        first, ctas = ctypes.c_int(), ctypes.c_int()
        smem = _ll()
        n = lib().ssamg_tail_levels(self.h, ctypes.byref(first), ctypes.byref(ctas),
                                    ctypes.byref(smem))
        if n < 0:
            raise SsamgError(n, "tail_levels")
        return first.value, n

    def stored_coefficients(self, level: int) -> int:
        v = _ll()
        _check(lib().ssamg_level_stored_coefficients(self.h, level, ctypes.byref(v)),
               "level_stored_coefficients")
        return int(v.value)

    def level_copy(self, level: int, what: int, part: int = 0, entry: int = 0, n: int = 0,
                   dtype=np.float64) -> np.ndarray:
        out = np.zeros(n, dtype)
        _check(lib().ssamg_level_copy(self.h, level, what, part, entry,
                                      out.ctypes.data_as(_vp), n), "level_copy")
        return out

    def time_kernel(self, kernel: int, level: int = 0, reps: int = 50, stream=None) -> float:
        """Mean microseconds per launch of one hot-path kernel (graph replay)."""
        us = ctypes.c_double()
        _check(lib().ssamg_time_kernel(self.h, kernel, level, reps, ctypes.byref(us),
                                       _stream(stream)), "time_kernel")
        return us.value

    # ---- tile forms (the tile table and its autotuner)
    def set_tile_table(self, table=None):
        """Tile table by level size class (TILE_CLASSES entries: 0, k or
        k | TILE_BRICKS, 1 <= k <= 4), or None for the built-in rule; it
        applies from the next setup."""
        _check(lib().ssamg_set_tile_table(self.h, None if table is None else _ints(table)),
               "set_tile_table")

    def tile_table(self) -> list:
        t = (ctypes.c_int * TILE_CLASSES)()
        _check(lib().ssamg_get_tile_table(self.h, t), "get_tile_table")
        return list(t)

    def level_tile(self, level: int):
        """(cells per thread, bricks) of a set-up level."""
        k, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().ssamg_level_tile(self.h, level, ctypes.byref(k), ctypes.byref(b)),
               "level_tile")
        return k.value, b.value

    def tile_key(self) -> str:
        """Cache key of a tuned tile table: the device, the cycle precision
        and the set-up hierarchy's level sizes."""
        import torch
        dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        sizes = ",".join(str(self.level_sizes(l)[0]) for l in range(self.num_levels()))
        return f"{dev}|p{self.params.precision}|b{self.params.use_bricks}|{sizes}"

    def autotune(self, reps: int = 30, stream=None, cache: Optional[str] = None,
                 resetup=None) -> list:
        """Tile autotuner (ssamg_autotune) on the set-up hierarchy; returns
        the table, which the solver keeps.  With `cache` (a JSON file), a
        table stored under tile_key() is taken instead of searching (the
        hierarchy is set up again with it, by `resetup` or setup() on the
        last matrix), and a searched table is stored."""
        key = self.tile_key()
        data = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
            if key in data:
                self.set_tile_table(data[key])
                (resetup or (lambda: self.setup(self.matrix, stream)))()
                return list(data[key])
        t = (ctypes.c_int * TILE_CLASSES)()
        _check(lib().ssamg_autotune(self.h, reps, _stream(stream), t), "autotune")
        table = list(t)
        if cache:
            data[key] = table
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return table

    def num_parts(self) -> int:
        return self._nparts()

    def spacings(self, nparts: Optional[int] = None):
        """Per-part coupling sums c and spacings W (n_parts x 3 each); the part
        count is the solver's (a given nparts must match it)."""
        np_solver = self._nparts()
        if nparts is not None and nparts != np_solver:
            raise ValueError(f"nparts {nparts} != the solver's {np_solver} parts")
        nparts = np_solver
        c = np.zeros(3 * nparts)
        W = np.zeros(3 * nparts)
        _check(lib().ssamg_spacings(self.h, c.ctypes.data_as(_dp), W.ctypes.data_as(_dp)),
               "spacings")
        return c.reshape(nparts, 3), W.reshape(nparts, 3)

    def residual_history(self, problem: int = 0, n: Optional[int] = None):
        """||r_k|| / ||b|| of the last solve, k = 0 .. iterations."""
        n = n if n is not None else 100000
        out = np.zeros(n)
        m = lib().ssamg_residual_history(self.h, problem, out.ctypes.data_as(_dp), n)
        if m < 0:
            _check(m, "residual_history")
        return out[:m]

    def set_spacings(self, W=None):
        """User representative grid spacings (n_parts x 3, > 0 or inf) used
        for coarsening from the next setup on; None returns to the ones
        computed from the coupling sums."""
        if W is None:
            _check(lib().ssamg_set_spacings(self.h, 0, None), "set_spacings")
            return
        a = np.ascontiguousarray(W, dtype=np.float64).reshape(-1, 3)
        _check(lib().ssamg_set_spacings(self.h, a.shape[0], a.ctypes.data_as(_dp)),
               "set_spacings")

    def coupling_sums_noalloc(self, level: int, c, stream=None):
        """Per-part coupling sums of `level` into the device tensor c (n_parts
        x 3 doubles), with no allocation or synchronisation (stream-ordered)."""
        _check(lib().ssamg_coupling_sums_noalloc(self.h, level, _dptr(c, 3 * self._nparts(), "c"),
                                                 _stream(stream)), "coupling_sums_noalloc")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None and getattr(self, "_owned", True):
            _lib.ssamg_solver_destroy(self.h)
        self.h = None


class Batch:
    """Many independent problems solved together (the batching form): one
    setup over all of them, and PCG with one instance per problem."""

    def __init__(self, matrices: Sequence["Matrix"], params: Optional[Params] = None, stream=None,
                 **kw):
        self.params = params if params is not None else default_params(**kw)
        self.matrices = list(matrices)
        arr = (_vp * len(self.matrices))(*[m.h for m in self.matrices])
        self.h = _vp()
        _check(lib().ssamg_batch_create(len(self.matrices), arr, ctypes.byref(self.params),
                                        _stream(stream), ctypes.byref(self.h)), "batch_create")
        self.nprob = len(self.matrices)

    def setup(self, stream=None):
        _check(lib().ssamg_batch_setup(self.h, _stream(stream)), "batch_setup")

    def num_cells(self) -> int:
        return int(lib().ssamg_batch_num_cells(self.h))

    def offsets(self):
        off = (_ll * (self.nprob + 1))()
        _check(lib().ssamg_batch_offsets(self.h, off), "batch_offsets")
        return [int(v) for v in off]

    def solve(self, b, x, nrhs: int = 1, stream=None, allow_not_converged=False):
        """b, x: contiguous float64 CUDA tensors of nrhs x N values; returns
        the nrhs x nprob stats (list of lists)."""
        st = (Stats * (nrhs * self.nprob))()
        n = nrhs * self.num_cells()
        rc = lib().ssamg_batch_solve(self.h, _dptr(b, n, "b"), _dptr(x, n, "x"), nrhs,
                                     _stream(stream), st)
        _check(rc, "batch_solve", (OK, NOT_CONVERGED) if allow_not_converged else (OK,))
        return [[st[j * self.nprob + k] for k in range(self.nprob)] for j in range(nrhs)]

    def autotune(self, reps: int = 30, stream=None, cache: Optional[str] = None) -> list:
        """Tile autotuner on the batch's hierarchy (see Solver.autotune)."""
        return self.solver().autotune(reps, stream, cache, resetup=lambda: self.setup(stream))

    def solver(self) -> "Solver":
        """The batch's solver (a view owned by the batch) for introspection
        and kernel timing."""
        sv = Solver.__new__(Solver)
        sv.params = self.params
        sv.h = _vp(lib().ssamg_batch_solver(self.h))
        sv.matrix = None
        sv._owned = False  # the batch destroys it
        sv._owner = self
        return sv

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ssamg_batch_destroy(self.h)
            self.h = None
