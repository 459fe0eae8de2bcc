"""Thin ctypes binding of the C ABI in ``include/exx.h``.

Argument marshalling only: every step of the pair path runs in the CUDA
library ``lib/libexx.so``.  Device buffers are passed as raw pointers (for
instance ``torch.Tensor.data_ptr()``); host buffers are numpy arrays with
``mem=MEM_HOST``.  A missing library raises ``RuntimeError`` -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_CELL, ERR_HALO, ERR_NK, ERR_CG, ERR_CAPACITY, ERR_BOX, ERR_OOM, ERR_CUDA = range(10)
FP64, MIXED = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
STRESS_FULL, STRESS_ISOTROPIC, STRESS_CUBIC = 0, 1, 2
PRECOND_NONE, PRECOND_MG = 0, 1
SOLVER_CTA, SOLVER_CLUSTER = 0, 1

_lib = None
_lock = threading.Lock()

EXPORTS = ("exx_ctx_create", "exx_ctx_destroy", "exx_plan_create", "exx_plan_destroy", "exx_plan_query",
           "exx_pairs_solve", "exx_pairs_solve_batch", "exx_get_pair_list", "exx_dbox_halfwidth",
           "exx_ctx_set_timing", "exx_ctx_get_timing", "exx_error_string", "exx_last_error_detail", "exx_version",
           "exx_pair_list_noalloc", "exx_ctx_set_solver", "exx_cell_strain", "exx_geometry_query",
           "exx_dbox_layout", "exx_plan_get_schedule", "exx_plan_set_schedule", "exx_plan_autotune",
           "exx_plan_set_shard", "exx_pair_partition")


class Cell(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("n", C.c_int * 3)]


class Params(C.Structure):
    _fields_ = [("r_pair", C.c_double), ("r_pe_self", C.c_double), ("r_pe_pair", C.c_double),
                ("r_me_self", C.c_double), ("r_me_pair", C.c_double), ("cg_tol", C.c_double),
                ("fd_order", C.c_int), ("lmax", C.c_int), ("cg_max_iter", C.c_int), ("nq", C.c_int),
                ("precision", C.c_int), ("frozen", C.c_int), ("stress_mode", C.c_int), ("warm_start", C.c_int),
                ("guess", C.c_int), ("precond", C.c_int)]


class Orbitals(C.Structure):
    _fields_ = [("n_orb", C.c_int), ("box", C.c_int * 3), ("centres", C.c_void_p), ("box_lo", C.c_void_p),
                ("phi", C.c_void_p), ("mem", C.c_int)]


class Result(C.Structure):
    _fields_ = [("dxx", C.c_void_p), ("dbox_lo", C.c_void_p), ("dbox", C.c_int * 3), ("mem", C.c_int),
                ("pair_cap", C.c_int), ("pair_e", C.c_void_p), ("pair_sig", C.c_void_p), ("pair_iter", C.c_void_p),
                ("e_xx", C.c_double), ("dedh", C.c_double * 9), ("stress", C.c_double * 9),
                ("n_pairs", C.c_int), ("n_aux", C.c_int), ("n_stcl", C.c_int), ("max_cg_iter", C.c_int),
                ("total_cg_iter", C.c_longlong), ("max_refine", C.c_int), ("failed_pair", C.c_int),
                ("total_refine", C.c_longlong), ("p_int", C.c_double), ("n_warm", C.c_int)]


class Schedule(C.Structure):
    _fields_ = [("precond", C.c_int), ("omega", C.c_float), ("inner_shift", C.c_int), ("ms", C.c_double)]


def schedule_dict(sc: Schedule) -> dict:
    return {"precond": "mg" if sc.precond == PRECOND_MG else "none", "omega": round(float(sc.omega), 4),
            "inner_shift": int(sc.inner_shift), "ms": float(sc.ms)}


class PlanInfo(C.Structure):
    _fields_ = [("n_pe_self", C.c_int), ("n_me_self", C.c_int), ("n_pe_pair", C.c_int), ("n_me_pair", C.c_int),
                ("n_halo_self", C.c_int), ("n_halo_pair", C.c_int), ("n_aux", C.c_int), ("n_stcl", C.c_int),
                ("dirs", C.c_int * 18), ("coef", C.c_double * 6), ("aux_frozen", C.c_int * 9),
                ("box_self", C.c_int * 3), ("box_pair", C.c_int * 3), ("workspace_bytes", C.c_longlong),
                ("pair_capacity", C.c_int), ("ctas", C.c_int), ("threads", C.c_int), ("cluster", C.c_int),
                ("mg_levels", C.c_int), ("mg_points", C.c_int * 6)]


class ExxError(RuntimeError):
    def __init__(self, code, where=""):
        msg = lib().exx_error_string(code).decode() if _lib is not None else str(code)
        if code == ERR_CUDA and _lib is not None:
            msg += " [" + lib().exx_last_error_detail().decode() + "]"
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libexx.so (raises if it is missing and not built here)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library {path} is missing: run paper_2011_07209_gb300.build.build()")
                _build.build()
            L = C.CDLL(path)
            L.exx_error_string.restype = C.c_char_p
            L.exx_version.restype = C.c_char_p
            L.exx_last_error_detail.restype = C.c_char_p
            L.exx_ctx_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
            L.exx_ctx_destroy.argtypes = [C.c_void_p]
            L.exx_ctx_destroy.restype = None
            L.exx_plan_create.argtypes = [C.c_void_p, C.POINTER(Cell), C.POINTER(Params), C.c_int,
                                          C.POINTER(C.c_int), C.POINTER(C.c_void_p)]
            L.exx_plan_destroy.argtypes = [C.c_void_p]
            L.exx_plan_destroy.restype = None
            L.exx_plan_query.argtypes = [C.c_void_p, C.POINTER(PlanInfo)]
            L.exx_pairs_solve.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(Cell), C.POINTER(Orbitals),
                                          C.POINTER(Result), C.c_void_p]
            L.exx_pairs_solve_batch.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(Cell),
                                                C.POINTER(Orbitals), C.POINTER(Result), C.c_void_p]
            L.exx_get_pair_list.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.exx_dbox_halfwidth.argtypes = [C.POINTER(Cell), C.POINTER(Params), C.POINTER(C.c_int)]
            L.exx_cell_strain.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.exx_geometry_query.argtypes = [C.POINTER(Cell), C.POINTER(Params), C.POINTER(PlanInfo)]
            L.exx_dbox_layout.argtypes = [C.POINTER(Cell), C.POINTER(Params), C.c_int, C.c_void_p,
                                          C.POINTER(C.c_int), C.c_void_p]
            L.exx_plan_set_shard.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.exx_pair_partition.argtypes = [C.POINTER(Cell), C.POINTER(Params), C.c_int, C.c_void_p, C.c_int,
                                             C.c_void_p]
            L.exx_plan_get_schedule.argtypes = [C.c_void_p, C.POINTER(Schedule)]
            L.exx_plan_set_schedule.argtypes = [C.c_void_p, C.POINTER(Schedule)]
            L.exx_plan_autotune.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(Cell), C.POINTER(Orbitals), C.c_int,
                                            C.POINTER(Schedule), C.c_void_p]
            L.exx_ctx_set_timing.argtypes = [C.c_void_p, C.c_int]
            L.exx_ctx_set_solver.argtypes = [C.c_void_p, C.c_int]
            L.exx_pair_list_noalloc.argtypes = [C.POINTER(Cell), C.c_void_p, C.c_int, C.c_double, C.c_int,
                                                C.c_void_p, C.c_void_p, C.c_void_p]
            L.exx_ctx_get_timing.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
            _lib = L
    return _lib


def _check(code, where):
    if code != OK:
        raise ExxError(code, where)


def make_cell(lattice, n) -> Cell:
    c = Cell()
    for k, v in enumerate(np.asarray(lattice, float).ravel()):
        c.lattice[k] = float(v)
    for k in range(3):
        c.n[k] = int(n[k])
    return c


def make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, r_pe_self=None, r_me_self=None, tol=1e-9, fd_order=3, lmax=6,
                max_iter=20000, nq=15, precision=MIXED, frozen=False, stress_mode=0, warm_start=False,
                guess=True, precond=PRECOND_MG) -> Params:
    p = Params()
    p.r_pair = r_pair
    p.r_pe_pair = r_pe
    p.r_me_pair = r_me
    p.r_pe_self = r_pe if r_pe_self is None else r_pe_self
    p.r_me_self = r_me if r_me_self is None else r_me_self
    p.cg_tol = tol
    p.fd_order = fd_order
    p.lmax = lmax
    p.cg_max_iter = max_iter
    p.nq = nq
    p.precision = precision
    p.frozen = int(frozen)   # 0, 1 (offsets frozen) or 2 (offsets and aux directions frozen)
    p.stress_mode = int(stress_mode)
    p.warm_start = int(bool(warm_start))
    p.guess = int(bool(guess))
    p.precond = int(precond)
    return p


def dbox_halfwidth(lattice, n, params: Params):
    hw = (C.c_int * 3)()
    _check(lib().exx_dbox_halfwidth(C.byref(make_cell(lattice, n)), C.byref(params), hw), "exx_dbox_halfwidth")
    return np.array(list(hw), np.int64)


def cell_strain(lattice0, lattice):
    """(largest |principal Green-Lagrange strain|, relative volume change) of
    `lattice` relative to `lattice0` (rows are lattice vectors)."""
    a = (C.c_double * 9)(*[float(x) for x in np.asarray(lattice0, float).ravel()])
    b = (C.c_double * 9)(*[float(x) for x in np.asarray(lattice, float).ravel()])
    out = (C.c_double * 2)()
    _check(lib().exx_cell_strain(a, b, out), "exx_cell_strain")
    return float(out[0]), float(out[1])


class Reassembly:
    """When to re-assemble frozen proto-subdomains from scratch (Sec. III B 2):
    once the strain of the current cell relative to the plan's reference cell
    exceeds `eps_max` (largest principal Green-Lagrange strain), or every
    `stride` steps since the last assembly (0: no stride).  Re-assembling
    means creating a new Plan whose reference cell is the current one; its
    pairs start without a warm start (their offsets changed)."""

    def __init__(self, eps_max=None, stride=0):
        if eps_max is not None and not eps_max > 0.0:
            raise ValueError("eps_max must be positive")
        if stride < 0:
            raise ValueError("stride must be >= 0")
        self.eps_max = eps_max
        self.stride = int(stride)

    def due(self, lattice0, lattice, steps_since: int) -> bool:
        if self.stride and steps_since >= self.stride:
            return True
        return self.eps_max is not None and cell_strain(lattice0, lattice)[0] > self.eps_max


def pair_partition(lattice, n, params: Params, rows, n_ranks: int) -> np.ndarray:
    """exx_pair_partition: the rank of every pair row (host arithmetic, no GPU)."""
    rows = np.ascontiguousarray(np.asarray(rows, np.int32).reshape(-1, 8))
    owner = np.zeros(rows.shape[0], np.int32)
    _check(lib().exx_pair_partition(C.byref(make_cell(lattice, n)), C.byref(params), rows.shape[0],
                                    rows.ctypes.data_as(C.c_void_p), int(n_ranks), owner.ctypes.data_as(C.c_void_p)),
           "exx_pair_partition")
    return owner


def dbox_layout(lattice, n, centres, params: Params, dbox=None):
    """exx_dbox_layout: D-box extent and per-orbital first index (box around
    each centre's grid point).  A caller-chosen dbox (at least the required
    extent) can be given, e.g. to share one D buffer between the steps of a
    trajectory."""
    cen = np.ascontiguousarray(np.asarray(centres, float).reshape(-1, 3))
    n_orb = cen.shape[0]
    db = (C.c_int * 3)(*([0, 0, 0] if dbox is None else [int(x) for x in dbox]))
    lo = np.zeros((n_orb, 3), np.int32)
    code = lib().exx_dbox_layout(C.byref(make_cell(lattice, n)), C.byref(params), n_orb,
                                 cen.ctypes.data_as(C.c_void_p), db, lo.ctypes.data_as(C.c_void_p))
    if code == ERR_ARG and dbox is not None:
        raise ValueError(f"dbox {list(dbox)} outside the allowed range for this cell")
    _check(code, "exx_dbox_layout")
    return np.array(list(db), np.int32), lo


class Context:
    def __init__(self, device: int = 0):
        import weakref
        self.handle = C.c_void_p()
        self._plans = weakref.WeakSet()
        _check(lib().exx_ctx_create(C.byref(self.handle), int(device)), "exx_ctx_create")

    def set_timing(self, enable: bool = True):
        _check(lib().exx_ctx_set_timing(self.handle, int(enable)), "exx_ctx_set_timing")

    def set_solver(self, solver: int):
        """SOLVER_CTA (default) or SOLVER_CLUSTER for the mixed-precision pair solver."""
        _check(lib().exx_ctx_set_solver(self.handle, int(solver)), "exx_ctx_set_solver")

    def timing(self) -> dict:
        ms = (C.c_double * 4)()
        _check(lib().exx_ctx_get_timing(self.handle, ms), "exx_ctx_get_timing")
        return {"tables_ms": ms[0], "pairlist_ms": ms[1], "solve_ms": ms[2], "finalize_ms": ms[3]}

    def close(self):
        """Destroy the context; plans made from it are closed first."""
        if self.handle:
            for p in list(self._plans):
                p.close()
            lib().exx_ctx_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _info_dict(pi: PlanInfo) -> dict:
    return {
        "n_pe_self": pi.n_pe_self, "n_me_self": pi.n_me_self, "n_pe_pair": pi.n_pe_pair,
        "n_me_pair": pi.n_me_pair, "n_halo_self": pi.n_halo_self, "n_halo_pair": pi.n_halo_pair,
        "n_aux": pi.n_aux, "n_stcl": pi.n_stcl,
        "dirs": np.array(list(pi.dirs)).reshape(6, 3)[:3 + pi.n_aux], "coef": np.array(list(pi.coef))[:3 + pi.n_aux],
        "aux": np.array(list(pi.aux_frozen)).reshape(3, 3)[:pi.n_aux],
        "box_self": list(pi.box_self), "box_pair": list(pi.box_pair), "workspace_bytes": pi.workspace_bytes,
        "pair_capacity": pi.pair_capacity, "ctas": pi.ctas, "threads": pi.threads, "cluster": pi.cluster,
        "mg_points": list(pi.mg_points)[:pi.mg_levels],
    }


def geometry(lattice, n, params: Params) -> dict:
    """Geometry of a plan at this cell (point counts, dense boxes, NK stencil),
    computed on the host without a GPU; solver fields are zero."""
    pi = PlanInfo()
    _check(lib().exx_geometry_query(C.byref(make_cell(lattice, n)), C.byref(params), C.byref(pi)),
           "exx_geometry_query")
    return _info_dict(pi)


class Plan:
    def __init__(self, ctx: Context, lattice, n, params: Params, max_orb: int, box):
        self.ctx = ctx
        self.params = params
        self.handle = C.c_void_p()
        bx = (C.c_int * 3)(*[int(b) for b in box])
        _check(lib().exx_plan_create(ctx.handle, C.byref(make_cell(lattice, n)), C.byref(params), int(max_orb), bx,
                                     C.byref(self.handle)), "exx_plan_create")
        ctx._plans.add(self)

    def info(self) -> dict:
        pi = PlanInfo()
        _check(lib().exx_plan_query(self.handle, C.byref(pi)), "exx_plan_query")
        return _info_dict(pi)

    def set_shard(self, rank: int, n_ranks: int):
        """Solve only this rank's share of the pairs (exx_plan_set_shard); results are partial sums."""
        _check(lib().exx_plan_set_shard(self.handle, int(rank), int(n_ranks)), "exx_plan_set_shard")

    def schedule(self) -> dict:
        sc = Schedule()
        _check(lib().exx_plan_get_schedule(self.handle, C.byref(sc)), "exx_plan_get_schedule")
        return schedule_dict(sc)

    def set_schedule(self, precond, omega=0.7, inner_shift=14):
        sc = Schedule(int(precond), float(omega), int(inner_shift), 0.0)
        _check(lib().exx_plan_set_schedule(self.handle, C.byref(sc)), "exx_plan_set_schedule")

    def autotune(self, ctx, lattice, n, orb, sample_pairs=304, stream=None) -> dict:
        """exx_plan_autotune on this cell's first `sample_pairs` pairs; returns the chosen schedule."""
        sc = Schedule()
        s = C.c_void_p(stream) if isinstance(stream, int) else stream
        _check(lib().exx_plan_autotune(ctx.handle, self.handle, C.byref(make_cell(lattice, n)), C.byref(orb),
                                       int(sample_pairs), C.byref(sc), s), "exx_plan_autotune")
        return schedule_dict(sc)

    def pair_list(self) -> np.ndarray:
        n = C.c_int()
        lib().exx_get_pair_list(self.handle, 0, C.byref(n), None)
        rows = np.zeros((max(n.value, 1), 8), np.int32)
        _check(lib().exx_get_pair_list(self.handle, rows.shape[0], C.byref(n),
                                       rows.ctypes.data_as(C.POINTER(C.c_int))), "exx_get_pair_list")
        return rows[:n.value].copy()

    def close(self):
        if self.handle:
            lib().exx_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def make_orbitals(n_orb, box, centres, box_lo, phi, mem=MEM_DEVICE) -> Orbitals:
    o = Orbitals()
    o.n_orb = int(n_orb)
    for k in range(3):
        o.box[k] = int(box[k])
    o.centres = _ptr(centres)
    o.box_lo = _ptr(box_lo)
    o.phi = _ptr(phi)
    o.mem = mem
    return o


def make_result(dxx=None, dbox=None, dbox_lo=None, mem=MEM_DEVICE, pair_cap=0, pair_e=None, pair_sig=None,
                pair_iter=None) -> Result:
    r = Result()
    r.dxx = _ptr(dxx)
    r.dbox_lo = _ptr(dbox_lo)
    if dbox is not None:
        for k in range(3):
            r.dbox[k] = int(dbox[k])
    r.mem = mem
    r.pair_cap = int(pair_cap)
    r.pair_e = _ptr(pair_e)
    r.pair_sig = _ptr(pair_sig)
    r.pair_iter = _ptr(pair_iter)
    return r


def solve(ctx: Context, plan: Plan, lattice, n, orb: Orbitals, res: Result, stream=None, check=True) -> int:
    """exx_pairs_solve; returns the status (raises on error when check=True)."""
    s = C.c_void_p(stream) if isinstance(stream, int) else stream
    code = lib().exx_pairs_solve(ctx.handle, plan.handle, C.byref(make_cell(lattice, n)), C.byref(orb),
                                 C.byref(res), s)
    if check:
        _check(code, "exx_pairs_solve")
    return code


def solve_batch(ctx: Context, plans, cells, orbs, results, stream=None, check=True) -> int:
    k = len(plans)
    ph = (C.c_void_p * k)(*[p.handle.value for p in plans])
    ca = (Cell * k)(*[make_cell(lat, n) for lat, n in cells])
    oa = (Orbitals * k)(*orbs)
    ra = (Result * k)(*results)
    s = C.c_void_p(stream) if isinstance(stream, int) else stream
    code = lib().exx_pairs_solve_batch(ctx.handle, k, ph, ca, oa, ra, s)
    for i in range(k):
        results[i] = ra[i]
    if check:
        _check(code, "exx_pairs_solve_batch")
    return code


def result_dict(r: Result) -> dict:
    return {"e_xx": r.e_xx, "dedh": np.array(list(r.dedh)).reshape(3, 3),
            "stress": np.array(list(r.stress)).reshape(3, 3), "n_pairs": r.n_pairs, "n_aux": r.n_aux,
            "n_stcl": r.n_stcl, "max_cg_iter": r.max_cg_iter, "total_cg_iter": r.total_cg_iter,
            "max_refine": r.max_refine, "failed_pair": r.failed_pair, "total_refine": r.total_refine,
            "p_int": r.p_int, "n_warm": r.n_warm}


def pair_list_noalloc(lattice, n, centres, n_orb, r_pair, rows, n_pairs, stream=None) -> int:
    """exx_pair_list_noalloc: centres, rows ([cap][8] int32) and n_pairs (int32) are
    device buffers (torch tensors); returns the status code."""
    cap = int(rows.shape[0]) if rows is not None else 0
    s = C.c_void_p(stream) if isinstance(stream, int) else stream
    return lib().exx_pair_list_noalloc(C.byref(make_cell(lattice, n)), _ptr(centres), int(n_orb), float(r_pair), cap,
                                       _ptr(rows), _ptr(n_pairs), s)
