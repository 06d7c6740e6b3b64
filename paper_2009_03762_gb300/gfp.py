"""Python binding of libgfp (ctypes): argument marshalling only; every step runs in the CUDA library.

There is no CPU fallback: if the shared library is missing, importing works but every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgfp.so")

TD, PCD = 0, 1
OPS = {"F": 0, "CD": 1, "ACD": 2, "HC": 3, "AHC": 4, "AFB_R": 5, "R": 5, "DGO": 6}
FP64, MIXED = 0, 1

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_UNSUPPORTED_SIZE", -3: "ERR_OOM", -4: "ERR_NOT_CONVERGED",
          -5: "ERR_DIVERGED", -6: "ERR_DEVICE_TIMEOUT", -7: "ERR_CUDA", -8: "ERR_UNSUPPORTED"}


class Scheme(ctypes.Structure):
    _fields_ = [("disc", ctypes.c_int), ("op", ctypes.c_int), ("dgo_m", ctypes.c_int), ("prec", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("dgo_power", ctypes.c_int), ("dgo_form", ctypes.c_int),
                ("dgo_range", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("residual", ctypes.c_double),
                ("sigma_mean", ctypes.c_double * 6), ("status", ctypes.c_int),
                ("residual_history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int),
                ("launches", ctypes.c_int)]


class GfpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = ""
        if code == -7 and _lib is not None:
            detail = ": " + _lib.gfp_last_error_detail().decode(errors="replace")
        super().__init__("%s failed: %s (%d)%s" % (where, STATUS.get(code, "?"), code, detail))


_lib = None

EXPORTS = ("gfp_create_grid", "gfp_set_phases", "gfp_solve", "gfp_get_strain", "gfp_effective_stiffness",
           "gfp_grad", "gfp_get_state", "gfp_set_state", "gfp_destroy_grid", "gfp_error_string",
           "gfp_time_passes", "gfp_last_error_detail", "gfp_solve_noalloc", "gfp_tune", "gfp_set_tiles",
           "gfp_solve_batch", "gfp_set_fault_injection", "gfp_set_eigenstrain", "gfp_get_displacement",
           "gfp_measure_fma_peak", "gfp_batch_create", "gfp_batch_solve", "gfp_batch_destroy", "gfp_get_plans",
           "gfp_set_plans")


def lib():
    """Load libgfp.so (built in-tree by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgfp.so not found at %s: build it with __graft_entry__.build(); "
                           "there is no CPU fallback" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.gfp_create_grid.argtypes = [ip, ip, ip, dp, vp, ctypes.POINTER(vp)]
    L.gfp_set_phases.argtypes = [vp, vp, vp, ip, vp]
    L.gfp_solve.argtypes = [vp, ctypes.POINTER(Scheme), vp, dp, ip, ctypes.POINTER(_Result)]
    L.gfp_get_strain.argtypes = [vp, vp, ip]
    L.gfp_effective_stiffness.argtypes = [vp, ctypes.POINTER(Scheme), dp, ip, vp, vp]
    L.gfp_grad.argtypes = [vp, ctypes.POINTER(Scheme), ip, ip, dp, ip, vp, vp, ip]
    L.gfp_get_state.argtypes = [vp, vp, ctypes.POINTER(ip)]
    L.gfp_set_state.argtypes = [vp, vp, ip]
    L.gfp_destroy_grid.argtypes = [vp]
    L.gfp_time_passes.argtypes = [vp, ctypes.POINTER(Scheme), ip, vp]
    L.gfp_error_string.argtypes = [ip]
    L.gfp_error_string.restype = ctypes.c_char_p
    L.gfp_solve_noalloc.argtypes = [ip, ip, ip, dp, vp, vp, vp, ctypes.POINTER(Scheme), vp, dp, ip, vp,
                                     ctypes.POINTER(_Result), vp]
    L.gfp_tune.argtypes = [vp, ctypes.POINTER(Scheme), ip, vp]
    L.gfp_solve_batch.argtypes = [ip, vp, ctypes.POINTER(Scheme), dp, ip, vp, vp]
    L.gfp_batch_create.argtypes = [ip, vp, ctypes.POINTER(Scheme), ctypes.POINTER(vp)]
    L.gfp_batch_solve.argtypes = [vp, dp, ip, vp, vp]
    L.gfp_batch_destroy.argtypes = [vp]
    L.gfp_set_fault_injection.argtypes = [ip, ip]
    L.gfp_measure_fma_peak.argtypes = [ip, ctypes.POINTER(ctypes.c_double)]
    L.gfp_set_tiles.argtypes = [vp, ip, vp]
    L.gfp_get_plans.argtypes = [vp, ip, vp, vp]
    L.gfp_set_plans.argtypes = [vp, ip, vp, vp]
    L.gfp_set_eigenstrain.argtypes = [vp, vp, ip]
    L.gfp_get_displacement.argtypes = [vp, ctypes.POINTER(Scheme), vp, ip]
    L.gfp_last_error_detail.argtypes = []
    L.gfp_last_error_detail.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("gfp_error_string", "gfp_last_error_detail"):
            getattr(L, name).restype = ip
    _lib = L
    return L


def _check(rc, where, ok=(0,)):
    if rc not in ok:
        raise GfpError(rc, where)
    return rc


def _gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "gpu"


def scheme(op="AFB_R", disc="TD", prec="FP64", dgo_m=0, stop_rule=0, dgo_power=2, dgo_form="polarization",
           dgo_range="printed"):
    """gfp_scheme; the dgo_* fields select the discrete-Green-operator variants (GFP_DGO only)."""
    return Scheme(TD if disc == "TD" else PCD, OPS[op], int(dgo_m), FP64 if prec == "FP64" else MIXED,
                  int(stop_rule), int(dgo_power), 1 if dgo_form == "stress" else 0,
                  1 if dgo_range == "symmetric" else 0)


def _ptr_where(a):
    """(pointer, where) for a numpy array (host) or a torch tensor (host or CUDA)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("expected a C-contiguous float64 array")
        return a.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    if not isinstance(a, torch.Tensor) or a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("expected a contiguous float64 tensor")
    return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)


class Result:
    def __init__(self, r, status, history):
        self.iters = r.iters
        self.outer = r.outer
        self.launches = r.launches
        self.residual = r.residual
        self.sigma_mean = np.array(list(r.sigma_mean))
        self.status = status
        self.converged = status == 0
        self.history = history


class Grid:
    """A periodic n1 x n2 x n3 cell on the GPU (owns all device buffers of the solver)."""

    def __init__(self, n1, n2, n3, h=1.0, stream=None):
        self.shape = (n3, n2, n1)
        self.N = n1 * n2 * n3
        L = lib()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self._h = ctypes.c_void_p()
        _check(L.gfp_create_grid(n1, n2, n3, float(h), ctypes.c_void_p(stream), ctypes.byref(self._h)),
               "gfp_create_grid")

    def close(self):
        if self._h:
            lib().gfp_destroy_grid(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_phases(self, lam, mu, ref=None):
        if isinstance(lam, np.ndarray):
            lam = np.ascontiguousarray(lam, dtype=np.float64)
            mu = np.ascontiguousarray(mu, dtype=np.float64)
        pl, wl = _ptr_where(lam)
        pm, wm = _ptr_where(mu)
        if wl != wm:
            raise ValueError("lambda and mu must live on the same side")
        refp = None
        if ref is not None:
            self._ref = (ctypes.c_double * 2)(float(ref[0]), float(ref[1]))
            refp = ctypes.cast(self._ref, ctypes.c_void_p)
        _check(lib().gfp_set_phases(self._h, pl, pm, wl, refp), "gfp_set_phases")

    def set_eigenstrain(self, estar):
        """Eigenstrain field [6, n3, n2, n1] float64 (numpy or torch), or None to remove it; the stress
        becomes C : (eps - estar)."""
        if estar is None:
            _check(lib().gfp_set_eigenstrain(self._h, None, 0), "gfp_set_eigenstrain")
            return
        if isinstance(estar, np.ndarray):
            estar = np.ascontiguousarray(estar, dtype=np.float64)
        count = estar.size if isinstance(estar, np.ndarray) else estar.numel()
        if count != 6 * int(np.prod(self.shape)):
            raise ValueError("eigenstrain must hold 6 x n3 x n2 x n1 values")
        p, w = _ptr_where(estar)
        _check(lib().gfp_set_eigenstrain(self._h, p, w), "gfp_set_eigenstrain")

    def displacement(self, sch, out=None):
        """Periodic displacement u^p [3, n3, n2, n1] of the last solve (scheme `sch`, as solved)."""
        if out is None:
            out = np.empty((3,) + self.shape)
        count = out.size if isinstance(out, np.ndarray) else out.numel()
        if count != 3 * int(np.prod(self.shape)):
            raise ValueError("displacement output must hold 3 x n3 x n2 x n1 values")
        p, w = _ptr_where(out)
        _check(lib().gfp_get_displacement(self._h, ctypes.byref(sch), p, w), "gfp_get_displacement")
        return out

    def solve(self, sch, E, tol=1e-8, maxit=1000, history=False, raise_on_error=False):
        E = (ctypes.c_double * 6)(*[float(v) for v in E])
        r = _Result()
        hist = None
        if history:
            hist = np.zeros(maxit)
            r.residual_history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            r.history_cap = maxit
        rc = lib().gfp_solve(self._h, ctypes.byref(sch), ctypes.cast(E, ctypes.c_void_p), float(tol), int(maxit),
                             ctypes.byref(r))
        if raise_on_error:
            _check(rc, "gfp_solve")
        elif rc not in (0, -4, -5, -6):
            raise GfpError(rc, "gfp_solve")
        if hist is not None:
            hist = hist[:r.iters]
        return Result(r, rc, hist)

    def strain(self, out=None):
        if out is None:
            out = np.empty((6,) + self.shape)
        p, w = _ptr_where(out)
        _check(lib().gfp_get_strain(self._h, p, w), "gfp_get_strain")
        return out

    def effective_stiffness(self, sch, tol=1e-8, maxit=1000):
        C = np.zeros(36)
        it = (ctypes.c_int * 6)()
        rc = lib().gfp_effective_stiffness(self._h, ctypes.byref(sch), float(tol), int(maxit),
                                           C.ctypes.data_as(ctypes.c_void_p), ctypes.cast(it, ctypes.c_void_p))
        _check(rc, "gfp_effective_stiffness", ok=(0, -4))
        return C.reshape(6, 6), list(it), rc

    def grad(self, sch, I, J, tol=1e-10, maxit=5000, out_lambda=None, out_mu=None):
        if out_lambda is None:
            out_lambda = np.empty(self.shape)
            out_mu = np.empty(self.shape)
        pl, wl = _ptr_where(out_lambda)
        pm, wm = _ptr_where(out_mu)
        if wl != wm:
            raise ValueError("outputs must live on the same side")
        _check(lib().gfp_grad(self._h, ctypes.byref(sch), int(I), int(J), float(tol), int(maxit), pl, pm, wl),
               "gfp_grad")
        return out_lambda, out_mu

    def time_passes(self, sch, iters):
        """Mean per-kernel durations (ms) of pass_x, pass_y, pass_z_gamma, reduce, pass_y inverse."""
        ms = np.zeros(5)
        _check(lib().gfp_time_passes(self._h, ctypes.byref(sch), int(iters), ms.ctypes.data_as(ctypes.c_void_p)),
               "gfp_time_passes")
        return ms

    def tune(self, sch, iters=5, cache=None):
        """Choose tile shapes and radix schedules with the native autotuner, or reuse them from a JSON cache.

        cache: path of a JSON file (default: $GFP_TUNE_CACHE if set); entries are keyed by grid size,
        precision and GPU name (the tiles) and by the same key + ":plans" (the radix schedules).
        Returns the tiles.
        """
        import json
        prec = sch.prec
        path = cache or os.environ.get("GFP_TUNE_CACHE")
        key = "%dx%dx%d:%d:%s" % (self.shape[2], self.shape[1], self.shape[0], prec, _gpu_name())
        table = {}
        if path and os.path.exists(path):
            try:
                with open(path) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if key in table:
            tiles = (ctypes.c_int * 3)(*table[key])
            _check(lib().gfp_set_tiles(self._h, int(prec), ctypes.cast(tiles, ctypes.c_void_p)), "gfp_set_tiles")
            if key + ":plans" in table:
                self.set_plans(prec, table[key + ":plans"])
            return list(table[key])
        out = (ctypes.c_int * 3)()
        _check(lib().gfp_tune(self._h, ctypes.byref(sch), int(iters), ctypes.cast(out, ctypes.c_void_p)), "gfp_tune")
        if path:
            table[key] = list(out)
            table[key + ":plans"] = self.get_plans(prec)
            with open(path, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return list(out)

    def get_plans(self, prec):
        """Radix schedules [axis][stage] of the shared-memory Stockham passes for one precision."""
        rad = (ctypes.c_int * 36)()
        nst = (ctypes.c_int * 3)()
        _check(lib().gfp_get_plans(self._h, int(prec), ctypes.cast(rad, ctypes.c_void_p),
                                   ctypes.cast(nst, ctypes.c_void_p)), "gfp_get_plans")
        return [[rad[12 * r + s] for s in range(nst[r])] for r in range(3)]

    def set_plans(self, prec, plans):
        rad = (ctypes.c_int * 36)()
        nst = (ctypes.c_int * 3)()
        for r, p in enumerate(plans):
            nst[r] = len(p)
            for s, v in enumerate(p[:12]):
                rad[12 * r + s] = int(v)
        _check(lib().gfp_set_plans(self._h, int(prec), ctypes.cast(rad, ctypes.c_void_p),
                                   ctypes.cast(nst, ctypes.c_void_p)), "gfp_set_plans")

    def set_tiles(self, prec, tiles):
        t = (ctypes.c_int * 3)(*[int(v) for v in tiles])
        _check(lib().gfp_set_tiles(self._h, int(prec), ctypes.cast(t, ctypes.c_void_p)), "gfp_set_tiles")

    def get_state(self):
        eps = np.empty((6,) + self.shape)
        it = ctypes.c_int()
        _check(lib().gfp_get_state(self._h, eps.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it)), "gfp_get_state")
        return eps, it.value

    def set_state(self, eps, iters):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        _check(lib().gfp_set_state(self._h, eps.ctypes.data_as(ctypes.c_void_p), int(iters)), "gfp_set_state")


def solve(lam, mu, op="AFB_R", E=(0.01, 0, 0, 0, 0, 0), tol=1e-8, maxit=1000, disc="TD", prec="FP64", h=1.0,
          ref=None, history=False):
    """One-shot convenience: create a grid, set the phases, solve, return (Result, strain)."""
    n3, n2, n1 = np.shape(lam)
    g = Grid(n1, n2, n3, h)
    try:
        g.set_phases(lam, mu, ref)
        r = g.solve(scheme(op, disc, prec), E, tol, maxit, history)
        return r, g.strain()
    finally:
        g.close()


class Batch:
    """A batch of cells (Grid objects with phases set) x 6 Voigt loads held as one CUDA graph
    (gfp_batch_create): slot buffers are allocated once, and each solve() is one graph launch."""

    def __init__(self, grids, sch):
        self.grids = list(grids)  # the handle uses the grids: keep them alive
        self.count = len(self.grids)
        handles = (ctypes.c_void_p * self.count)(*[g._h.value for g in self.grids])
        self._h = ctypes.c_void_p()
        _check(lib().gfp_batch_create(self.count, ctypes.cast(handles, ctypes.c_void_p), ctypes.byref(sch),
                                      ctypes.byref(self._h)), "gfp_batch_create")

    def solve(self, tol=1e-8, maxit=5000):
        """Returns (C_eff [count, 6, 6], inner iterations [count, 6], status)."""
        C = np.zeros((self.count, 36))
        its = np.zeros((self.count, 6), dtype=np.int32)
        rc = lib().gfp_batch_solve(self._h, float(tol), int(maxit), C.ctypes.data_as(ctypes.c_void_p),
                                   its.ctypes.data_as(ctypes.c_void_p))
        _check(rc, "gfp_batch_solve", ok=(0, -4))
        return C.reshape(self.count, 6, 6), its, rc

    def close(self):
        if self._h:
            lib().gfp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(grids, sch, tol=1e-8, maxit=5000):
    """Effective stiffness of several cells (Grid objects with phases set) in one batch: one graph
    launch in which every (cell, load) slot loops on the device until it converges (gfp_solve_batch).

    Returns (C_eff [count, 6, 6], inner iterations [count, 6], status).
    """
    count = len(grids)
    handles = (ctypes.c_void_p * count)(*[g._h.value for g in grids])
    C = np.zeros((count, 36))
    its = np.zeros((count, 6), dtype=np.int32)
    rc = lib().gfp_solve_batch(count, ctypes.cast(handles, ctypes.c_void_p), ctypes.byref(sch), float(tol), int(maxit),
                               C.ctypes.data_as(ctypes.c_void_p), its.ctypes.data_as(ctypes.c_void_p))
    _check(rc, "gfp_solve_batch", ok=(0, -4))
    return C.reshape(count, 6, 6), its, rc


def measure_fma_peak(dtype="f64"):
    """Peak FMA rate of the current GPU in TFLOP/s (gfp_measure_fma_peak), dtype "f64" or "f32"."""
    v = ctypes.c_double(0.0)
    _check(lib().gfp_measure_fma_peak(0 if dtype == "f64" else 1, ctypes.byref(v)), "gfp_measure_fma_peak")
    return v.value


def batch_shard(costs, rank, world):
    """Cells of a batch that rank `rank` of `world` solves.  Cells are dealt in order of decreasing cost
    (e.g. voxel count) to the rank with the least total so far, ties to the lower rank: deterministic,
    disjoint, covering, and balanced within one cell's cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += float(costs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def gather_batch(C_local, iters_local, idx_local, count, group=None):
    """All-gather of every rank's batch results (torch.distributed, any backend) into C_eff [count, 6, 6]
    and inner iterations [count, 6] on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    payload = ([int(i) for i in idx_local], np.asarray(C_local, dtype=np.float64).reshape(-1, 6, 6),
               np.asarray(iters_local, dtype=np.int64).reshape(-1, 6))
    objs = [None] * world
    dist.all_gather_object(objs, payload, group=group)
    C = np.full((count, 6, 6), np.nan)
    its = np.full((count, 6), -1, dtype=np.int64)
    for idx, Cl, il in objs:
        if len(idx):
            C[idx] = Cl
            its[idx] = il
    return C, its


def _solve_cells(cells, sch, tol, maxit):
    """gfp_solve_batch over (lam, mu) cells on this process's GPU; returns (C_eff, iterations, status)."""
    import torch
    grids = []
    try:
        for lam, mu in cells:
            n3, n2, n1 = np.shape(lam)
            g = Grid(n1, n2, n3, 1.0, torch.cuda.current_stream().cuda_stream)
            g.set_phases(lam, mu)
            grids.append(g)
        if not grids:
            return np.zeros((0, 6, 6)), np.zeros((0, 6), dtype=np.int32), 0
        return solve_batch(grids, sch, tol, maxit)
    finally:
        for g in grids:
            g.close()


def solve_batch_sharded(make_cell, costs, sch, tol=1e-8, maxit=5000, group=None, solver=None):
    """Batched homogenization across the ranks of torch.distributed (one GPU per rank): rank r builds the
    cells batch_shard(costs, r, world) with make_cell(i) -> (lam, mu), solves them with gfp_solve_batch,
    and every rank receives the full C_eff [count, 6, 6] and iterations [count, 6].  The only exchange is
    the gather of the results; there is no collective on the data path.  `solver` replaces the local
    solve (same signature as _solve_cells), e.g. in tests without a GPU.  Returns (C, iters, status)
    with the worst local status over the ranks."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    idx = batch_shard(costs, rank, world)
    C_l, it_l, rc = (solver or _solve_cells)([make_cell(i) for i in idx], sch, tol, maxit)
    C, its = gather_batch(C_l, it_l, idx, len(costs), group)
    codes = [None] * world
    dist.all_gather_object(codes, int(rc), group=group)
    worst = min(codes) if min(codes) < 0 else 0
    return C, its, worst


def solve_noalloc(lam, mu, eps, sch, E, tol=1e-8, maxit=1000, h=1.0, ref=None, stream=None):
    """Allocation-free FP64 solve through gfp_solve_noalloc.

    lam, mu: CUDA float64 tensors [n3, n2, n1]; eps: CUDA float64 tensor [6, n3, n2, n1] that receives
    the strain.  The library allocates no device memory for this call (its scratch is a fixed device
    array inside the library), so it suits callers that must not allocate.  Returns (status, Result).
    """
    import torch
    for a in (lam, mu, eps):
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise ValueError("expected contiguous CUDA float64 tensors")
    if lam.dim() != 3 or tuple(mu.shape) != tuple(lam.shape) or tuple(eps.shape) != (6,) + tuple(lam.shape):
        raise ValueError("expected lam, mu of shape (n3, n2, n1) and eps of shape (6, n3, n2, n1); got %s, %s, %s"
                         % (tuple(lam.shape), tuple(mu.shape), tuple(eps.shape)))
    if not (lam.device == mu.device == eps.device):
        raise ValueError("lam, mu and eps must be on one device")
    n3, n2, n1 = lam.shape
    with torch.cuda.device(lam.device):
        return _solve_noalloc_call(lam, mu, eps, sch, E, tol, maxit, h, ref, stream, n1, n2, n3)


def _solve_noalloc_call(lam, mu, eps, sch, E, tol, maxit, h, ref, stream, n1, n2, n3):
    """The C call of solve_noalloc with the tensors' device current (the library looks up its scratch there)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(lam.device).cuda_stream
    Ec = (ctypes.c_double * 6)(*[float(v) for v in E])
    refp = None
    if ref is not None:
        refa = (ctypes.c_double * 2)(float(ref[0]), float(ref[1]))
        refp = ctypes.cast(refa, ctypes.c_void_p)
    r = _Result()
    rc = lib().gfp_solve_noalloc(n1, n2, n3, float(h), ctypes.c_void_p(lam.data_ptr()),
                                 ctypes.c_void_p(mu.data_ptr()), refp, ctypes.byref(sch),
                                 ctypes.cast(Ec, ctypes.c_void_p), float(tol), int(maxit),
                                 ctypes.c_void_p(eps.data_ptr()), ctypes.byref(r), ctypes.c_void_p(stream))
    if rc not in (0, -4, -5):
        raise GfpError(rc, "gfp_solve_noalloc")
    return rc, Result(r, rc, None)


def _autograd():
    import torch

    class GfpCeff(torch.autograd.Function):
        """C_eff,IJ of a cell as a differentiable function of the voxel Lame fields (float64 tensors).

        forward runs the solve of load J on the GPU; backward calls gfp_grad, whose adjoint field is the
        forward solution of load I (Gamma is real and symmetric), and returns grad_out * dC/dlambda,
        grad_out * dC/dmu.
        """

        @staticmethod
        def forward(ctx, lam, mu, I, J, op, tol, maxit):
            n3, n2, n1 = lam.shape
            g = Grid(n1, n2, n3)
            lam_c = lam.detach().contiguous()
            mu_c = mu.detach().contiguous()
            g.set_phases(lam_c, mu_c)
            E = np.zeros(6)
            E[J] = 1.0 if J < 3 else 0.5
            r = g.solve(scheme(op), E, tol, maxit, raise_on_error=True)
            ctx.grid = g
            ctx.args = (I, J, op, tol, maxit)
            return torch.tensor(r.sigma_mean[I], dtype=torch.float64, device=lam.device)

        @staticmethod
        def backward(ctx, gout):
            I, J, op, tol, maxit = ctx.args
            g = ctx.grid
            shape = g.shape
            dev = gout.device
            dl = torch.empty(shape, dtype=torch.float64, device=dev)
            dm = torch.empty(shape, dtype=torch.float64, device=dev)
            g.grad(scheme(op), I, J, tol, maxit, dl, dm)
            g.close()
            return gout * dl, gout * dm, None, None, None, None, None

    return GfpCeff


def ceff_entry(lam, mu, I=0, J=0, op="AFB_R", tol=1e-10, maxit=5000):
    """Differentiable C_eff,IJ (torch autograd; backward via the hand-written adjoint and contraction kernel)."""
    return _autograd().apply(lam, mu, I, J, op, tol, maxit)
