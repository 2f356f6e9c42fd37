"""FP64 CPU oracle for the PPM sweep (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never links or calls it.

``ppm_oracle.c`` holds the method (see its header for the paper sections it
follows); this module compiles it with gcc (no FMA contraction) and wraps it with
ctypes.  ``mlp.py`` holds the FP64 reference of the learned p* guess.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("rho_floor", ctypes.c_double),
                ("p_floor", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("newton_max", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("options", ctypes.c_int32)]


class OrStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("interfaces", "newton_iters", "newton_nonconv", "hll_cells", "neg_after",
                 "rho_floor_hits", "p_floor_hits", "ge_pressure")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


@dataclass
class Params:
    gamma: float = 5.0 / 3.0
    rho_floor: float = 1e-30
    p_floor: float = 1e-30
    newton_tol: float = 1e-14
    newton_max: int = 20
    fallback: int = 1
    solver: int = 0          # interface fluxes: 0 two-shock, 1 HLL, 2 HLLC
    options: int = 0         # bit 0 contact steepening, bit 1 flattening, bit 2 diffusive flux

    def c(self) -> OrParams:
        return OrParams(self.gamma, self.rho_floor, self.p_floor, self.newton_tol,
                        self.newton_max, self.fallback, self.solver, self.options)


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            five = [_D] * 5
            L.or_fill_periodic.argtypes = five + [_I32, ctypes.c_int32]
            L.or_fill_periodic.restype = None
            L.or_cfl_rate.argtypes = five + [_I32, ctypes.c_int32, _D, ctypes.POINTER(OrParams)]
            L.or_cfl_rate.restype = ctypes.c_double
            L.or_sweep.argtypes = five + [_I32, ctypes.c_int32, _D, ctypes.c_int32, ctypes.c_double,
                                          _I32, _I32, ctypes.POINTER(OrParams), ctypes.POINTER(OrStats)]
            L.or_sweep.restype = ctypes.c_int
            L.or_sweep_fluxes.argtypes = five + [_I32, ctypes.c_int32, _D, ctypes.c_int32, ctypes.c_double,
                                                 _I32, _I32, ctypes.POINTER(OrParams), ctypes.POINTER(OrStats), _D]
            L.or_sweep_fluxes.restype = ctypes.c_int
            L.or_sweep_fluxes_dual.argtypes = five + [_D, _I32, ctypes.c_int32, _D, ctypes.c_int32, ctypes.c_double,
                                                      _I32, _I32, ctypes.POINTER(OrParams), ctypes.POINTER(OrStats),
                                                      _D]
            L.or_sweep_fluxes_dual.restype = ctypes.c_int
            L.or_step_periodic.argtypes = five + [_I32, ctypes.c_int32, _D, ctypes.c_double,
                                                  ctypes.c_int32, ctypes.POINTER(OrParams),
                                                  ctypes.POINTER(OrStats)]
            L.or_step_periodic.restype = ctypes.c_int
            L.or_riemann_batch.argtypes = [ctypes.c_int64] + [_D] * 7 + [ctypes.POINTER(OrParams)] \
                + [_D] * 5 + [_I32]
            L.or_riemann_batch.restype = None
            L.or_flux_batch.argtypes = [ctypes.c_int64, ctypes.c_int32] + [_D] * 10 + \
                [ctypes.POINTER(OrParams), _D]
            L.or_flux_batch.restype = None
            L.or_pencil_debug.argtypes = [ctypes.c_int32, ctypes.c_int32, _D, ctypes.c_double,
                                          ctypes.POINTER(OrParams)] + [_D] * 7 + [ctypes.POINTER(OrStats)]
            L.or_pencil_debug.restype = ctypes.c_int
            L.or_fill_boundary.argtypes = five + [_I32, ctypes.c_int32, _I32]
            L.or_fill_boundary.restype = None
            L.or_step_boundary.argtypes = five + [_I32, ctypes.c_int32, _D, ctypes.c_double, ctypes.c_int32,
                                                  _I32, ctypes.POINTER(OrParams), ctypes.POINTER(OrStats)]
            L.or_step_boundary.restype = ctypes.c_int
            L.or_step_periodic_dual.argtypes = five + [_D, _I32, ctypes.c_int32, _D, ctypes.c_double,
                                                       ctypes.c_int32, ctypes.POINTER(OrParams),
                                                       ctypes.POINTER(OrStats)]
            L.or_step_periodic_dual.restype = ctypes.c_int
            L.or_num_threads.argtypes = []
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            L.or_set_num_threads.restype = None
        return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i32(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data_as(_I32)


def _fields(U):
    assert len(U) == 5
    return [_dp(u) for u in U]


def _n_of(U, ng):
    nz, ny, nx = U[0].shape
    return (nx - 2 * ng, ny - 2 * ng, nz - 2 * ng)


def fill_periodic(U, ng=3):
    """Periodic ghost fill of the five fields (and of a sixth, the dual-energy
    gas energy, when U has one: a scalar, filled like the density)."""
    n = _n_of(U, ng)
    na, npn = _i32(n)
    lib().or_fill_periodic(*_fields(U[:5]), npn, ng)
    if len(U) == 6:
        lib().or_fill_periodic(*_fields([U[5]] * 5), npn, ng)


BC_PERIODIC, BC_REFLECT, BC_OUTFLOW = 0, 1, 2


def fill_boundary(U, bc, ng=3):
    """External boundaries of a single grid, bc = (bc_x, bc_y, bc_z)."""
    na, npn = _i32(_n_of(U, ng))
    ba, bp = _i32(bc)
    lib().or_fill_boundary(*_fields(U[:5]), npn, ng, bp)
    if len(U) == 6:
        # the gas energy is a scalar: it takes the density's rule (the momentum
        # slots, whose reflection negates them, are scratch here)
        scratch = [np.zeros_like(U[5]) for _ in range(4)]
        lib().or_fill_boundary(*_fields([U[5]] + scratch), npn, ng, bp)


def step_boundary(U, dx, dt, step, bc, params: Params, ng=3) -> dict:
    """One step of a single grid with external boundaries bc (ghosts refilled first)."""
    na, npn = _i32(_n_of(U, ng))
    ba, bp = _i32(bc)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    p = params.c()
    st = OrStats()
    r = lib().or_step_boundary(*_fields(U), npn, ng, _dp(dxa), dt, step, bp, ctypes.byref(p), ctypes.byref(st))
    if r:
        raise MemoryError("oracle step could not allocate pencil scratch")
    return st.as_dict()


def cfl_rate(U, dx, params: Params, ng=3) -> float:
    na, npn = _i32(_n_of(U, ng))
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    p = params.c()
    return lib().or_cfl_rate(*_fields(U), npn, ng, _dp(dxa), ctypes.byref(p))


def cfl_dt(U, dx, params: Params, cfl=0.4, ng=3) -> float:
    return cfl / cfl_rate(U, dx, params, ng)


def sweep(U, dx, direction, dt, lo, hi, params: Params, ng=3) -> dict:
    na, npn = _i32(_n_of(U, ng))
    la, lp = _i32(lo)
    ha, hp = _i32(hi)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    p = params.c()
    st = OrStats()
    r = lib().or_sweep(*_fields(U), npn, ng, _dp(dxa), direction, dt, lp, hp,
                       ctypes.byref(p), ctypes.byref(st))
    if r:
        raise MemoryError("oracle sweep could not allocate pencil scratch")
    return st.as_dict()


def sweep_fluxes(U, dx, direction, dt, lo, hi, params: Params, ng=3, ge=None):
    """As sweep(), also returning the final face fluxes of the active pencils as
    an array [n_a2, n_a1, n_dir + 1, 5] (pencil field order rho, m_n, m_t1, m_t2, E).
    With ge (the dual-energy gas energy, updated in place) the array has a
    sixth component, the gas-energy flux."""
    n = _n_of(U, ng)
    na, npn = _i32(n)
    la, lp = _i32(lo)
    ha, hp = _i32(hi)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    a1 = 1 if direction == 0 else 0
    a2 = 1 if direction == 2 else 2
    F = np.zeros((n[a2], n[a1], n[direction] + 1, 5 if ge is None else 6))
    p = params.c()
    st = OrStats()
    if ge is None:
        r = lib().or_sweep_fluxes(*_fields(U), npn, ng, _dp(dxa), direction, dt, lp, hp, ctypes.byref(p),
                                  ctypes.byref(st), _dp(F))
    else:
        r = lib().or_sweep_fluxes_dual(*_fields(U), _dp(ge), npn, ng, _dp(dxa), direction, dt, lp, hp,
                                       ctypes.byref(p), ctypes.byref(st), _dp(F))
    if r:
        raise MemoryError("oracle sweep could not allocate pencil scratch" if r == -1 else
                          "oracle dual-energy sweep needs option bit 8 and the gas-energy field")
    return F, st.as_dict()


def step_periodic(U, dx, dt, step, params: Params, ng=3) -> dict:
    na, npn = _i32(_n_of(U, ng))
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    p = params.c()
    st = OrStats()
    r = lib().or_step_periodic(*_fields(U), npn, ng, _dp(dxa), dt, step, ctypes.byref(p),
                               ctypes.byref(st))
    if r:
        raise MemoryError("oracle step could not allocate pencil scratch")
    return st.as_dict()


def step_periodic_dual(U, ge, dx, dt, step, params: Params, ng=3) -> dict:
    """One periodic step with the dual-energy option on; ge (a ghost-zoned
    array like the fields) is the gas energy rho eps, updated in place."""
    na, npn = _i32(_n_of(U, ng))
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    p = params.c()
    st = OrStats()
    r = lib().or_step_periodic_dual(*_fields(U), _dp(ge), npn, ng, _dp(dxa), dt, step, ctypes.byref(p),
                                    ctypes.byref(st))
    if r:
        raise ValueError("oracle dual-energy step failed (option bit 8 needs the gas-energy field)")
    return st.as_dict()


def evolve_periodic(U, dx, nsteps, params: Params, cfl=0.4, step0=0, ng=3, dts=None):
    """Advance a periodic patch nsteps steps; dt from the CFL rule before each step
    (or from `dts` when given).  Returns (list of dt, summed stats)."""
    out_dt = []
    tot = None
    for s in range(nsteps):
        dt = dts[s] if dts is not None else cfl / cfl_rate(U, dx, params, ng)
        st = step_periodic(U, dx, dt, step0 + s, params, ng)
        tot = st if tot is None else {k: tot[k] + st[k] for k in tot}
        out_dt.append(dt)
    return out_dt, tot


def riemann(rl, ul, pl, rr, ur, pr, params: Params, pguess=None):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rl, ul, pl, rr, ur, pr)]
    n = arrs[0].size
    g = None if pguess is None else np.ascontiguousarray(pguess, dtype=np.float64)
    outs = [np.empty(n) for _ in range(5)]
    it = np.empty(n, dtype=np.int32)
    p = params.c()
    lib().or_riemann_batch(n, *[_dp(a) for a in arrs], _dp(g), ctypes.byref(p),
                           *[_dp(o) for o in outs], it.ctypes.data_as(_I32))
    return dict(pstar=outs[0], ustar=outs[1], rho=outs[2], u=outs[3], p=outs[4], iters=it)


SOLVER_TWOSHOCK, SOLVER_HLL, SOLVER_HLLC = 0, 1, 2
OPT_STEEPEN, OPT_FLATTEN, OPT_DIFFUSE, OPT_DUAL = 1, 2, 4, 8


def flux(left, right, params: Params, solver="twoshock"):
    """Fluxes for primitive states left/right = (rho, u, p, ut1, ut2) arrays;
    solver "twoshock", "hll" or "hllc"."""
    L = [np.ascontiguousarray(a, dtype=np.float64) for a in left]
    R = [np.ascontiguousarray(a, dtype=np.float64) for a in right]
    n = L[0].size
    F = np.empty((n, 5))
    p = params.c()
    lib().or_flux_batch(n, {"twoshock": 0, "hll": 1, "hllc": 2}[solver], *[_dp(a) for a in L],
                        *[_dp(a) for a in R], ctypes.byref(p), _dp(F))
    return F


def pencil_debug(Upen, dtdx, params: Params, ng=3) -> dict:
    """Run one pencil (array [5, L] of rho, m_n, m_t1, m_t2, E) and return its
    intermediate arrays, each [5, L]: qL, qR, q6, sL (left state at s+1/2),
    sR (right state at s-1/2), F (flux at s+1/2), Unew, plus stats."""
    U = np.ascontiguousarray(Upen, dtype=np.float64)
    L = U.shape[1]
    outs = {k: np.full((5, L), np.nan) for k in ("qL", "qR", "q6", "sL", "sR", "F", "Unew")}
    p = params.c()
    st = OrStats()
    r = lib().or_pencil_debug(L, ng, _dp(U), dtdx, ctypes.byref(p),
                              *[_dp(outs[k]) for k in ("qL", "qR", "q6", "sL", "sR", "F", "Unew")],
                              ctypes.byref(st))
    if r:
        raise MemoryError
    outs["stats"] = st.as_dict()
    return outs


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's pencil loops (timing only)."""
    lib().or_set_num_threads(int(n))
