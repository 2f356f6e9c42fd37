"""Python binding of libenzo_ppm, the GB300 split PPM hydro sweep.

This module only marshals arguments: every step of the method runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There is
no CPU fallback; if the library cannot be built or loaded, `lib()` raises.

Entry points mirror include/enzo_ppm.h: ppm_sweep, ghost_fill_periodic,
timestep_cfl, step, riemann_solve (and read_status, strerror).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

FP64, FP32 = 0, 1
GUESS_PLAIN, GUESS_MLP = 0, 1
SOLVER_TWOSHOCK, SOLVER_HLL, SOLVER_HLLC = 0, 1, 2
OPT_STEEPEN, OPT_FLATTEN, OPT_DIFFUSE, OPT_DUAL = 1, 2, 4, 8
PATCH_PERIODIC = 1
STATUS_WORDS = 16
STATUS_NAMES = ("interfaces", "newton_iters", "newton_nonconv", "hll_cells", "neg_after",
                "rho_floor_hits", "p_floor_hits", "nan", "bad_patch", "fp64_eke",
                "guess_restarts", "guess_calls", "timeout", "ge_pressure")

PATCH_DTYPE = np.dtype([("n", "<i4", (3,)), ("ng", "<i4"), ("off", "<i8"), ("dx", "<f8", (3,)),
                        ("level", "<i4"), ("flags", "<i4"), ("freg_all", "<i8"), ("freg_bnd", "<i8")])
assert PATCH_DTYPE.itemsize == 72


class EnzoError(RuntimeError):
    pass


class _Batch(ctypes.Structure):
    _fields_ = [("npatch", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("patches", ctypes.c_void_p), ("field_len", ctypes.c_int64),
                ("U", ctypes.c_void_p * 5), ("workspace", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t), ("status", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("freg", ctypes.c_void_p), ("ge", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("precision", ctypes.c_int32), ("guess", ctypes.c_int32),
                ("newton_tol", ctypes.c_double), ("newton_max", ctypes.c_int32),
                ("fallback", ctypes.c_int32), ("rho_floor", ctypes.c_double),
                ("p_floor", ctypes.c_double), ("mlp", ctypes.c_void_p),
                ("tile", ctypes.c_int32 * 3), ("solver", ctypes.c_int32), ("mlp_gate", ctypes.c_double),
                ("options", ctypes.c_int32)]


class _Riemann(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in
                ("rhoL", "uL", "pL", "rhoR", "uR", "pR", "pguess", "pstar", "ustar",
                 "rho_face", "u_face", "p_face", "iters", "stream")]


_lib = None
_lock = threading.Lock()


def lib():
    """Load (building first if stale) libenzo_ppm.so; raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.enzo_workspace_size.argtypes = [i32]
            L.enzo_workspace_size.restype = ctypes.c_size_t
            L.enzo_validate_patches.argtypes = [vp, i32, i64, ctypes.POINTER(i32)]
            L.enzo_ppm_sweep.argtypes = [ctypes.POINTER(_Batch), i32, d, i32, ctypes.POINTER(_Params)]
            L.enzo_ppm_sweep_dev.argtypes = [ctypes.POINTER(_Batch), i32, vp, i32, ctypes.POINTER(_Params)]
            L.enzo_ppm_sweep_noalloc.argtypes = [ctypes.POINTER(_Batch), i32, d, i32, ctypes.POINTER(_Params)]
            L.enzo_ppm_sweep_logged.argtypes = [ctypes.POINTER(_Batch), i32, d, i32, ctypes.POINTER(_Params),
                                                vp, vp, i64, i32]
            L.enzo_ghost_fill_periodic.argtypes = [ctypes.POINTER(_Batch)]
            L.enzo_timestep_cfl.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(_Params), vp, i32]
            L.enzo_step.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(_Params), i32, vp]
            L.enzo_ghost_fill_boundary.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(i32)]
            L.enzo_step_boundary.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(_Params), i32, vp,
                                             ctypes.POINTER(i32)]
            L.enzo_riemann_solve.argtypes = [ctypes.POINTER(_Riemann), ctypes.POINTER(_Params)]
            L.enzo_pack_active.argtypes = [ctypes.POINTER(_Batch), vp, vp, vp]
            L.enzo_unpack_active.argtypes = [ctypes.POINTER(_Batch), vp, vp, vp]
            L.enzo_strerror.argtypes = [ctypes.c_int]
            L.enzo_strerror.restype = ctypes.c_char_p
            L.enzo_launch_count.argtypes = []
            L.enzo_launch_count.restype = ctypes.c_ulonglong
            for name in ("enzo_validate_patches", "enzo_ppm_sweep", "enzo_ppm_sweep_dev", "enzo_ppm_sweep_noalloc",
                         "enzo_ghost_fill_periodic", "enzo_ppm_sweep_logged",
                         "enzo_timestep_cfl", "enzo_step", "enzo_riemann_solve",
                         "enzo_ghost_fill_boundary", "enzo_step_boundary", "enzo_pack_active",
                         "enzo_unpack_active"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
        return _lib


def strerror(code: int) -> str:
    return lib().enzo_strerror(code).decode()


def _check(code: int, what: str):
    if code != 0:
        raise EnzoError(f"{what}: {strerror(code)} ({code})")


def launch_count() -> int:
    return int(lib().enzo_launch_count())


class Params:
    """Method parameters (enzo_params)."""

    def __init__(self, gamma=5.0 / 3.0, cfl=0.4, precision=FP64, guess=GUESS_PLAIN, newton_tol=0.0,
                 newton_max=0, fallback=1, rho_floor=1e-30, p_floor=1e-30, mlp=None, tile=(0, 0, 0),
                 mlp_gate=0.0, solver=SOLVER_TWOSHOCK, options=0):
        self.gamma, self.cfl, self.precision, self.guess = gamma, cfl, precision, guess
        self.newton_tol, self.newton_max, self.fallback = newton_tol, newton_max, fallback
        self.rho_floor, self.p_floor, self.mlp = rho_floor, p_floor, mlp
        self.tile = tuple(tile)
        self.mlp_gate = mlp_gate
        self.solver = solver
        self.options = options

    def c(self) -> _Params:
        mlp_ptr = 0 if self.mlp is None else (self.mlp.data_ptr() if hasattr(self.mlp, "data_ptr") else int(self.mlp))
        return _Params(self.gamma, self.cfl, self.precision, self.guess, self.newton_tol,
                       self.newton_max, self.fallback, self.rho_floor, self.p_floor, mlp_ptr,
                       (ctypes.c_int32 * 3)(*self.tile), self.solver, self.mlp_gate, self.options)


def patch_table(sizes, offsets, dx, flags=0, ng=3, level=0) -> np.ndarray:
    """Host descriptor table (PATCH_DTYPE) for patches of active sizes (nx,ny,nz)."""
    sizes = np.asarray(sizes, dtype=np.int64).reshape(-1, 3)
    t = np.zeros(len(sizes), dtype=PATCH_DTYPE)
    t["n"] = sizes
    t["ng"] = ng
    t["off"] = np.asarray(offsets, dtype=np.int64)
    t["dx"] = np.broadcast_to(np.asarray(dx, dtype=np.float64), (len(sizes), 3))
    t["level"] = level
    t["flags"] = flags
    t["freg_all"] = -1
    t["freg_bnd"] = -1
    return t


class PatchBatch:
    """A batch of patches sharing one timestep, with device fields, descriptors,
    workspace and status counters held in torch tensors on one CUDA device."""

    def __init__(self, table: np.ndarray, fields, device="cuda", stream=None, ge=None):
        """fields: the five conserved fields (rho, m_x, m_y, m_z, E), flat over
        the batch's storage; ge: optional gas-energy field rho e of the same
        length (needed by sweeps with OPT_DUAL, carried by the ghost fills)."""
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.table = np.ascontiguousarray(table, dtype=PATCH_DTYPE)
        if isinstance(fields[0], torch.Tensor):
            self.U = [f.to(self.device, torch.float64).contiguous() for f in fields]
        else:
            self.U = [torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64)).to(self.device) for f in fields]
        self.field_len = int(self.U[0].numel())
        assert all(int(u.numel()) == self.field_len for u in self.U)
        bad = ctypes.c_int32(-1)
        _check(lib().enzo_validate_patches(self.table.ctypes.data, len(self.table), self.field_len,
                                           ctypes.byref(bad)), f"patch {bad.value}")
        raw = np.frombuffer(self.table.tobytes(), dtype=np.uint8).copy()
        self.patches = torch.from_numpy(raw).to(self.device)
        ws = int(lib().enzo_workspace_size(len(self.table)))
        self.workspace = torch.zeros(ws // 8 + 32, dtype=torch.float64, device=self.device)
        self.status = torch.zeros(STATUS_WORDS, dtype=torch.int64, device=self.device)
        self.dt_dev = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.stream = stream
        self._ws_bytes = ws
        self.freg = None
        self.ge = None
        if ge is not None:
            if isinstance(ge, torch.Tensor):
                self.ge = ge.to(self.device, torch.float64).contiguous()
            else:
                self.ge = torch.from_numpy(np.ascontiguousarray(ge, dtype=np.float64)).to(self.device)
            assert int(self.ge.numel()) == self.field_len

    @classmethod
    def wrap(cls, table, U, patches, workspace, ws_bytes, status, stream, freg=None, ge=None):
        """A batch over device tensors that already hold its state (descriptors,
        five fields, workspace, status words; flux registers and gas energy
        optional), e.g. a level of a native hierarchy.  Nothing is copied."""
        import torch
        b = cls.__new__(cls)
        b.torch = torch
        b.device = U[0].device
        b.table = np.ascontiguousarray(table, dtype=PATCH_DTYPE)
        b.U = list(U)
        b.field_len = int(U[0].numel())
        b.patches = patches
        b.workspace = workspace
        b._ws_bytes = int(ws_bytes)
        b.status = status
        b.dt_dev = torch.zeros(1, dtype=torch.float64, device=b.device)
        b.stream = stream
        b.freg = freg
        b.ge = ge
        return b

    def c(self) -> _Batch:
        b = _Batch()
        b.npatch = len(self.table)
        b.patches = self.patches.data_ptr()
        b.field_len = self.field_len
        for i in range(5):
            b.U[i] = self.U[i].data_ptr()
        b.workspace = self.workspace.data_ptr()
        b.ws_bytes = self._ws_bytes
        b.status = self.status.data_ptr()
        s = self.stream if self.stream is not None else self.torch.cuda.current_stream(self.device)
        b.stream = s.cuda_stream
        b.freg = self.freg.data_ptr() if self.freg is not None else None
        b.ge = self.ge.data_ptr() if self.ge is not None else None
        return b

    def read_status(self) -> dict:
        v = self.status.cpu().numpy().astype(np.uint64)
        return {n: int(v[i]) for i, n in enumerate(STATUS_NAMES)}

    def reset_status(self):
        self.status.zero_()

    def patch_fields(self, i):
        """Device views (z, y, x) of patch i's five stored fields."""
        nx, ny, nz = (int(v) for v in self.table["n"][i])
        g = int(self.table["ng"][i])
        off = int(self.table["off"][i])
        cnt = (nx + 2 * g) * (ny + 2 * g) * (nz + 2 * g)
        return [u[off:off + cnt].view(nz + 2 * g, ny + 2 * g, nx + 2 * g) for u in self.U]

    def patch_ge(self, i):
        """Device view (z, y, x) of patch i's stored gas energy (OPT_DUAL)."""
        nx, ny, nz = (int(v) for v in self.table["n"][i])
        g = int(self.table["ng"][i])
        off = int(self.table["off"][i])
        cnt = (nx + 2 * g) * (ny + 2 * g) * (nz + 2 * g)
        return self.ge[off:off + cnt].view(nz + 2 * g, ny + 2 * g, nx + 2 * g)


def ppm_sweep(batch: PatchBatch, direction: int, dt: float, cover_mask: int, params: Params):
    b, p = batch.c(), params.c()
    _check(lib().enzo_ppm_sweep(ctypes.byref(b), direction, dt, cover_mask, ctypes.byref(p)), "enzo_ppm_sweep")


def ppm_sweep_dev(batch: PatchBatch, direction: int, dt_dev, cover_mask: int, params: Params):
    """Sweep with dt read on the device from the 1-element float64 tensor dt_dev."""
    b, p = batch.c(), params.c()
    _check(lib().enzo_ppm_sweep_dev(ctypes.byref(b), direction, dt_dev.data_ptr(), cover_mask, ctypes.byref(p)),
           "enzo_ppm_sweep_dev")


def ppm_sweep_noalloc(batch: PatchBatch, direction: int, dt: float, cover_mask: int, params: Params):
    """Same sweep as ppm_sweep, for callers that cannot allocate device memory:
    the library keeps the scratch in its own fixed device array (at most 32000
    patches per call; calls that overlap on the GPU race on it), so the batch's
    workspace is not used."""
    b, p = batch.c(), params.c()
    b.workspace = None
    b.ws_bytes = 0
    _check(lib().enzo_ppm_sweep_noalloc(ctypes.byref(b), direction, dt, cover_mask, ctypes.byref(p)),
           "enzo_ppm_sweep_noalloc")


def ppm_sweep_logged(batch: PatchBatch, direction: int, dt: float, cover_mask: int, params: Params,
                     log, log_count, stride: int):
    """Sweep that appends sampled traced interface states to log (float32 [cap, 6])."""
    b, p = batch.c(), params.c()
    _check(lib().enzo_ppm_sweep_logged(ctypes.byref(b), direction, dt, cover_mask, ctypes.byref(p),
                                       log.data_ptr(), log_count.data_ptr(), log.shape[0], stride),
           "enzo_ppm_sweep_logged")


def ghost_fill_periodic(batch: PatchBatch):
    b = batch.c()
    _check(lib().enzo_ghost_fill_periodic(ctypes.byref(b)), "enzo_ghost_fill_periodic")


def active_offsets(table) -> np.ndarray:
    """Offsets of each patch's block in the packed active-cell layout of
    pack_active / unpack_active (blocks in patch order, no gaps)."""
    cells = np.prod(np.asarray(table["n"], dtype=np.int64), axis=1)
    return np.concatenate([[0], np.cumsum(cells)[:-1]]).astype(np.int64)


def _pack(batch: PatchBatch, packed, act_off, packed_ge, name):
    if len(packed) != 5:
        raise ValueError("five packed fields")
    b = batch.c()
    arr = (ctypes.c_void_p * 5)(*[t.data_ptr() for t in packed])
    _check(getattr(lib(), name)(ctypes.byref(b), arr, packed_ge.data_ptr() if packed_ge is not None else None,
                                act_off.data_ptr()), name)


def pack_active(batch: PatchBatch, packed, act_off, packed_ge=None):
    """Copy every patch's active cells into the packed device arrays `packed`
    (five float64 tensors; patch i's cells, x fastest, from act_off[i], a
    device int64 tensor), and the gas energy into packed_ge when given."""
    _pack(batch, packed, act_off, packed_ge, "enzo_pack_active")


def unpack_active(batch: PatchBatch, packed, act_off, packed_ge=None):
    """The reverse of pack_active: active cells from the packed arrays; ghost
    zones are left as they are."""
    _pack(batch, packed, act_off, packed_ge, "enzo_unpack_active")


def timestep_cfl(batch: PatchBatch, params: Params, out=None):
    """Level dt (Sec. 9).  With `out` (a 1-element float64 CUDA tensor) the result
    stays on the device; otherwise it is returned as a Python float."""
    b, p = batch.c(), params.c()
    if out is not None:
        _check(lib().enzo_timestep_cfl(ctypes.byref(b), ctypes.byref(p), out.data_ptr(), 1), "enzo_timestep_cfl")
        return out
    host = ctypes.c_double(0.0)
    _check(lib().enzo_timestep_cfl(ctypes.byref(b), ctypes.byref(p), ctypes.addressof(host), 0), "enzo_timestep_cfl")
    return host.value


def step(batch: PatchBatch, params: Params, step_index: int, dt_dev):
    """Ghost fill + three split sweeps in the order of step_index; dt read on the device."""
    b, p = batch.c(), params.c()
    _check(lib().enzo_step(ctypes.byref(b), ctypes.byref(p), step_index, dt_dev.data_ptr()), "enzo_step")


BC_PERIODIC, BC_REFLECT, BC_OUTFLOW = 0, 1, 2


def _bc(bc):
    if len(bc) != 3:
        raise ValueError("bc needs one condition per axis")
    return (ctypes.c_int32 * 3)(*[int(v) for v in bc])


def ghost_fill_boundary(batch: PatchBatch, bc):
    """Ghost fill of each non-periodic patch as a grid with external boundaries
    bc = (bc_x, bc_y, bc_z), each BC_PERIODIC, BC_REFLECT or BC_OUTFLOW."""
    b = batch.c()
    _check(lib().enzo_ghost_fill_boundary(ctypes.byref(b), _bc(bc)), "enzo_ghost_fill_boundary")


def step_boundary(batch: PatchBatch, params: Params, step_index: int, dt_dev, bc):
    """As step(), with the external boundaries bc of ghost_fill_boundary()."""
    b, p = batch.c(), params.c()
    _check(lib().enzo_step_boundary(ctypes.byref(b), ctypes.byref(p), step_index, dt_dev.data_ptr(), _bc(bc)),
           "enzo_step_boundary")


def riemann_solve(rl, ul, pl, rr, ur, pr, params: Params, pguess=None, stream=None):
    """Batched Riemann problems on device tensors (float64 for FP64, float32 for FP32)."""
    import torch
    n = rl.numel()
    dt = torch.float64 if params.precision == FP64 else torch.float32
    ins = [t.contiguous() for t in (rl, ul, pl, rr, ur, pr)]
    assert all(t.dtype == dt and t.is_cuda for t in ins)
    outs = [torch.empty(n, dtype=dt, device=rl.device) for _ in range(5)]
    iters = torch.empty(n, dtype=torch.int32, device=rl.device)
    s = _Riemann()
    s.n = n
    s.rhoL, s.uL, s.pL, s.rhoR, s.uR, s.pR = (t.data_ptr() for t in ins)
    s.pguess = 0 if pguess is None else pguess.contiguous().data_ptr()
    s.pstar, s.ustar, s.rho_face, s.u_face, s.p_face = (t.data_ptr() for t in outs)
    s.iters = iters.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream(rl.device)
    s.stream = st.cuda_stream
    p = params.c()
    _check(lib().enzo_riemann_solve(ctypes.byref(s), ctypes.byref(p)), "enzo_riemann_solve")
    return dict(pstar=outs[0], ustar=outs[1], rho=outs[2], u=outs[3], p=outs[4], iters=iters)


def evolve(batch: PatchBatch, params: Params, nsteps: int, step0: int = 0, use_step=True):
    """Advance nsteps steps: device CFL dt, then enzo_step (all on the stream)."""
    for s in range(nsteps):
        timestep_cfl(batch, params, out=batch.dt_dev)
        step(batch, params, step0 + s, batch.dt_dev)


# ---------------------------------------------------------------------------
# learned Newton starting guess (enzo_mlp_*)
# ---------------------------------------------------------------------------
MLP_PARAMS = 4673
MLP_BLOB_BYTES = 19456
MLP_SLICES = {"W1": (0, (64, 6)), "b1": (384, (64,)), "W2": (448, (64, 64)), "b2": (4544, (64,)),
              "w3": (4608, (64,)), "b3": (4672, (1,))}


def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.enzo_mlp_pack.argtypes = [vp, vp, vp]
        L.enzo_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp]
        L.enzo_mlp_features.argtypes = [vp] * 6 + [ctypes.c_double, vp, i64, vp]
        L.enzo_mlp_train_step.argtypes = [vp, vp, vp, i32, vp, vp, i64, ctypes.c_float, vp, vp, vp, vp, vp]
        for n in ("enzo_mlp_pack", "enzo_mlp_forward", "enzo_mlp_features", "enzo_mlp_train_step"):
            getattr(L, n).restype = ctypes.c_int
        L._mlp_ready = True
    return L


def _stream_ptr(device=None):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


class MLP:
    """Learned p* guess: FP32 master weights, Adam moments and the packed BF16
    blob on one CUDA device (all tensors owned here, kernels in libenzo_ppm)."""

    def __init__(self, params=None, device="cuda", seed=0):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if params is None:
            rng = np.random.default_rng(seed)
            flat = np.zeros(MLP_PARAMS)
            flat[0:384] = rng.normal(0, np.sqrt(2 / 6), 384)
            flat[448:4544] = rng.normal(0, np.sqrt(2 / 64), 4096)
            flat[4608:4672] = rng.normal(0, np.sqrt(1 / 64), 64)
        else:
            flat = np.concatenate([np.asarray(params[k], dtype=np.float64).reshape(-1) for k in MLP_SLICES])
        self.master = torch.tensor(flat, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.grad = torch.zeros_like(self.master)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.blob = torch.zeros(MLP_BLOB_BYTES // 4, dtype=torch.float32, device=self.device)
        self.status = torch.zeros(STATUS_WORDS, dtype=torch.int64, device=self.device)
        self.step = 0
        self.pack()

    def pack(self):
        _check(_mlp_lib().enzo_mlp_pack(self.master.data_ptr(), self.blob.data_ptr(), _stream_ptr(self.device)),
               "enzo_mlp_pack")

    def params(self) -> dict:
        flat = self.master.double().cpu().numpy()
        return {k: flat[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in MLP_SLICES.items()}

    def forward(self, x):
        x = x.contiguous().float()
        y = self.torch.empty(x.shape[0], dtype=self.torch.float32, device=self.device)
        _check(_mlp_lib().enzo_mlp_forward(self.blob.data_ptr(), x.data_ptr(), y.data_ptr(), x.shape[0],
                                           self.status.data_ptr(), _stream_ptr(self.device)), "enzo_mlp_forward")
        return y

    def train_step(self, x, t, lr):
        """One Adam step (lr > 0) or a gradient-only pass (lr = 0); returns the loss tensor."""
        x = x.contiguous().float()
        t = t.contiguous().float()
        if lr > 0:
            self.step += 1
        _check(_mlp_lib().enzo_mlp_train_step(self.master.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                              max(self.step, 1), x.data_ptr(), t.data_ptr(), x.shape[0], lr,
                                              self.grad.data_ptr(), self.loss.data_ptr(), self.blob.data_ptr(),
                                              self.status.data_ptr(), _stream_ptr(self.device)),
               "enzo_mlp_train_step")
        return self.loss

    def grads(self) -> dict:
        flat = self.grad.double().cpu().numpy()
        return {k: flat[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in MLP_SLICES.items()}


def mlp_features(rl, ul, pl, rr, ur, pr, gamma):
    import torch
    ins = [t.contiguous().float() for t in (rl, ul, pl, rr, ur, pr)]
    n = ins[0].numel()
    x = torch.empty((n, 6), dtype=torch.float32, device=ins[0].device)
    _check(_mlp_lib().enzo_mlp_features(*[t.data_ptr() for t in ins], float(gamma), x.data_ptr(), n,
                                        _stream_ptr(ins[0].device)), "enzo_mlp_features")
    return x


PROBE_DFMA, PROBE_DADD, PROBE_DMUL, PROBE_DSQRT, PROBE_DDIV = 0, 1, 2, 3, 4
PROBE_BLOCKS_PER_SM = 4


def probe_fp64(op: int, n: int, sink, stream=None) -> int:
    """Launch the FP64-pipe throughput probe (enzo_probe_fp64) on `stream`;
    returns the number of operations launched.  sink: a float64 CUDA tensor of
    at least PROBE_BLOCKS_PER_SM x SMs + 1 elements.  The caller times it."""
    L = lib()
    if not getattr(L, "_probe_ready", False):
        L.enzo_probe_fp64.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
        L.enzo_probe_fp64.restype = ctypes.c_int
        L._probe_ready = True
    ops = ctypes.c_int64(0)
    st = stream.cuda_stream if stream is not None else _stream_ptr(sink.device)
    _check(L.enzo_probe_fp64(op, n, sink.data_ptr(), ctypes.byref(ops), st), "enzo_probe_fp64")
    return int(ops.value)
