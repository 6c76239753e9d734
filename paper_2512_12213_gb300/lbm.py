"""Thin Python binding of the C ABI in include/lbm.h (ctypes).

The functions named ``lbm_*`` marshal arguments to the library functions of
the same name and raise :class:`LbmError` on a non-zero status; no lattice
Boltzmann arithmetic happens here.  :class:`Sim` allocates the caller-owned
device buffers with PyTorch and passes torch's current CUDA stream.

The library is loaded on first use; if ``liblbm.so`` has not been built this
raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

D2Q9, D3Q19 = 9, 19
FORCE = {"a": 0, "b": 1, "c": 2, "d": 3, "e": 4}
STORE = {"f64": 0, "f32": 1, "f16s": 2, "bf16s": 3}
ROUND = {"nearest": 0, "stochastic": 1}
STEP_KERNEL = {"auto": 0, "register": 1, "staged": 2}
S1, S2, S3, S4 = 1, 2, 3, 4
MOVING_CORR, MAXWELL_REMOVE, ACCUMULATE = 1, 2, 4
OUT_DEVICE, OUT_HOST, OUT_HOST_ASYNC = 0, 1, 2
(BUF_POP_A, BUF_POP_B, BUF_NODE, BUF_LINKS, BUF_SCRATCH, BUF_STAGE, BUF_PHI, BUF_MAG_A, BUF_MAG_B,
 NUM_BUFFERS) = range(10)
MAX_WALLS = 16
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_UNSUPPORTED", 5: "ERR_NAN",
          6: "ERR_STATE", 7: "ERR_NOT_CONVERGED"}
ERR_ARG, ERR_NAN, ERR_NOT_CONVERGED = 1, 5, 7


class LbmError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("force_model", ctypes.c_int32),
        ("g", ctypes.c_double * 3),
        ("lorentz", ctypes.c_int32),
        ("B", ctypes.c_double * 3), ("E", ctypes.c_double * 3),
        ("sigma_e", ctypes.c_double), ("mu", ctypes.c_double),
        ("maxwell", ctypes.c_int32),
        ("les", ctypes.c_int32), ("cs", ctypes.c_double),
        ("storage", ctypes.c_int32),
        ("n_walls", ctypes.c_int32),
        ("wall_u", (ctypes.c_double * 3) * MAX_WALLS),
        ("face_wall", ctypes.c_int32 * 6),
        ("rounding", ctypes.c_int32),
        ("seed", ctypes.c_uint32),
        ("insulating", ctypes.c_int32),
        ("curved", ctypes.c_int32),
        ("stokes", ctypes.c_int32),
        ("darcy", ctypes.c_double),
        ("induced", ctypes.c_int32),
        ("eta", ctypes.c_double),
        ("mag_conducting", ctypes.c_int32),
        ("step_kernel", ctypes.c_int32),
    ]


_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_SIGS = {
    "lbm_buffer_sizes": [_P(LbmConfig), _vp, _P(ctypes.c_size_t)],
    "lbm_config_error": [],
    "lbm_create": [_P(LbmConfig), _vp, _P(_vp), _P(ctypes.c_size_t), _vp, _P(_vp)],
    "lbm_destroy": [_vp],
    "lbm_last_error": [_vp],
    "lbm_link_count": [_vp, _i, _P(ctypes.c_int64)],
    "lbm_set_body_force": [_vp, _P(_d)],
    "lbm_set_wall_velocity": [_vp, _i, _P(_d)],
    "lbm_init_equilibrium": [_vp, _vp, _vp, _vp, _i, _vp],
    "lbm_import_f": [_vp, _vp, _i, _i, _vp],
    "lbm_export_f": [_vp, _vp, _i, _i, _vp],
    "lbm_step": [_vp, _i, _vp],
    "lbm_step_from": [_vp, _vp, _vp, ctypes.c_int64, _vp],
    "lbm_save_state": [_vp, _vp, _vp],
    "lbm_load_state": [_vp, _vp, ctypes.c_int64, _vp],
    "lbm_time": [_vp, _P(ctypes.c_int64)],
    "lbm_step_kernel": [_vp, _P(ctypes.c_int32)],
    "lbm_electric_field": [_vp, _P(ctypes.c_double), _vp],
    "lbm_set_wall_distance": [_vp, _P(ctypes.c_float), _vp],
    "lbm_export_field": [_vp, _vp, _i, _vp],
    "lbm_device_status": [_vp, _P(ctypes.c_uint32), _i, _vp],
    "lbm_stress": [_vp, _i, _vp, _vp, _vp, _vp, _vp],
    "lbm_wall_force": [_vp, _i, ctypes.c_uint, _d, _vp, _i, _vp],
    "lbm_wall_force_noalloc": [_vp, _i, ctypes.c_uint, _d, _vp, _i, _vp],
    "lbm_step_force": [_vp, _i, ctypes.c_uint, _d, _vp, _i, _vp],
    "lbm_balance": [_vp, _vp, _i, _vp],
    "lbm_residual": [_vp, _vp, _i, _vp, _i, _vp],
    "lbm_run_steady": [_vp, _i, _d, ctypes.c_int64, _vp, _P(_d), _P(ctypes.c_int64), _vp],
    "lbm_adjoint_buffer_bytes": [_vp, _P(ctypes.c_size_t)],
    "lbm_adjoint_reset": [_vp, _vp],
    "lbm_adjoint_step": [_vp, _vp, _vp, _vp, _i, _P(_d), _d, _vp],
    "lbm_adjoint_gradient": [_vp, _vp, _i, _vp],
}
EXPORTED = tuple(_SIGS)


def load():
    """Load liblbm.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2512_12213_gb300.build.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name in ("lbm_config_error", "lbm_last_error") else ctypes.c_int
        _lib = lib
    return _lib


def _check(status, ctx=None):
    if status != 0:
        lib = load()
        msg = (lib.lbm_last_error(ctx) if ctx else lib.lbm_config_error()) or b""
        raise LbmError(status, msg.decode())


def make_config(lattice=9, nx=4, ny=4, nz=1, periodic=(1, 1, 1), dx=1.0, dt=1.0, tau=0.8, rho0=1.0,
                force_model="e", g=(0.0, 0.0, 0.0), lorentz=0, B=(0.0, 0.0, 0.0), E=(0.0, 0.0, 0.0),
                sigma_e=0.0, mu=1.0, maxwell=0, les=0, cs=0.1, storage="f64", wall_u=(),
                face_wall=(1, 1, 1, 1, 1, 1), rounding="nearest", seed=0, insulating=0, curved=0,
                stokes=0, darcy=0.0, induced=0, eta=0.0, mag_conducting=0, step_kernel="auto",
                **_ignored) -> LbmConfig:
    c = LbmConfig()
    c.lattice, c.nx, c.ny, c.nz = int(lattice), int(nx), int(ny), int(nz)
    for k in range(3):
        c.periodic[k] = int(periodic[k])
        c.g[k], c.B[k], c.E[k] = float(g[k]), float(B[k]), float(E[k])
    c.dx, c.dt, c.tau, c.rho0 = float(dx), float(dt), float(tau), float(rho0)
    c.force_model = FORCE[force_model] if isinstance(force_model, str) else int(force_model)
    c.lorentz, c.sigma_e, c.mu = int(lorentz), float(sigma_e), float(mu)
    c.maxwell, c.les, c.cs = int(maxwell), int(les), float(cs)
    c.storage = STORE[storage] if isinstance(storage, str) else int(storage)
    c.n_walls = len(wall_u)
    for i, u in enumerate(wall_u):
        for k in range(3):
            c.wall_u[i][k] = float(u[k])
    for k in range(6):
        c.face_wall[k] = int(face_wall[k])
    c.rounding = ROUND[rounding] if isinstance(rounding, str) else int(rounding)
    c.seed = int(seed) & 0xFFFFFFFF
    c.insulating = int(insulating)
    c.curved = int(curved)
    c.stokes, c.darcy = int(stokes), float(darcy)
    c.induced, c.eta, c.mag_conducting = int(induced), float(eta), int(mag_conducting)
    c.step_kernel = STEP_KERNEL[step_kernel] if isinstance(step_kernel, str) else int(step_kernel)
    return c


def _ptr(x):
    """Address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ------------------------------------------------------------ the C ABI
def lbm_buffer_sizes(cfg: LbmConfig, wall_id: np.ndarray):
    w = np.ascontiguousarray(wall_id, dtype=np.uint8)
    sizes = (ctypes.c_size_t * NUM_BUFFERS)()
    _check(load().lbm_buffer_sizes(ctypes.byref(cfg), w.ctypes.data, sizes))
    return list(sizes)


def lbm_create(cfg, wall_id, buffers, sizes, stream):
    w = np.ascontiguousarray(wall_id, dtype=np.uint8)
    bufs = (_vp * NUM_BUFFERS)(*[_ptr(b) for b in buffers])
    szs = (ctypes.c_size_t * NUM_BUFFERS)(*sizes)
    h = _vp()
    _check(load().lbm_create(ctypes.byref(cfg), w.ctypes.data, bufs, szs, stream, ctypes.byref(h)))
    return h


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


def lbm_last_error(ctx):
    return load().lbm_last_error(ctx).decode()


def lbm_link_count(ctx, wall=-1):
    n = ctypes.c_int64()
    _check(load().lbm_link_count(ctx, int(wall), ctypes.byref(n)), ctx)
    return n.value


def lbm_set_body_force(ctx, g):
    _check(load().lbm_set_body_force(ctx, (_d * 3)(*[float(v) for v in g])), ctx)


def lbm_set_wall_velocity(ctx, wall, u):
    _check(load().lbm_set_wall_velocity(ctx, int(wall), (_d * 3)(*[float(v) for v in u])), ctx)


def lbm_init_equilibrium(ctx, rho, u, xi, on_host, stream):
    _check(load().lbm_init_equilibrium(ctx, _ptr(rho), _ptr(u), _ptr(xi), int(on_host), stream), ctx)


def lbm_import_f(ctx, src, dtype, on_host, stream):
    _check(load().lbm_import_f(ctx, _ptr(src), int(dtype), int(on_host), stream), ctx)


def lbm_export_f(ctx, dst, dtype, on_host, stream):
    _check(load().lbm_export_f(ctx, _ptr(dst), int(dtype), int(on_host), stream), ctx)


def lbm_step(ctx, nsteps, stream):
    _check(load().lbm_step(ctx, int(nsteps), stream), ctx)


def lbm_step_from(ctx, src, dst, t, stream):
    _check(load().lbm_step_from(ctx, _ptr(src), _ptr(dst), int(t), stream), ctx)


def lbm_save_state(ctx, dst, stream):
    _check(load().lbm_save_state(ctx, _ptr(dst), stream), ctx)


def lbm_load_state(ctx, src, t, stream):
    _check(load().lbm_load_state(ctx, _ptr(src), int(t), stream), ctx)


def lbm_time(ctx):
    t = ctypes.c_int64()
    _check(load().lbm_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def lbm_step_kernel(ctx):
    """'staged' or 'register': the kernel that runs this context's step."""
    k = ctypes.c_int32()
    _check(load().lbm_step_kernel(ctx, ctypes.byref(k)), ctx)
    return {1: "register", 2: "staged"}[k.value]


def lbm_set_wall_distance(ctx, phi, stream):
    """Signed wall distance of a curved-wall context (canonical node order,
    float32 host array), or None for halfway bounce-back everywhere."""
    if phi is None:
        _check(load().lbm_set_wall_distance(ctx, None, stream), ctx)
        return
    a = np.ascontiguousarray(phi, dtype=np.float32)
    _check(load().lbm_set_wall_distance(ctx, a.ctypes.data_as(_P(ctypes.c_float)), stream), ctx)


def lbm_electric_field(ctx, stream):
    """The field the next step uses (insulating walls: set by the last step)."""
    E = (ctypes.c_double * 3)()
    _check(load().lbm_electric_field(ctx, E, stream), ctx)
    return np.array(list(E))


def lbm_export_field(ctx, B, on_host, stream):
    """The induced field B(x, T) into B[3][N] doubles (device tensor or host array)."""
    _check(load().lbm_export_field(ctx, _ptr(B), int(on_host), stream), ctx)


def lbm_device_status(ctx, clear, stream):
    f = ctypes.c_uint32()
    _check(load().lbm_device_status(ctx, ctypes.byref(f), int(clear), stream), ctx)
    return f.value


def lbm_stress(ctx, variant, sigma, S, rho, v, stream):
    _check(load().lbm_stress(ctx, int(variant), _ptr(sigma), _ptr(S), _ptr(rho), _ptr(v), stream), ctx)


def lbm_wall_force(ctx, wall, flags, weight, out, out_on_host, stream):
    _check(load().lbm_wall_force(ctx, int(wall), int(flags), float(weight), _ptr(out), int(out_on_host), stream),
           ctx)


def lbm_wall_force_noalloc(ctx, wall, flags, weight, out, out_on_host, stream):
    """lbm_wall_force without device memory from the caller (static library
    scratch; at most 1,048,576 links per call; overlapping calls race)."""
    _check(load().lbm_wall_force_noalloc(ctx, int(wall), int(flags), float(weight), _ptr(out),
                                         int(out_on_host), stream), ctx)


def lbm_step_force(ctx, wall, flags, weight, out, out_on_host, stream):
    """One step with the wall force of the step before it fused in."""
    _check(load().lbm_step_force(ctx, int(wall), int(flags), float(weight), _ptr(out), int(out_on_host), stream),
           ctx)


def lbm_balance(ctx, out, out_on_host, stream):
    _check(load().lbm_balance(ctx, _ptr(out), int(out_on_host), stream), ctx)


def lbm_residual(ctx, v_ref, update, out, out_on_host, stream):
    _check(load().lbm_residual(ctx, _ptr(v_ref), int(update), _ptr(out), int(out_on_host), stream), ctx)


def lbm_run_steady(ctx, every, tol, max_steps, v_ref, stream):
    """Returns (residual, steps taken); raises LbmError (status
    ERR_NOT_CONVERGED) when max_steps is reached first."""
    r = ctypes.c_double(-1.0)
    n = ctypes.c_int64(0)
    st = load().lbm_run_steady(ctx, int(every), float(tol), int(max_steps), _ptr(v_ref), ctypes.byref(r),
                               ctypes.byref(n), stream)
    _check(st, ctx)
    return r.value, n.value


def lbm_adjoint_buffer_bytes(ctx):
    n = ctypes.c_size_t()
    _check(load().lbm_adjoint_buffer_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def lbm_adjoint_reset(ctx, stream):
    _check(load().lbm_adjoint_reset(ctx, stream), ctx)


def lbm_adjoint_step(ctx, state_prev, phi_next, phi_out, wall, direction, seed_weight, stream):
    _check(load().lbm_adjoint_step(ctx, _ptr(state_prev), _ptr(phi_next), _ptr(phi_out), int(wall),
                                   (_d * 3)(*[float(v) for v in direction]), float(seed_weight), stream), ctx)


def lbm_adjoint_gradient(ctx, out, out_on_host, stream):
    _check(load().lbm_adjoint_gradient(ctx, _ptr(out), int(out_on_host), stream), ctx)


# ------------------------------------------------------------ convenience
class Sim:
    """A context with its buffers allocated as torch uint8 tensors on `device`.

    ``cfg`` is an :class:`LbmConfig` or a dict for :func:`make_config`;
    ``wall_id`` a uint8 array (nz, ny, nx).  All methods run on torch's
    current stream of that device.
    """

    def __init__(self, cfg, wall_id, device="cuda", stage=True):
        import torch
        self.torch = torch
        self.cfg = cfg if isinstance(cfg, LbmConfig) else make_config(**cfg)
        self.device = torch.device(device)
        self.wall_id = np.ascontiguousarray(wall_id, dtype=np.uint8)
        self.sizes = lbm_buffer_sizes(self.cfg, self.wall_id)
        if not stage:
            self.sizes[BUF_STAGE] = 0
        self.buffers = [torch.empty(max(s, 1), dtype=torch.uint8, device=self.device) if s else None
                        for s in self.sizes]
        self.ctx = None
        self.ctx = lbm_create(self.cfg, self.wall_id, self.buffers, self.sizes, self.stream)
        self.Q = self.cfg.lattice
        self.shape = (self.cfg.nz, self.cfg.ny, self.cfg.nx)
        self.N = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.rdtype = torch.float64 if self.cfg.storage == 0 else torch.float32
        self.ncomp = 3 if self.Q == 9 else 6

    @property
    def stream(self):
        with self.torch.cuda.device(self.device):
            return self.torch.cuda.current_stream().cuda_stream

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state
    def init_equilibrium(self, rho, u, xi=None):
        """rho (nz,ny,nx), u (3,nz,ny,nx), xi (Q,nz,ny,nx) or None; numpy (host) or torch float64."""
        if isinstance(rho, np.ndarray):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in (rho, u, xi)]
            lbm_init_equilibrium(self.ctx, arrs[0], arrs[1], arrs[2], 1, self.stream)
        else:
            arrs = [a.to(self.device, self.torch.float64).contiguous() if a is not None else None
                    for a in (rho, u, xi)]
            lbm_init_equilibrium(self.ctx, arrs[0], arrs[1], arrs[2], 0, self.stream)
            self._keep = arrs

    def rest(self):
        rho = np.full(self.shape, self.cfg.rho0)
        self.init_equilibrium(rho, np.zeros((3,) + self.shape))

    def import_f(self, f):
        if isinstance(f, np.ndarray):
            a = np.ascontiguousarray(f, dtype=np.float64)
            lbm_import_f(self.ctx, a, 0, 1, self.stream)
        else:
            a = f.contiguous()
            lbm_import_f(self.ctx, a, 0 if a.dtype == self.torch.float64 else 1, 0, self.stream)
            self._keep = [a]

    def export_f(self, dtype=None):
        t = self.torch
        dtype = dtype or t.float64
        out = t.empty((self.Q,) + self.shape, dtype=dtype, device=self.device)
        lbm_export_f(self.ctx, out, 0 if dtype == t.float64 else 1, 0, self.stream)
        return out

    def step(self, n=1):
        lbm_step(self.ctx, n, self.stream)

    @property
    def step_kernel(self):
        return lbm_step_kernel(self.ctx)

    @property
    def time(self):
        return lbm_time(self.ctx)

    def device_status(self, clear=True):
        return lbm_device_status(self.ctx, clear, self.stream)

    def electric_field(self):
        return lbm_electric_field(self.ctx, self.stream)

    def set_wall_distance(self, phi):
        lbm_set_wall_distance(self.ctx, phi, self.stream)

    def export_field(self):
        """The induced field B(x, T), (3, nz, ny, nx) float64 on the device."""
        B = self.torch.empty((3,) + self.shape, dtype=self.torch.float64, device=self.device)
        lbm_export_field(self.ctx, B, 0, self.stream)
        return B

    # diagnostics
    def stress(self, variant):
        t = self.torch
        sig = t.empty((self.ncomp,) + self.shape, dtype=self.rdtype, device=self.device)
        S = t.empty_like(sig)
        rho = t.empty(self.shape, dtype=self.rdtype, device=self.device)
        v = t.empty((3,) + self.shape, dtype=self.rdtype, device=self.device)
        lbm_stress(self.ctx, variant, sig, S, rho, v, self.stream)
        return sig, S, rho, v

    def wall_force(self, wall=-1, flags=0):
        out = np.zeros(3)
        lbm_wall_force(self.ctx, wall, flags, 1.0, out, 1, self.stream)
        return out

    def balance(self):
        out = np.zeros(7)
        lbm_balance(self.ctx, out, 1, self.stream)
        return out[0], out[1:4].copy(), out[4:7].copy()

    def velocity_buffer(self):
        """A zeroed device array for the residual's reference velocity, (3, nz, ny, nx) float64."""
        return self.torch.zeros((3,) + self.shape, dtype=self.torch.float64, device=self.device)

    def residual(self, v_ref, update=True):
        """(sum |v - v_ref|, sum |v|, r) of the current state; updates v_ref."""
        out = np.zeros(3)
        lbm_residual(self.ctx, v_ref, update, out, OUT_HOST, self.stream)
        return float(out[0]), float(out[1]), float(out[2])

    def run_steady(self, every, tol, max_steps, v_ref=None):
        v = self.velocity_buffer() if v_ref is None else v_ref
        return lbm_run_steady(self.ctx, every, tol, max_steps, v, self.stream)

    def link_count(self, wall=-1):
        return lbm_link_count(self.ctx, wall)
