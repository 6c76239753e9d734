"""ctypes wrapper of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle restates the lattice Boltzmann method of
arXiv 2512.12213 (Sec. 2: Eqs. 1-5 and 10; Sec. 3: Eqs. 8-9; Sec. 5: Eqs. 25-30;
Sec. 6: Eq. 32) in plain double precision, node by node.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this module; the
CUDA library never does, and this module imports nothing from it.

Arrays use numpy: populations are shaped ``(Q, nz, ny, nx)`` (C order), which
is the canonical interchange layout ``f[a][z][y][x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "lbm_oracle.c"), os.path.join(_HERE, "oracle_node.inc"),
        os.path.join(_HERE, "lbm_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_OMP_PATH = os.path.join(_HERE, "liblbm_oracle_omp.so")

MAX_WALLS = 16
FORCE = {"a": 0, "b": 1, "c": 2, "d": 3, "e": 4}
MOVING_CORR = 1
MAXWELL_REMOVE = 2


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction).  The
    parity build is single threaded; omp=True builds the timing copy, the
    same source with OpenMP over the independent node loops of a step (the
    per-node arithmetic, and so every result, is the same)."""
    path = _OMP_PATH if omp else _LIB_PATH
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
        tmp = path + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-Wl,-Bsymbolic", *(["-fopenmp"] if omp else []),
                        "-o", tmp, _SRC[0], "-lm"], check=True)
        os.replace(tmp, path)
    return path


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("force_model", ctypes.c_int),
        ("g", ctypes.c_double * 3),
        ("lorentz", ctypes.c_int),
        ("B", ctypes.c_double * 3), ("E", ctypes.c_double * 3),
        ("sigma_e", ctypes.c_double), ("mu", ctypes.c_double),
        ("maxwell", ctypes.c_int),
        ("les", ctypes.c_int), ("cs", ctypes.c_double),
        ("n_walls", ctypes.c_int),
        ("wall_u", (ctypes.c_double * 3) * MAX_WALLS),
        ("face_wall", ctypes.c_int * 6),
        ("phi", ctypes.c_void_p),
        ("insulating", ctypes.c_int),
        ("stokes", ctypes.c_int),
        ("darcy", ctypes.c_double),
        ("induced", ctypes.c_int),
        ("eta", ctypes.c_double),
        ("mag_conducting", ctypes.c_int),
        ("Bfield", ctypes.c_void_p),
    ]


_libs = {}


def lib(omp: bool = False):
    """The parity build (default) or the OpenMP timing build of the oracle."""
    _lib = _libs.get(omp)
    if _lib is None:
        _lib = _libs[omp] = ctypes.CDLL(build(omp=omp))
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        ub = P(ctypes.c_ubyte)
        cp = P(OrcCfg)
        sig = {
            "orc_threads": (ctypes.c_int, []),
            "orc_lattice": (ctypes.c_int, [ctypes.c_int, P(ctypes.c_int), dp, P(ctypes.c_int)]),
            "orc_feq": (None, [cp, d, dp, dp]),
            "orc_node_macro": (None, [cp, dp, dp]),
            "orc_force_term": (None, [cp, dp, dp]),
            "orc_collide_node": (None, [cp, dp, dp]),
            "orc_init": (None, [cp, ub, dp, dp, dp, dp]),
            "orc_step": (None, [cp, ub, dp, dp]),
            "orc_run": (None, [cp, ub, dp, ctypes.c_int]),
            "orc_step_e": (None, [cp, ub, dp, dp, dp]),
            "orc_run_e": (None, [cp, ub, dp, ctypes.c_int, dp]),
            "orc_mag_q": (ctypes.c_int, [ctypes.c_int]),
            "orc_mag_init": (None, [cp, ub, dp]),
            "orc_mag_field": (None, [cp, ub, dp, dp]),
            "orc_run_mhd": (None, [cp, ub, dp, dp, ctypes.c_int, dp]),
            "orc_wall_force": (None, [cp, ub, dp, dp, ctypes.c_int, ctypes.c_int, dp]),
            "orc_count_links": (ctypes.c_long, [cp, ub, ctypes.c_int]),
            "orc_stress": (None, [cp, ub, dp, dp, dp, ctypes.c_int, dp, dp, dp, dp]),
            "orc_balance": (None, [cp, ub, dp, dp]),
            "orc_residual": (None, [cp, ub, dp, dp, dp, dp]),
            "orc_adjoint_drag": (ctypes.c_int, [cp, ub, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]),
            "orc_drag_average": (d, [cp, ub, dp, ctypes.c_int, ctypes.c_int, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def make_cfg(q=9, nx=4, ny=4, nz=1, periodic=(1, 1, 1), dx=1.0, dt=1.0, tau=0.8, rho0=1.0,
             force_model="e", g=(0.0, 0.0, 0.0), lorentz=0, B=(0.0, 0.0, 0.0), E=(0.0, 0.0, 0.0),
             sigma_e=0.0, mu=1.0, maxwell=0, les=0, cs=0.1, wall_u=(), face_wall=(1, 1, 1, 1, 1, 1),
             insulating=0, phi=None, stokes=0, darcy=0.0, induced=0, eta=0.0, mag_conducting=0,
             **_ignored) -> OrcCfg:
    """Build an oracle configuration.  ``wall_u`` lists the velocity of walls
    1..n; ``force_model`` is one of 'a'..'e' (Sec. 2)."""
    c = OrcCfg()
    c.q, c.nx, c.ny, c.nz = q, nx, ny, nz
    for k in range(3):
        c.periodic[k] = int(periodic[k])
        c.g[k] = float(g[k])
        c.B[k] = float(B[k])
        c.E[k] = float(E[k])
    c.dx, c.dt, c.tau, c.rho0 = float(dx), float(dt), float(tau), float(rho0)
    c.force_model = FORCE[force_model] if isinstance(force_model, str) else int(force_model)
    c.lorentz, c.sigma_e, c.mu = int(lorentz), float(sigma_e), float(mu)
    c.maxwell, c.les, c.cs = int(maxwell), int(les), float(cs)
    c.n_walls = len(wall_u)
    for i, u in enumerate(wall_u):
        for k in range(3):
            c.wall_u[i][k] = float(u[k])
    for k in range(6):
        c.face_wall[k] = int(face_wall[k])
    c.insulating = int(insulating)
    c.stokes, c.darcy = int(stokes), float(darcy)
    c.induced, c.eta, c.mag_conducting = int(induced), float(eta), int(mag_conducting)
    if phi is not None:
        # signed wall distance per node (float32, the library's precision too)
        c._phi = np.ascontiguousarray(phi, dtype=np.float32)
        c.phi = c._phi.ctypes.data
    return c


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ub(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def threads(omp=False):
    """Threads of a step's node loops in the parity (1) or timing build."""
    return int(lib(omp).orc_threads())


def lattice(q):
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    lib().orc_lattice(q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                      opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e, w, opp


def feq(cfg, rho, u):
    out = np.zeros(cfg.q)
    lib().orc_feq(ctypes.byref(cfg), float(rho), _dp(_f64(u)), _dp(out))
    return out


def node_macro(cfg, f):
    out = np.zeros(18)
    lib().orc_node_macro(ctypes.byref(cfg), _dp(_f64(f)), _dp(out))
    return {"rho": out[0], "u": out[1:4], "v": out[4:7], "a": out[7:10], "ueq": out[10:13],
            "uF": out[13:16], "C": out[16], "tau": out[17]}


def force_term(cfg, f):
    out = np.zeros(cfg.q)
    lib().orc_force_term(ctypes.byref(cfg), _dp(_f64(f)), _dp(out))
    return out


def collide_node(cfg, f):
    out = np.zeros(cfg.q)
    lib().orc_collide_node(ctypes.byref(cfg), _dp(_f64(f)), _dp(out))
    return out


def shape(cfg):
    return (cfg.q, cfg.nz, cfg.ny, cfg.nx)


def init(cfg, wall_id, rho, u, xi=None):
    """f = f^eq(rho, u) (1 + xi) at fluid nodes; rho (nz,ny,nx), u (3,nz,ny,nx)."""
    f = np.zeros(shape(cfg))
    xi_a = _f64(xi) if xi is not None else None
    rho_a, u_a, w_a = _f64(rho), _f64(u), _u8(wall_id)
    lib().orc_init(ctypes.byref(cfg), _ub(w_a), _dp(rho_a), _dp(u_a),
                   _dp(xi_a) if xi_a is not None else None, _dp(f))
    return f


def step(cfg, wall_id, f):
    """One step of Eq. (2); returns (f(t+dt), f^rel(t))."""
    fn = _f64(f).copy()
    frel = np.zeros_like(fn)
    lib().orc_step(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(fn), _dp(frel))
    return fn, frel


def run(cfg, wall_id, f, n, omp=False):
    """n steps; omp=True runs the OpenMP timing build (same results)."""
    fn = _f64(f).copy()
    lib(omp).orc_run(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(fn), int(n))
    return fn


def run_e(cfg, wall_id, f, n, E=None):
    """n steps with the field E as state (insulating walls update it each
    step, Eq. 36); returns (f, E of the next step)."""
    fn = _f64(f).copy()
    e = np.array(list(cfg.E) if E is None else E, dtype=np.float64)
    lib().orc_run_e(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(fn), int(n), _dp(e))
    return fn, e


def mag_init(cfg, wall_id):
    """Field distributions at rest in the external field, g[3][Qm][N]."""
    qm = lib().orc_mag_q(cfg.q)
    g = np.zeros((3, qm, cfg.nz, cfg.ny, cfg.nx))
    lib().orc_mag_init(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(g))
    return g


def mag_field(cfg, wall_id, g):
    B = np.zeros((3, cfg.nz, cfg.ny, cfg.nx))
    lib().orc_mag_field(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(g)), _dp(B))
    return B


def run_mhd(cfg, wall_id, f, g, n):
    """n coupled fluid / induced-field steps; returns (f, g, f^rel of the last step)."""
    fn, gn = _f64(f).copy(), _f64(g).copy()
    fr = np.zeros_like(fn)
    lib().orc_run_mhd(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(fn), _dp(gn), int(n), _dp(fr))
    return fn, gn, fr


def with_field(cfg, B):
    """A copy of cfg whose stress and wall force use the local field B[3][N]."""
    c = OrcCfg.from_buffer_copy(cfg)
    for k in ("_phi",):
        if hasattr(cfg, k):
            setattr(c, k, getattr(cfg, k))
    c._B = np.ascontiguousarray(B, dtype=np.float64)
    c.Bfield = c._B.ctypes.data
    return c


def step_e(cfg, wall_id, f, E=None):
    """One step with the field E as state; returns (f(t+dt), f^rel(t), E of
    the next step)."""
    fn = _f64(f).copy()
    frel = np.zeros_like(fn)
    e = np.array(list(cfg.E) if E is None else E, dtype=np.float64)
    lib().orc_step_e(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(fn), _dp(frel), _dp(e))
    return fn, frel, e


def wall_force(cfg, wall_id, frel, fnext, wall=-1, flags=0):
    out = np.zeros(3)
    lib().orc_wall_force(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(frel)), _dp(_f64(fnext)),
                         int(wall), int(flags), _dp(out))
    return out


def count_links(cfg, wall_id, wall=-1):
    return int(lib().orc_count_links(ctypes.byref(cfg), _ub(_u8(wall_id)), int(wall)))


def stress(cfg, wall_id, f, frel, fnext, variant):
    """Returns sigma (ncomp, nz, ny, nx), S, rho (nz,ny,nx), v (3, nz, ny, nx)."""
    N = cfg.nx * cfg.ny * cfg.nz
    nc = 6 if cfg.q == 19 else 3
    sig = np.zeros((nc, cfg.nz, cfg.ny, cfg.nx))
    S = np.zeros_like(sig)
    rho = np.zeros((cfg.nz, cfg.ny, cfg.nx))
    v = np.zeros((3, cfg.nz, cfg.ny, cfg.nx))
    f = _f64(f)
    frel = _f64(frel if frel is not None else f)
    fnext = _f64(fnext if fnext is not None else f)
    lib().orc_stress(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(f), _dp(frel), _dp(fnext),
                     int(variant), _dp(sig), _dp(S), _dp(rho), _dp(v))
    assert sig.size == nc * N
    return sig, S, rho, v


def balance(cfg, wall_id, f):
    """(mass, momentum[3], sum rho a [3]) of the canonical state, times dx^D."""
    out = np.zeros(7)
    lib().orc_balance(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(f)), _dp(out))
    return out[0], out[1:4].copy(), out[4:7].copy()


def residual(cfg, wall_id, f, vref=None):
    """Steady-state residual of the canonical state f against the velocity
    field vref (3, nz, ny, nx) of an earlier time (None: zero).  Returns
    (sum |v - vref|, sum |v|, r, v) with v the flow velocity (3, nz, ny, nx)."""
    out = np.zeros(3)
    v = np.zeros((3, cfg.nz, cfg.ny, cfg.nx))
    vr = _f64(vref) if vref is not None else None
    lib().orc_residual(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(f)),
                       _dp(vr) if vr is not None else None, _dp(v), _dp(out))
    return float(out[0]), float(out[1]), float(out[2]), v


def adjoint_drag(cfg, wall_id, f0, T, wall, d=(1.0, 0.0, 0.0)):
    J = np.zeros(1)
    grad = np.zeros(6)
    rc = lib().orc_adjoint_drag(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(f0)), int(T),
                                int(wall), _dp(_f64(d)), _dp(J), _dp(grad))
    if rc != 0:
        raise MemoryError("oracle adjoint: allocation failed")
    return float(J[0]), grad


def drag_average(cfg, wall_id, f0, T, wall, d=(1.0, 0.0, 0.0)):
    return float(lib().orc_drag_average(ctypes.byref(cfg), _ub(_u8(wall_id)), _dp(_f64(f0)),
                                        int(T), int(wall), _dp(_f64(d))))
