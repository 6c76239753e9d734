"""Pins of the oracle's whole-lattice behaviour against closed forms and exact
identities (no GPU).

* exact discrete momentum balance of every step (the discrete form of Eq. 32):
  F_wall(t) = sum rho a - [M(t+dt) - M(t)]/dt;
* Poiseuille channel at steady state: the flow velocity is the parabola of the
  recovered Navier-Stokes equation (Eq. 7) plus the known halfway-bounce-back
  slip of BGK, (g/2nu)(16 Lambda - 3)/12 with Lambda = (tau - 1/2)^2; each wall
  carries half the body force (Eq. 33); the shear stress of Eqs. (8)-(9) is
  rho g (H - 1 - 2y)/2;
* Hartmann-Couette channel: second-order convergence to the cosh profile and
  wall shear, exact global balance with the Lorentz force included;
* moving-wall correction (Sec. 5): rho_w u_w (u_w . n) per flat wall node,
  zero on a closed body;
* Maxwell stress: with a uniform field f_B(t) = f_0(t) + Delta exactly, the
  momentum exchange contains -L n per flat wall node (Sec. 5, Eq. 28), its
  removal restores the field-free force, and it cancels on a closed body
  (Eq. 36);
* half-step consistency at steady state (Eqs. 29-30);
* insulating walls (Eq. 36): with E = -<v> x B the Hartmann profile
  converges at second order to nu u'' + g - K (u - <u>) = 0, u(+-H) = 0, and at
  steady state the total Lorentz force vanishes, so the walls carry exactly
  the body force of g (Eq. 34 with a zero Lorentz term);
* walls off the half-grid (discussion after Eq. 25, end of Sec. 6), linear
  interpolated bounce-back from a signed wall distance: q = 1/2 is halfway
  bounce-back exactly; Poiseuille between walls at arbitrary positions
  converges at second order to the parabola of the true walls (halfway
  bounce-back on the same nodes only at first order); the exact per-step
  momentum balance holds with the interpolated values (momentum exchange at
  the imaginary points).
"""
import numpy as np
import pytest

from paper_2512_12213_gb300 import inputs


def _channel_cfg(orc, H, tau, model, g, nx=2, **kw):
    base = dict(q=9, nx=nx, ny=H, nz=1, periodic=(1, 0, 1), tau=tau, force_model=model,
                g=(g, 0, 0), wall_u=((0, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    base.update(kw)
    return orc.make_cfg(**base)


def _rest(orc, cfg, mask):
    nz, ny, nx = mask.shape
    return orc.init(cfg, mask, np.full((nz, ny, nx), cfg.rho0), np.zeros((3, nz, ny, nx)))


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("model", list("abcde"))
def test_exact_momentum_balance_every_step(orc, q, model):
    """Every step, the momentum lost to walls equals the body-force impulse
    minus the change of fluid momentum, for moving walls, Lorentz force and the
    Maxwell equilibrium together, at non-unit dx and dt."""
    if q == 9:
        nx, ny, nz, per = 12, 9, 1, (1, 0, 1)
    else:
        nx, ny, nz, per = 7, 6, 5, (1, 0, 0)
    mask = inputs.random_solids(nx, ny, nz, 0.12, n_walls=2, seed=11 + q)
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=per, dx=0.5, dt=0.2, tau=0.81,
                       force_model=model, g=(3e-2, -1e-2, 5e-3), lorentz=1, B=(0.1, 0.25, -0.05),
                       E=(1e-3, 0, 2e-3), sigma_e=0.8, maxwell=1, mu=1.3,
                       wall_u=((0.01, 0.02, -0.01), (0.0, -0.015, 0.02), (0.03, 0, 0)),
                       face_wall=(3, 3, 3, 2, 1, 3))
    c = cfg.dx / cfg.dt
    D = 2 if q == 9 else 3
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, seed=5)
    f = orc.init(cfg, mask, rho, u * 0.5 * c, inputs.noise(q, nx, ny, nz, 1e-2, seed=6))
    for _ in range(4):
        _, M0, rhoa = orc.balance(cfg, mask, f)
        fn, fr = orc.step(cfg, mask, f)
        _, M1, _ = orc.balance(cfg, mask, fn)
        F = orc.wall_force(cfg, mask, fr, fn, -1, 0)
        ref = rhoa - (M1 - M0) / cfg.dt
        scale = np.abs(M0).max() / cfg.dt + np.abs(F).max()
        assert np.allclose(F, ref, rtol=0, atol=2e-14 * scale), (F, ref)
        f = fn


@pytest.mark.parametrize("model,tau", [("a", 0.8), ("b", 0.8), ("c", 0.8), ("d", 0.8),
                                       ("e", 0.8), ("e", 0.6), ("d", 1.0)])
def test_poiseuille_steady_state(orc, model, tau):
    H, g, nx = 16, 1e-6, 2
    cfg = _channel_cfg(orc, H, tau, model, g, nx=nx)
    mask = inputs.empty_mask(nx, H)
    nu = (tau - 0.5) / 3
    steps = int(40 / (nu * np.pi ** 2 / H ** 2))      # slowest mode decayed by e^-40
    f = orc.run(cfg, mask, _rest(orc, cfg, mask), steps)
    fn, fr = orc.step(cfg, mask, f)
    sig, S, rho, v = orc.stress(cfg, mask, f, fr, fn, 2)
    y = np.arange(H)
    lam = (tau - 0.5) ** 2
    v_exact = g / (2 * nu) * ((y + 0.5) * (H - 0.5 - y) + (16 * lam - 3) / 12)
    vx = v[0, 0, :, 0]
    assert np.abs(vx - v_exact).max() < 1e-9 * v_exact.max()
    assert np.abs(v[1]).max() < 1e-9 * v_exact.max()
    # shear stress sigma_xy = rho nu du/dy, linear between the walls
    sxy = sig[2, 0, :, 0]
    s_exact = rho[0, :, 0] * g * (H - 1 - 2 * y) / 2
    assert np.abs(sxy - s_exact).max() < 1e-9 * s_exact.max()
    assert np.allclose(S[2], sig[2] / (2 * rho * nu), rtol=1e-13)
    # each wall carries half of the body force (Eq. 33 and symmetry)
    mass, M, rhoa = orc.balance(cfg, mask, f)
    Fb = orc.wall_force(cfg, mask, fr, fn, 1)
    Ft = orc.wall_force(cfg, mask, fr, fn, 2)
    assert np.isclose(Fb[0], 0.5 * g * mass, rtol=1e-9)
    assert np.isclose(Ft[0], 0.5 * g * mass, rtol=1e-9)
    assert np.isclose(Fb[0] + Ft[0], rhoa[0], rtol=1e-9)


def _hartmann(orc, H, tau, Ha=10.0, Uw=0.05, B0=0.05, model="e", maxwell=0):
    nu = (tau - 0.5) / 3
    K = nu * Ha ** 2 / H ** 2
    g = 0.05 * K / (1 - 1 / np.cosh(Ha))
    ny = 2 * H
    cfg = orc.make_cfg(q=9, nx=1, ny=ny, nz=1, periodic=(1, 0, 1), tau=tau, force_model=model,
                       g=(g, 0, 0), lorentz=1, B=(0, B0, 0), sigma_e=K / B0 ** 2, maxwell=maxwell,
                       wall_u=((0, 0, 0), (Uw, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    mask = inputs.empty_mask(1, ny)
    f = orc.run(cfg, mask, _rest(orc, cfg, mask), int(36 / K))
    fn, fr = orc.step(cfg, mask, f)
    m = Ha / H
    y = np.arange(ny) - H + 0.5
    u_exact = (g / K) * (1 - np.cosh(m * y) / np.cosh(m * H)) + Uw * np.sinh(m * (y + H)) / np.sinh(2 * m * H)
    dudy = lambda yy: (g / K) * (-m * np.sinh(m * yy) / np.cosh(m * H)) + Uw * m * np.cosh(m * (yy + H)) / np.sinh(2 * m * H)
    return dict(cfg=cfg, mask=mask, f=f, fn=fn, fr=fr, u_exact=u_exact, y=y, nu=nu,
                shear=(nu * dudy(-H), -nu * dudy(H)), dudy=dudy)


def test_hartmann_couette_convergence(orc):
    """Hartmann number 10, moving top wall: velocity and wall shear converge
    at second order to nu u'' - K u + g = 0 with u(-H) = 0, u(H) = U_w; the
    sum of wall forces equals sum rho a including the Lorentz force."""
    errs, shear_b, shear_t = [], [], []
    for H in (16, 32, 64):
        r = _hartmann(orc, H, 0.8)
        cfg, mask = r["cfg"], r["mask"]
        _, _, _, v = orc.stress(cfg, mask, r["f"], r["fr"], r["fn"], 2)
        errs.append(np.abs(v[0, 0, :, 0] - r["u_exact"]).max() / np.abs(r["u_exact"]).max())
        Fb = orc.wall_force(cfg, mask, r["fr"], r["fn"], 1)
        Ft = orc.wall_force(cfg, mask, r["fr"], r["fn"], 2)
        _, _, rhoa = orc.balance(cfg, mask, r["f"])
        assert np.isclose(Fb[0] + Ft[0], rhoa[0], rtol=1e-10)
        shear_b.append(abs(Fb[0] / r["shear"][0] - 1))
        shear_t.append(abs(Ft[0] / r["shear"][1] - 1))
    assert errs[-1] < 2e-3 and errs[-2] / errs[-1] > 3.0
    for s in (shear_b, shear_t):
        assert s[-1] < 1e-3
        assert 3.8 < s[0] / s[1] < 4.2 and 3.8 < s[1] / s[2] < 4.2


@pytest.mark.parametrize("model", ["e", "d"])
def test_half_step_consistency(orc, model):
    """Eqs. (29)-(30) at steady state: the half-step stress about
    f^eq(rho-bar, u-bar) plus Theta/2 equals the full-step stress (variant 2)
    plus rho (v v - u^eq u^eq), which vanishes for Guo's model [e] where
    u^eq = v."""
    r = _hartmann(orc, 16, 0.7, model=model)
    cfg, mask = r["cfg"], r["mask"]
    s2, _, rho, v = orc.stress(cfg, mask, r["f"], r["fr"], r["fn"], 2)
    s4, _, rb, ub = orc.stress(cfg, mask, r["f"], r["fr"], r["fn"], 4)
    s3, _, _, _ = orc.stress(cfg, mask, r["f"], r["fr"], r["fn"], 3)
    vx = v[0]
    ueq = vx if model == "e" else None
    if model == "d":
        # u^eq = u = v - dt a/2 with a_x = g - K v_x (Lorentz), a_y = 0
        g = cfg.g[0]
        K = cfg.sigma_e * cfg.B[1] ** 2 / rho
        ueq = vx - 0.5 * cfg.dt * (g - K * vx)
    corr_xx = rho * (vx * vx - ueq * ueq)
    scale = np.abs(s2).max()
    assert np.allclose(rb, rho, rtol=1e-13)
    assert np.allclose(ub[0], vx, rtol=0, atol=1e-13 * np.abs(vx).max())
    assert np.allclose(s4[0], s2[0] + corr_xx, rtol=0, atol=1e-10 * scale)
    assert np.allclose(s4[1:], s2[1:], rtol=0, atol=1e-10 * scale)
    # and variant 3 differs from variant 4 by Theta/2, which is O(tau dt u a)
    assert np.abs(s4 - s3).max() < 1e-2 * scale


@pytest.mark.parametrize("q", [9, 19])
def test_moving_wall_correction(orc, q):
    """Wen's Galilean correction adds rho_w u_w (u_w . n) dx^(D-1) per flat
    wall node (it offsets the momentum flux -rho u u n contained in Eq. 25);
    tangential wall motion gets exactly zero."""
    D = 2 if q == 9 else 3
    nx, ny, nz = (6, 8, 1) if q == 9 else (4, 5, 6)
    ax = 1 if q == 9 else 2            # closed axis
    per = [1, 1, 1]
    per[ax] = 0
    fw = [3] * 6
    fw[2 * ax], fw[2 * ax + 1] = 1, 2
    ub = np.array([0.02, 0.01, 0.0])
    ut = np.array([-0.01, 0.015, 0.0]) if q == 9 else np.array([0.01, -0.02, 0.015])
    if q == 19:
        ub = np.array([0.02, -0.01, 0.03])
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=per, dx=0.5, dt=0.25, tau=0.9,
                       force_model="e", g=(1e-3, 0, 0), wall_u=(ub, ut, (0, 0, 0)), face_wall=fw)
    mask = inputs.empty_mask(nx, ny, nz)
    f = orc.init(cfg, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)),
                 inputs.noise(q, nx, ny, nz, 1e-3))
    fn, fr = orc.step(cfg, mask, f)
    n_nodes = nx * ny * nz // [nx, ny, nz][ax]
    area = cfg.dx ** (D - 1)
    for wall, uw, nsign in ((1, ub, 1.0), (2, ut, -1.0)):
        F0 = orc.wall_force(cfg, mask, fr, fn, wall, 0)
        d = orc.wall_force(cfg, mask, fr, fn, wall, orc.MOVING_CORR) - F0
        un = uw[ax] * nsign
        # tolerance: rounding of the difference of two forces of size |F0|
        assert np.allclose(d, n_nodes * area * cfg.rho0 * uw * un, rtol=0,
                           atol=1e-14 * np.abs(F0).max())
    # tangential motion only: exactly zero correction
    ut2 = ut.copy()
    ut2[ax] = 0
    cfg2 = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=per, dx=0.5, dt=0.25, tau=0.9,
                        force_model="e", wall_u=(ut2, ut2, (0, 0, 0)), face_wall=fw)
    fn, fr = orc.step(cfg2, mask, f)
    for wall in (1, 2):
        d = orc.wall_force(cfg2, mask, fr, fn, wall, orc.MOVING_CORR) - orc.wall_force(cfg2, mask, fr, fn, wall, 0)
        assert np.abs(d).max() < 1e-15


@pytest.mark.parametrize("q", [9, 19])
def test_closed_body_corrections_cancel(orc, q):
    """On a closed staircase body with uniform wall velocity the moving-wall
    correction sums to zero, and the Maxwell part of the momentum exchange
    cancels (the discrete form of Eq. 36)."""
    if q == 9:
        nx, ny, nz = 16, 12, 1
        mask = inputs.cylinder_mask(nx, ny, (7.3, 5.6), 3.2)
        B = (0.1, 0.2, 0.0)
    else:
        nx, ny, nz = 10, 9, 8
        mask = inputs.sphere_mask(nx, ny, nz, (4.5, 4.2, 3.7), 2.6)
        B = (0.1, 0.2, -0.15)
    uw = (0.02, -0.01, 0.015 if q == 19 else 0.0)
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.75, force_model="d",
                       g=(1e-4, 0, 0), maxwell=1, B=B, wall_u=(uw,))
    f = _rest(orc, cfg, mask)
    f = orc.run(cfg, mask, f, 3)
    fn, fr = orc.step(cfg, mask, f)
    F0 = orc.wall_force(cfg, mask, fr, fn, 1, 0)
    Fm = orc.wall_force(cfg, mask, fr, fn, 1, orc.MOVING_CORR)
    Fx = orc.wall_force(cfg, mask, fr, fn, 1, orc.MAXWELL_REMOVE)
    nl = orc.count_links(cfg, mask, 1)
    assert nl > 0
    # tolerance: rounding of a sum of nl link terms of size ~ rho0 c dx^D / dt
    tol = 1e-15 * nl * cfg.rho0 * (cfg.dx / cfg.dt) * cfg.dx ** (2 if q == 9 else 3) / cfg.dt
    assert np.abs(Fm - F0).max() < tol
    assert np.abs(Fx - F0).max() < tol


@pytest.mark.parametrize("q", [9, 19])
def test_maxwell_equilibrium_shift_and_removal(orc, q):
    """With a uniform B, the Maxwell term Delta of Eq. (10) has zero zeroth and
    first moments and is even in e, so f_B(t) = f_0(t) + Delta exactly; the
    momentum exchange then contains -L n per flat wall node, and the Maxwell
    removal gives back the field-free force."""
    D = 2 if q == 9 else 3
    nx, ny, nz = (6, 8, 1) if q == 9 else (4, 5, 6)
    ax = 1 if q == 9 else 2
    per = [1, 1, 1]
    per[ax] = 0
    fw = [3] * 6
    fw[2 * ax], fw[2 * ax + 1] = 1, 2
    B = np.array([0.07, -0.12, 0.05 if q == 19 else 0.0])
    kw = dict(q=q, nx=nx, ny=ny, nz=nz, periodic=per, dx=0.5, dt=0.25, tau=0.9, force_model="b",
              g=(2e-3, 0, 0), B=B, mu=0.8, wall_u=((0.01, 0, 0), (0, 0, 0), (0, 0, 0)), face_wall=fw)
    c0 = orc.make_cfg(maxwell=0, **kw)
    cB = orc.make_cfg(maxwell=1, **kw)
    mask = inputs.empty_mask(nx, ny, nz)
    f0 = orc.init(c0, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)),
                  inputs.noise(q, nx, ny, nz, 1e-3))
    delta = orc.feq(cB, 1.0, np.zeros(3)) - orc.feq(c0, 1.0, np.zeros(3))
    fB = f0 + delta[:, None, None, None]
    for _ in range(5):
        f0n, f0r = orc.step(c0, mask, f0)
        fBn, fBr = orc.step(cB, mask, fB)
        assert np.allclose(fBn - f0n, delta[:, None, None, None], rtol=0, atol=1e-15)
        d = np.diag([1.0] * D + [0.0] * (3 - D))
        L = (B @ B * d / 2 - np.outer(B, B)) / cB.mu
        n_nodes = nx * ny * nz // [nx, ny, nz][ax]
        area = cB.dx ** (D - 1)
        for wall, nsign in ((1, 1.0), (2, -1.0)):
            n = np.zeros(3)
            n[ax] = nsign
            P0 = orc.wall_force(c0, mask, f0r, f0n, wall, 0)
            PB = orc.wall_force(cB, mask, fBr, fBn, wall, 0)
            PR = orc.wall_force(cB, mask, fBr, fBn, wall, orc.MAXWELL_REMOVE)
            # tolerance: rounding relative to the wall's pressure force |P0|
            tol = 1e-14 * np.abs(P0).max()
            assert np.allclose(PB - P0, -n_nodes * area * (L @ n), rtol=0, atol=tol)
            assert np.allclose(PR, P0, rtol=0, atol=tol)
        f0, fB = f0n, fBn


def _insulating(orc, H, tau=0.8, Ha=4.0, nx=2):
    ny = 2 * H
    nu = (tau - 0.5) / 3
    K = nu * Ha ** 2 / H ** 2
    B0 = 0.05
    m = Ha / H
    g = 1e-5 * (16.0 / H) ** 2
    kw = dict(q=9, nx=nx, ny=ny, nz=1, periodic=(1, 0, 1), tau=tau, force_model="e", g=(g, 0, 0),
              lorentz=1, B=(0, B0, 0), sigma_e=K / B0 ** 2, insulating=1, wall_u=((0, 0, 0),))
    cfg = orc.make_cfg(**kw)
    mask = np.zeros((1, ny, nx), np.uint8)
    f0 = orc.init(cfg, mask, np.ones((1, ny, nx)), np.zeros((3, 1, ny, nx)))
    f, E = orc.run_e(cfg, mask, f0, int(60 * H * H))
    y = np.arange(ny) - H + 0.5
    # nu u'' + g - K (u - <u>) = 0 with u(+-H) = 0:
    # u = (g/K) mH coth(mH) (1 - cosh(m y)/cosh(m H)), m = Ha/H
    u_exact = (g / K) * m * H / np.tanh(m * H) * (1 - np.cosh(m * y) / np.cosh(m * H))
    return dict(cfg=orc.make_cfg(**dict(kw, E=tuple(E))), kw=kw, mask=mask, f=f, E=E, u_exact=u_exact, g=g, B0=B0)


def test_insulating_hartmann_convergence_and_zero_lorentz_force(orc):
    """Insulating walls, E = -<v> x B updated every step from the previous
    step's mean flow velocity: second-order convergence to the closed form,
    E_z = -B0 <v_x> at steady state, zero total Lorentz force, and the walls
    carry exactly sum rho g."""
    errs = []
    for H in (8, 16, 32):
        r = _insulating(orc, H)
        cfg, mask, f = r["cfg"], r["mask"], r["f"]
        vx = np.array([orc.node_macro(cfg, f[:, 0, j, 0])["v"][0] for j in range(2 * H)])
        errs.append(np.abs(vx - r["u_exact"]).max() / r["u_exact"].max())
        # the field is the zero-current field of the (steady) flow
        assert abs(r["E"][2] / (-r["B0"] * vx.mean()) - 1) < 1e-10
        assert abs(r["E"][0]) < 1e-20 and abs(r["E"][1]) < 1e-20
        # total Lorentz force: sum rho a = sum rho g (Eq. 36)
        mass, _, rhoa = orc.balance(cfg, mask, f)
        assert abs(rhoa[0] / (r["g"] * mass) - 1) < 1e-9
        # the walls carry the body force of g alone (steady Eq. 34)
        fn, fr, _ = orc.step_e(cfg, mask, f, r["E"])
        Fb = orc.wall_force(cfg, mask, fr, fn, 1)
        assert abs(Fb[0] / (r["g"] * mass) - 1) < 1e-8
    assert errs[-1] < 1.5e-3
    assert 2.5 < errs[0] / errs[1] < 4.5 and 2.5 < errs[1] / errs[2] < 4.5


def test_insulating_field_differs_from_conducting(orc):
    """Without the zero-current field (E = 0, conducting walls) the same
    channel runs slower: the Lorentz force then brakes the mean flow too."""
    r = _insulating(orc, 16)
    kw = dict(r["kw"], insulating=0)
    cfg = orc.make_cfg(**kw)
    f0 = orc.init(cfg, r["mask"], np.ones((1, 32, 2)), np.zeros((3, 1, 32, 2)))
    fc = orc.run(cfg, r["mask"], f0, 60 * 16 * 16)
    vi = orc.node_macro(r["cfg"], r["f"][:, 0, 16, 0])["v"][0]
    vc = orc.node_macro(cfg, fc[:, 0, 16, 0])["v"][0]
    assert vc < 0.5 * vi


def _offgrid_channel(orc, H, q1, q2, tau=0.8, model="e", nx=2, interpolate=True):
    """Channel with solid rows y = 0 and y = ny-1 and walls at y = 1 - q1 and
    y = ny - 2 + q2 (q the distance of the first fluid row to the wall)."""
    ny = 2 * H + 2
    yw_lo, yw_hi = 1 - q1, ny - 2 + q2
    y = np.arange(ny, dtype=float)
    phi = np.repeat(np.minimum(y - yw_lo, yw_hi - y)[None, :, None], nx, axis=2).astype(np.float32)
    mask = (phi < 0).astype(np.uint8)
    nu = (tau - 0.5) / 3
    L = yw_hi - yw_lo
    g = 8 * nu * 0.02 / L ** 2
    cfg = orc.make_cfg(q=9, nx=nx, ny=ny, nz=1, periodic=(1, 1, 1), tau=tau, force_model=model, g=(g, 0, 0),
                       wall_u=((0, 0, 0),), phi=phi if interpolate else None)
    f = _rest(orc, cfg, mask)
    f = orc.run(cfg, mask, f, int(20 * L * L / nu / 3))
    v = np.array([orc.node_macro(cfg, f[:, 0, j, 0])["v"][0] for j in range(1, ny - 1)])
    yy = np.arange(1, ny - 1)
    exact = g / (2 * nu) * (yy - yw_lo) * (yw_hi - yy)
    return np.abs(v - exact).max() / exact.max()


@pytest.mark.parametrize("q1,q2", [(0.3, 0.8), (0.15, 0.65)])
def test_interpolated_walls_second_order(orc, q1, q2):
    e = [_offgrid_channel(orc, H, q1, q2) for H in (4, 8, 16)]
    assert e[-1] < 2e-3
    assert 3.3 < e[0] / e[1] < 4.6 and 3.3 < e[1] / e[2] < 4.6
    # the same nodes with halfway bounce-back see the walls half a node off
    h = [_offgrid_channel(orc, H, q1, q2, interpolate=False) for H in (4, 8, 16)]
    assert h[-1] > 10 * e[-1] and h[0] / h[1] < 2.2 and h[1] / h[2] < 2.2


def test_interpolated_walls_halfway_limit(orc):
    """phi = +-1/2 on every solid link gives q = 1/2: the interpolation is the
    halfway rule, bit for bit, with moving walls."""
    nx, ny, nz = 11, 9, 8
    mask = inputs.sphere_mask(nx, ny, nz, (5.2, 4.1, 3.9), 2.6, wall=1)
    mask[:, 0, :] = 2
    phi = np.where(mask > 0, -0.5, 0.5).astype(np.float32)
    kw = dict(q=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), tau=0.7, force_model="d", g=(1e-3, 0, 2e-4),
              wall_u=((0.01, -0.02, 0.0), (0.03, 0, 0.01)), face_wall=(1, 1, 1, 1, 2, 1))
    a, b = orc.make_cfg(**kw), orc.make_cfg(**kw, phi=phi)
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=3, seed=2)
    f0 = orc.init(a, mask, rho, u * 0.5, inputs.noise(19, nx, ny, nz, 1e-2, seed=3))
    assert np.array_equal(orc.run(a, mask, f0, 6), orc.run(b, mask, f0, 6))


@pytest.mark.parametrize("model", ["e", "c"])
def test_interpolated_walls_exact_momentum_balance(orc, model):
    """F_wall = sum rho a - [M(t+dt) - M(t)]/dt every step with the
    interpolated incoming populations: the momentum exchange of Eq. (25) at
    the imaginary points closes the balance exactly."""
    nx, ny, nz = 14, 12, 10
    c0 = np.array([6.3, 5.8, 4.6])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = (np.sqrt((x - c0[0]) ** 2 + (y - c0[1]) ** 2 + (z - c0[2]) ** 2) - 3.4).astype(np.float32)
    mask = (phi < 0).astype(np.uint8)
    cfg = orc.make_cfg(q=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), dx=0.5, dt=0.2, tau=0.74,
                       force_model=model, g=(3e-2, -1e-2, 5e-3), wall_u=((0.02, 0.01, -0.01),), phi=phi)
    c = cfg.dx / cfg.dt
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=3, seed=7)
    f = orc.init(cfg, mask, rho, u * 0.5 * c, inputs.noise(19, nx, ny, nz, 1e-2, seed=8))
    for _ in range(4):
        _, M0, rhoa = orc.balance(cfg, mask, f)
        fn, fr = orc.step(cfg, mask, f)
        _, M1, _ = orc.balance(cfg, mask, fn)
        F = orc.wall_force(cfg, mask, fr, fn, -1, 0)
        ref = rhoa - (M1 - M0) / cfg.dt
        scale = np.abs(M0).max() / cfg.dt + np.abs(F).max()
        assert np.allclose(F, ref, rtol=0, atol=2e-14 * scale), (F, ref)
        f = fn


def test_stokes_equilibrium_moments(orc):
    """The linear equilibrium (note after Eq. 11): mass and momentum as Eq. (1),
    second moment c^2 rho delta / 3 without rho u u, third moment as Eq. (1)."""
    rng = np.random.default_rng(3)
    for q in (9, 19):
        e, w, _ = orc.lattice(q)
        D = 2 if q == 9 else 3
        for dx, dt in ((1.0, 1.0), (0.5, 0.2)):
            c = dx / dt
            cfg = orc.make_cfg(q=q, dx=dx, dt=dt, stokes=1)
            full = orc.make_cfg(q=q, dx=dx, dt=dt)
            rho = rng.uniform(0.9, 1.1)
            u = np.zeros(3)
            u[:D] = rng.uniform(-0.1, 0.1, D) * c
            f, ff = orc.feq(cfg, rho, u), orc.feq(full, rho, u)
            E = c * e.astype(float)
            assert np.isclose(f.sum(), rho, rtol=1e-14)
            assert np.allclose(E.T @ f, rho * u, rtol=0, atol=1e-14 * c)
            M2 = np.einsum("ai,aj,a->ij", E, E, f)
            ref = np.zeros((3, 3))
            ref[:D, :D] = c * c * rho / 3 * np.eye(D)
            assert np.allclose(M2, ref, rtol=0, atol=1e-14 * c * c)
            assert np.allclose(np.einsum("ai,aj,a->ij", E, E, ff) - M2, rho * np.outer(u, u), rtol=0,
                               atol=1e-14 * c * c)
            M3, M3f = (np.einsum("ai,aj,ak,a->ijk", E, E, E, x) for x in (f, ff))
            assert np.allclose(M3, M3f, rtol=0, atol=1e-13 * c ** 3)


def test_stokes_shear_wave_is_not_advected(orc):
    """A shear wave u_y = eps sin(kx) on a uniform stream u0 along x: the full
    equilibrium carries the momentum flux rho u u and advects the wave at u0
    (phase -k u0 t); the linear equilibrium has none, so the wave decays in
    place at exp(-nu k^2 t) (Stokes equation)."""
    nx, ny, T, u0, eps, tau = 64, 2, 400, 0.05, 1e-4, 0.8
    k = 2 * np.pi / nx
    nu = (tau - 0.5) / 3
    x = np.arange(nx)
    for stokes in (1, 0):
        cfg = orc.make_cfg(q=9, nx=nx, ny=ny, periodic=(1, 1, 1), tau=tau, force_model="e", stokes=stokes)
        mask = np.zeros((1, ny, nx), np.uint8)
        u = np.zeros((3, 1, ny, nx))
        u[0] = u0
        u[1] = eps * np.sin(k * x)[None, None, :]
        f = orc.run(cfg, mask, orc.init(cfg, mask, np.ones((1, ny, nx)), u), T)
        uy = np.array([orc.node_macro(cfg, f[:, 0, 0, i])["u"][1] for i in range(nx)])
        c1 = np.fft.rfft(uy)[1]
        phase = np.angle(c1 * 1j)              # 0 for eps sin(k x)
        amp = 2 * abs(c1) / nx
        if stokes:
            assert abs(phase) < 1e-10
            assert abs(amp / (eps * np.exp(-nu * k * k * T)) - 1) < 2e-3
        else:
            assert abs(np.angle(np.exp(1j * (phase + k * u0 * T)))) < 1e-3


def _brinkman(orc, H, tau=0.8, Da=0.02, model="e"):
    """Stokes equilibrium with a Darcy resistance between halfway walls:
    nu u'' - lambda u + g = 0, u(+-H) = 0; Da = k / H^2 with lambda = nu / k."""
    ny, nx = 2 * H, 2
    nu = (tau - 0.5) / 3
    lam = nu / (Da * H * H)
    m = np.sqrt(lam / nu)
    g = 0.02 * lam / (1 - 1 / np.cosh(m * H))
    cfg = orc.make_cfg(q=9, nx=nx, ny=ny, periodic=(1, 0, 1), tau=tau, force_model=model, g=(g, 0, 0),
                       stokes=1, darcy=lam, wall_u=((0, 0, 0),))
    mask = np.zeros((1, ny, nx), np.uint8)
    # decay of the resisted flow (1/lambda) and of the acoustic modes across the channel
    steps = int(30 / lam) + int(25 / (nu * (np.pi / (2 * H)) ** 2))
    f = orc.run(cfg, mask, _rest(orc, cfg, mask), steps)
    y = np.arange(ny) - H + 0.5
    exact = (g / lam) * (1 - np.cosh(m * y) / np.cosh(m * H))
    v = np.array([orc.node_macro(cfg, f[:, 0, j, 0])["v"][0] for j in range(ny)])
    return np.abs(v - exact).max() / exact.max(), cfg, mask, f, g


def test_brinkman_channel_second_order_and_balance(orc):
    errs = []
    for H in (8, 16, 32):
        e, cfg, mask, f, g = _brinkman(orc, H)
        errs.append(e)
        # steady: the walls carry sum rho a, which now includes the resistance
        fn, fr = orc.step(cfg, mask, f)
        F = orc.wall_force(cfg, mask, fr, fn, 1)
        _, _, rhoa = orc.balance(cfg, mask, f)
        assert abs(F[0] / rhoa[0] - 1) < 1e-9
    # the Brinkman layer (sqrt(k) = 0.14 H) is resolved better as H grows: the
    # ratio climbs towards 4 (2.8, then 3.3)
    assert errs[-1] < 3e-3
    assert 2.5 < errs[0] / errs[1] < 4.6 and 3.0 < errs[1] / errs[2] < 4.6 and errs[1] / errs[2] > errs[0] / errs[1]


def _induced_hartmann(orc, H, conducting, tau=0.8, Ha=4.0, B0=0.05):
    """Channel between walls at y = +-H in an external field (0, B0, 0) with
    the field induced (Dellar's vector lattice Boltzmann model, Sec. 4) and
    coupled through the Maxwell equilibrium of Eq. (10).  Steady equations:
    nu u'' + (B0/mu rho) b' + g = 0 and eta b'' + B0 u' = 0, u(+-H) = 0 and
    b(+-H) = 0 (insulating) or b'(+-H) = 0 (conducting, zero mean b)."""
    ny, nx = 2 * H, 2
    nu = (tau - 0.5) / 3
    K = nu * Ha ** 2 / H ** 2                   # B0^2 / (mu rho eta), mu = rho = 1
    eta = B0 ** 2 / K
    m = np.sqrt(K / nu)
    t = np.tanh(m * H) / (m * H)
    gain = 1 / (K * t) if not conducting else 1 / K
    g = 0.01 / (gain * (1 - 1 / np.cosh(m * H)))
    cfg = orc.make_cfg(q=9, nx=nx, ny=ny, nz=1, periodic=(1, 0, 1), tau=tau, force_model="e", g=(g, 0, 0),
                       B=(0, B0, 0), maxwell=1, mu=1.0, induced=1, eta=eta, mag_conducting=int(conducting),
                       wall_u=((0, 0, 0),))
    mask = np.zeros((1, ny, nx), np.uint8)
    f = orc.init(cfg, mask, np.ones((1, ny, nx)), np.zeros((3, 1, ny, nx)))
    f, gm, _ = orc.run_mhd(cfg, mask, f, orc.mag_init(cfg, mask), 80 * H * H)
    B = orc.mag_field(cfg, mask, gm)
    _, _, _, v = orc.stress(orc.with_field(cfg, B), mask, f, None, None, 2)
    y = np.arange(ny) - H + 0.5
    u = g * gain * (1 - np.cosh(m * y) / np.cosh(m * H))
    # integral of u from -H to y
    intu = g * gain * ((y + H) - (np.sinh(m * y) + np.sinh(m * H)) / (m * np.cosh(m * H)))
    if conducting:
        b = -(B0 / eta) * intu
        b -= b.mean()
    else:
        b = (B0 / eta) * (u.mean() * (y + H) - intu)
    eu = np.abs(v[0, 0, :, 0] - u).max() / u.max()
    eb = np.abs(B[0, 0, :, 0] - b).max() / np.abs(b).max()
    return eu, eb, B


@pytest.mark.parametrize("conducting", [False, True])
def test_induced_field_hartmann_second_order(orc, conducting):
    eu, eb = [], []
    for H in (8, 16, 32):
        a, b, B = _induced_hartmann(orc, H, conducting)
        eu.append(a)
        eb.append(b)
        # the normal component is uniform (div B = 0 across the channel)
        assert np.abs(B[1] - 0.05).max() < 1e-13
    assert eu[-1] < 2e-3 and eb[-1] < 6e-3
    for e in (eu, eb):
        assert 2.8 < e[0] / e[1] < 4.6 and 3.2 < e[1] / e[2] < 4.6


def test_induced_field_total_conserved_by_conducting_walls(orc):
    """Relaxation keeps sum_i g_ik = B_k at each node and bounce-back keeps
    the population at its node: the total field is conserved every step with
    conducting walls (not with insulating ones, which exchange with B_ext)."""
    nx, ny, nz = 12, 9, 7
    mask = inputs.random_solids(nx, ny, nz, 0.1, n_walls=1, seed=23)
    for conducting in (1, 0):
        cfg = orc.make_cfg(q=19, nx=nx, ny=ny, nz=nz, periodic=(1, 0, 1), tau=0.7, force_model="d",
                           g=(2e-3, 0, 1e-3), B=(0.02, 0.05, -0.03), maxwell=1, mu=1.0, induced=1, eta=0.05,
                           mag_conducting=conducting, wall_u=((0.01, 0, 0), (0, 0, 0)), face_wall=(1, 1, 2, 2, 1, 1))
        rho, u = inputs.smooth_fields(nx, ny, nz, dims=3, seed=4)
        f = orc.init(cfg, mask, rho, u * 0.5, inputs.noise(19, nx, ny, nz, 1e-2, seed=5))
        g = orc.mag_init(cfg, mask)
        B0 = orc.mag_field(cfg, mask, g).sum(axis=(1, 2, 3))
        drift = 0.0
        for _ in range(5):
            f, g, _ = orc.run_mhd(cfg, mask, f, g, 1)
            drift = max(drift, np.abs(orc.mag_field(cfg, mask, g).sum(axis=(1, 2, 3)) - B0).max())
        if conducting:
            assert drift < 1e-14 * nx * ny * nz
        else:
            assert drift > 1e-6


@pytest.mark.parametrize("q", [9, 19])
def test_induced_field_equilibrium_moments_and_relaxation(orc, q):
    """On a one-node periodic box propagation maps every field population to
    itself, so one step is g1 = g0 - (g0 - g^eq)/tau_m.  Recovering g^eq with
    tau_m = 1/2 + eta/(theta c^2 dt) must give the moments of Dellar's vector
    equilibrium (Sec. 4): sum_i g^eq_ik = B_k, sum_i e_il g^eq_ik =
    (v_l B_k - B_l v_k)/c and sum_i e_il e_im g^eq_ik = theta delta_lm B_k,
    with v the node's flow velocity (no body force: v = u).  The field
    directions are the rest and axis directions of the fluid lattice, in the
    fluid lattice's order (D2Q5: 0, +x, +y, -x, -y; D3Q7: 0, +-x, +-y, +-z)."""
    dx, dt = 0.5, 0.2
    c = dx / dt
    eta = 0.07
    if q == 9:
        e = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]])
        theta, dims = 1 / 3, 2
        B = np.array([0.03, -0.05, 0.0])
        u = c * np.array([0.02, -0.013, 0.0])
    else:
        e = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
        theta, dims = 1 / 4, 3
        B = np.array([0.03, -0.05, 0.02])
        u = c * np.array([0.02, -0.013, 0.017])
    cfg = orc.make_cfg(q=q, nx=1, ny=1, nz=1, periodic=(1, 1, 1), dx=dx, dt=dt, tau=0.8, force_model="e",
                       B=tuple(B), maxwell=1, mu=1.0, induced=1, eta=eta, wall_u=((0, 0, 0),))
    mask = np.zeros((1, 1, 1), np.uint8)
    f0 = orc.init(cfg, mask, np.full((1, 1, 1), 1.02), u.reshape(3, 1, 1, 1))
    g0 = orc.mag_init(cfg, mask)
    _, g1, _ = orc.run_mhd(cfg, mask, f0, g0, 1)
    om = 1 / (0.5 + eta / (theta * c * c * dt))
    geq = (g0 - (g0 - g1) / om)[:, :, 0, 0, 0]          # [k][i]
    assert np.allclose(geq.sum(axis=1), B, rtol=0, atol=1e-15)
    for l in range(dims):
        first = (e[:, l][None, :] * geq).sum(axis=1)
        want = (u[l] * B - B[l] * u) / c
        assert np.allclose(first, want, rtol=0, atol=1e-15), l
        for m in range(dims):
            second = (e[:, l][None, :] * e[:, m][None, :] * geq).sum(axis=1)
            assert np.allclose(second, theta * (l == m) * B, rtol=0, atol=1e-15), (l, m)
    # a wrong relaxation time would leave a spurious part: the recovered
    # equilibrium with 1.05 tau_m misses the moments
    bad = (g0 - (g0 - g1) * (0.5 + eta / (theta * c * c * dt)) * 1.05)[:, :, 0, 0, 0]
    assert np.abs(sum((e[:, 0][None, :] * bad).sum(axis=1)) - sum((u[0] * B - B[0] * u) / c)) > 1e-6


@pytest.mark.parametrize("q,model,conducting", [(9, "e", 0), (9, "c", 1), (19, "d", 0), (19, "e", 1)])
def test_induced_field_momentum_balance_every_step(orc, q, model, conducting):
    """The Maxwell term of Eq. (10) at the node's induced field carries no
    momentum, so every coupled fluid/field step changes the fluid momentum by
    the body force less what the walls take: the momentum exchange of
    Eq. (25) (no corrections) equals sum rho a - (M(t+1) - M(t))/dt to
    rounding (Eq. 32 per step), with moving walls, scattered solids, closed
    faces, non-unit dx and dt, and the field evolving with either wall rule."""
    if q == 9:
        nx, ny, nz, per = 12, 9, 1, (1, 0, 1)
        B = (0.12, 0.2, 0.0)
    else:
        nx, ny, nz, per = 7, 6, 5, (1, 0, 0)
        B = (0.1, 0.25, -0.05)
    mask = inputs.random_solids(nx, ny, nz, 0.12, n_walls=2, seed=21 + q)
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=per, dx=0.5, dt=0.2, tau=0.81,
                       force_model=model, g=(3e-2, -1e-2, 5e-3 if q == 19 else 0.0), B=B, maxwell=1, mu=1.3,
                       induced=1, eta=0.06, mag_conducting=conducting,
                       wall_u=((0.01, 0.02, -0.01), (0.0, -0.015, 0.02), (0.03, 0, 0)),
                       face_wall=(3, 3, 3, 2, 1, 3))
    c = cfg.dx / cfg.dt
    D = 2 if q == 9 else 3
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, seed=8)
    f = orc.init(cfg, mask, rho, u * 0.5 * c, inputs.noise(q, nx, ny, nz, 1e-2, seed=9))
    g = orc.mag_init(cfg, mask)
    B0 = orc.mag_field(cfg, mask, g)
    for _ in range(4):
        _, M0, rhoa = orc.balance(cfg, mask, f)
        fn, gn, fr = orc.run_mhd(cfg, mask, f, g, 1)
        _, M1, _ = orc.balance(cfg, mask, fn)
        F = orc.wall_force(cfg, mask, fr, fn, -1, 0)
        ref = rhoa - (M1 - M0) / cfg.dt
        scale = np.abs(M0).max() / cfg.dt + np.abs(F).max()
        # rounding of sums over every node and direction: N Q 2^-52 of the scale
        assert np.allclose(F, ref, rtol=0, atol=nx * ny * nz * q * 2.0 ** -52 * scale), (F, ref)
        f, g = fn, gn
    # the field did evolve (the Maxwell term was not the uniform one)
    assert np.abs(orc.mag_field(cfg, mask, g) - B0).max() > 1e-6
