"""Pins of the oracle's per-node arithmetic against what the paper and the
mathematics fix (no GPU).

* lattice tables: weights, isotropy up to fourth order, opposites;
* equilibrium moments of Eq. (11), including the Maxwell stress L_ij of Eq. (10);
* force-term moments of Eqs. (4)-(5) with the C and u^F of each model (Sec. 2);
* the Shan-Chen and exact-difference forms that models [c] and [d] reformulate;
* the total momentum increment dt rho a of every model (Sec. 2);
* the implicit flow velocity v = u + dt a/2 under the Lorentz force;
* the artefact term E_ij (Eq. 9) against its closed forms per model;
* the Smagorinsky relaxation time against the eddy-viscosity relation;
* the odd part of the collision written from the momentum j, the form the
  FP32 node codes evaluate, for every model, with the Lorentz force, LES and
  the Maxwell term.
"""
import itertools

import numpy as np
import pytest

RNG = np.random.default_rng(12345)


def _moments(e, w, f, c):
    ce = c * e.astype(float)
    m0 = f.sum()
    m1 = ce.T @ f
    m2 = np.einsum("ai,aj,a->ij", ce, ce, f)
    m3 = np.einsum("ai,aj,ak,a->ijk", ce, ce, ce, f)
    return m0, m1, m2, m3


@pytest.mark.parametrize("q", [9, 19])
def test_lattice_isotropy(orc, q):
    e, w, opp = orc.lattice(q)
    D = 2 if q == 9 else 3
    ef = e.astype(float)[:, :D]
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(w @ ef, 0, atol=1e-16)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, ef, ef), np.eye(D) / 3, atol=1e-16)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, ef, ef, ef), 0, atol=1e-16)
    d = np.eye(D)
    iso4 = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
            + np.einsum("il,jk->ijkl", d, d)) / 9
    assert np.allclose(np.einsum("a,ai,aj,ak,al->ijkl", w, ef, ef, ef, ef), iso4, atol=1e-16)
    assert np.array_equal(e[opp], -e)
    # the standard velocity sets: unique vectors, speed classes 1/4/4 and 1/6/12
    assert len({tuple(x) for x in e}) == q
    n2 = (e * e).sum(1)
    counts = [int((n2 == k).sum()) for k in (0, 1, 2, 3)]
    assert counts == ([1, 4, 4, 0] if q == 9 else [1, 6, 12, 0])
    if q == 9:
        assert np.all(e[:, 2] == 0)


def _random_cfg(orc, q, model="e", **kw):
    base = dict(q=q, nx=4, ny=4, nz=4 if q == 19 else 1, dx=0.5, dt=0.25, tau=0.73, rho0=1.0,
                force_model=model, g=tuple(RNG.uniform(-1e-2, 1e-2, 3)))
    base.update(kw)
    return orc.make_cfg(**base)


def _random_f(orc, cfg):
    c = cfg.dx / cfg.dt
    D = 2 if cfg.q == 9 else 3
    u = np.zeros(3)
    u[:D] = RNG.uniform(-0.1, 0.1, D) * c
    rho = RNG.uniform(0.9, 1.1)
    feq = orc.feq(cfg, rho, u)
    return feq * (1 + RNG.uniform(-0.05, 0.05, cfg.q))


@pytest.mark.parametrize("q,maxwell", list(itertools.product([9, 19], [0, 1])))
def test_equilibrium_moments(orc, q, maxwell):
    """Eq. (11): M = rho, M_i = rho u, M_ij = c^2 rho delta/3 + rho u u + L,
    M_ijk = c^2 rho (delta u + delta u + delta u)/3, L = (B^2 delta/2 - B B)/mu."""
    D = 2 if q == 9 else 3
    B = np.array([0.03, -0.02, 0.04 if D == 3 else 0.0])
    cfg = _random_cfg(orc, q, maxwell=maxwell, B=B, mu=1.7)
    c = cfg.dx / cfg.dt
    e, w, _ = orc.lattice(q)
    for _ in range(5):
        rho = RNG.uniform(0.9, 1.1)
        u = np.zeros(3)
        u[:D] = RNG.uniform(-0.1, 0.1, D) * c
        f = orc.feq(cfg, rho, u)
        m0, m1, m2, m3 = _moments(e, w, f, c)
        d = np.diag([1.0] * D + [0.0] * (3 - D))
        Bd = B.copy()
        L = (Bd @ Bd * d / 2 - np.outer(Bd, Bd)) / cfg.mu if maxwell else 0 * d
        if D == 2:
            L[2, :] = 0
            L[:, 2] = 0
        assert np.isclose(m0, rho, rtol=1e-14)
        assert np.allclose(m1, rho * u, rtol=0, atol=1e-15 * c)
        assert np.allclose(m2, c * c * rho * d / 3 + rho * np.outer(u, u) + L, rtol=0,
                           atol=1e-14 * c * c)
        m3e = c * c * rho / 3 * (np.einsum("ij,k->ijk", d, u) + np.einsum("ik,j->ijk", d, u)
                                 + np.einsum("jk,i->ijk", d, u))
        assert np.allclose(m3, m3e, rtol=0, atol=1e-14 * c ** 3)


@pytest.mark.parametrize("q,model", list(itertools.product([9, 19], "abcde")))
def test_force_term_moments(orc, q, model):
    """Eqs. (4)-(5): sum F = 0, sum e F = C dt rho a, sum e e F = Theta with
    Theta = C dt rho (u^F a + a u^F) for [b]-[e] and 0 for [a]; C and u^F per
    Sec. 2: [a],[b] u; [c] u + tau dt a/2; [d],[e] v = u + dt a/2; C = 1
    except [e] with C = 1 - 1/(2 tau)."""
    cfg = _random_cfg(orc, q, model)
    c = cfg.dx / cfg.dt
    e, w, _ = orc.lattice(q)
    D = 2 if q == 9 else 3
    for _ in range(5):
        f = _random_f(orc, cfg)
        F = orc.force_term(cfg, f)
        m0, m1, m2, _ = _moments(e, w, f, c)
        rho, u = m0, m1 / m0
        a = np.array(cfg.g[:])
        a[D:] = 0
        v = u + 0.5 * cfg.dt * a
        uF = {"a": u, "b": u, "c": u + 0.5 * cfg.tau * cfg.dt * a, "d": v, "e": v}[model]
        C = 1 - 1 / (2 * cfg.tau) if model == "e" else 1.0
        F0, F1, F2, _ = _moments(e, w, F, c)
        scale = rho * np.abs(a).max() * cfg.dt * c
        assert abs(F0) < 1e-14 * scale / c
        assert np.allclose(F1, C * cfg.dt * rho * a, rtol=0, atol=1e-13 * scale)
        Theta = 0 * np.eye(3) if model == "a" else C * cfg.dt * rho * (np.outer(uF, a) + np.outer(a, uF))
        assert np.allclose(F2, Theta, rtol=0, atol=1e-13 * scale * c)


@pytest.mark.parametrize("q", [9, 19])
def test_reformulated_models_equal_originals(orc, q):
    """[c] is the Shan-Chen scheme f + (f^eq(rho, u + tau dt a) - f)/tau, and
    [d] is the exact difference method f + (f^eq(u) - f)/tau + f^eq(u + dt a)
    - f^eq(u) (Sec. 2): the reformulations must equal them identically."""
    e, w, _ = orc.lattice(q)
    for tau in (0.6, 0.73, 1.0, 1.7):
        for model in "cd":
            cfg = _random_cfg(orc, q, model, tau=tau)
            c = cfg.dx / cfg.dt
            D = 2 if q == 9 else 3
            a = np.array(cfg.g[:])
            a[D:] = 0
            for _ in range(4):
                f = _random_f(orc, cfg)
                rho = f.sum()
                u = (c * e.astype(float)).T @ f / rho
                if model == "c":
                    ref = f + (orc.feq(cfg, rho, u + tau * cfg.dt * a) - f) / tau
                else:
                    ref = (f + (orc.feq(cfg, rho, u) - f) / tau
                           + orc.feq(cfg, rho, u + cfg.dt * a) - orc.feq(cfg, rho, u))
                got = orc.collide_node(cfg, f)
                assert np.allclose(got, ref, rtol=0, atol=1e-15), (model, tau)


@pytest.mark.parametrize("q,model", list(itertools.product([9, 19], "abcde")))
def test_collision_mass_and_momentum_increment(orc, q, model):
    """Every model adds exactly dt rho a of momentum per node (force term plus
    relaxation, Sec. 2) and conserves mass."""
    cfg = _random_cfg(orc, q, model)
    c = cfg.dx / cfg.dt
    e, w, _ = orc.lattice(q)
    D = 2 if q == 9 else 3
    a = np.array(cfg.g[:])
    a[D:] = 0
    for _ in range(5):
        f = _random_f(orc, cfg)
        fr = orc.collide_node(cfg, f)
        m0, m1, _, _ = _moments(e, w, f, c)
        r0, r1, _, _ = _moments(e, w, fr, c)
        assert np.isclose(r0, m0, rtol=1e-15, atol=0)
        assert np.allclose(r1 - m1, cfg.dt * m0 * a, rtol=0, atol=1e-15 * c)


@pytest.mark.parametrize("q", [9, 19])
def test_lorentz_implicit_velocity(orc, q):
    """With the imposed-field Lorentz force, the node's v and a satisfy
    v = u + dt a/2 and a = g + (sigma_e/rho)(E + v x B) x B simultaneously."""
    D = 2 if q == 9 else 3
    for model in "abcde":
        B = RNG.uniform(-0.3, 0.3, 3)
        E = RNG.uniform(-0.01, 0.01, 3)
        cfg = _random_cfg(orc, q, model, lorentz=1, B=B, E=E, sigma_e=RNG.uniform(0.5, 2.0))
        for _ in range(3):
            f = _random_f(orc, cfg)
            m = orc.node_macro(cfg, f)
            v, a, u, rho = m["v"], m["a"], m["u"], m["rho"]
            aL = cfg.sigma_e / rho * np.cross(np.array(cfg.E[:]) + np.cross(v, B), B)
            a_ref = np.array(cfg.g[:]) + aL
            a_ref[D:] = 0
            assert np.allclose(a, a_ref, rtol=0, atol=1e-15)
            assert np.allclose(v, u + 0.5 * cfg.dt * a, rtol=0, atol=1e-16)
            assert np.allclose(v[D:], 0)


@pytest.mark.parametrize("q,model", list(itertools.product([9, 19], "abcde")))
def test_artefact_term_closed_forms(orc, q, model):
    """Variant 1 minus variant 2 of the stress is -(1 - 1/(2 tau)) E_ij, and
    E_ij = tau dt rho(u^eq a + a u^eq) - tau Theta reduces per model to
    [a] tau dt rho (u a + a u); [b] 0; [c] -tau^2 dt^2 rho a a;
    [d] -tau dt^2 rho a a; [e] dt/2 rho (v a + a v) (the last two also in the
    commented case list after Eq. 9)."""
    D = 2 if q == 9 else 3
    nx, ny, nz = 4, 3, (2 if q == 19 else 1)
    cfg = _random_cfg(orc, q, model, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1),
                      g=tuple(RNG.uniform(-5e-2, 5e-2, 3)))
    from paper_2512_12213_gb300 import inputs
    mask = inputs.empty_mask(nx, ny, nz)
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, seed=3)
    f = orc.init(cfg, mask, rho, u * cfg.dx / cfg.dt, inputs.noise(q, nx, ny, nz, 2e-2, seed=4))
    s1, _, r1, v1 = orc.stress(cfg, mask, f, None, None, 1)
    s2, _, _, _ = orc.stress(cfg, mask, f, None, None, 2)
    tau, dt = cfg.tau, cfg.dt
    a = np.array(cfg.g[:])
    a[D:] = 0
    comps = [(0, 0), (1, 1), (0, 1)] if D == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    N = nx * ny * nz
    r1 = r1.reshape(N)
    v1 = v1.reshape(3, N)
    for n in range(N):
        rho_n, v = r1[n], v1[:, n]
        uu = v - 0.5 * dt * a
        sym = lambda x, y: np.outer(x, y) + np.outer(y, x)
        E = {"a": tau * dt * rho_n * sym(uu, a), "b": 0 * np.eye(3),
             "c": -tau * tau * dt * dt * rho_n * np.outer(a, a),
             "d": -tau * dt * dt * rho_n * np.outer(a, a),
             "e": 0.5 * dt * rho_n * sym(v, a)}[model]
        for k, (i, j) in enumerate(comps):
            got = s1.reshape(len(comps), N)[k, n] - s2.reshape(len(comps), N)[k, n]
            # tolerance: rounding of the two stress evaluations
            assert np.isclose(got, -(1 - 1 / (2 * tau)) * E[i, j], rtol=0,
                              atol=1e-12 * np.abs(s2).max() + 1e-12 * abs(E).max()), (model, n, i, j)


@pytest.mark.parametrize("q", [9, 19])
def test_smagorinsky_relation(orc, q):
    """LES: nu_eff - nu_0 = (Cs dx)^2 |S| with |S| = sqrt(2 S:S) and
    S = -3 Pi^neq/(2 tau_eff rho dt c^2) (Eq. 9 without E_ij), where
    nu = dt c^2 (tau - 1/2)/3."""
    cfg = _random_cfg(orc, q, "b", les=1, cs=0.17, g=(0, 0, 0))
    c, dt = cfg.dx / cfg.dt, cfg.dt
    e, w, _ = orc.lattice(q)
    ce = c * e.astype(float)
    for _ in range(6):
        f = _random_f(orc, cfg)
        m = orc.node_macro(cfg, f)
        rho, u, te = m["rho"], m["u"], m["tau"]
        fe = orc.feq(cfg, rho, u)
        P = np.einsum("ai,aj,a->ij", ce, ce, f - fe)
        S = -3 * P / (2 * te * rho * dt * c * c)
        Smag = np.sqrt(2 * (S * S).sum())
        lhs = dt * c * c * (te - cfg.tau) / 3
        assert te > cfg.tau
        assert np.isclose(lhs, (cfg.cs * cfg.dx) ** 2 * Smag, rtol=1e-12)


@pytest.mark.parametrize("q,model,extra", list(itertools.product(
    [9, 19], "abcde", ["plain", "lorentz", "les", "maxwell"])))
def test_odd_part_from_the_momentum(orc, q, model, extra):
    """The odd part of the collision, per opposite pair (a, opp a),
    (f'_a - f'_opp)/2 = (1 - om)(f_a - f_opp)/2 + 3 w_a (om E_a.j + rho dt E_a.a / c)
    with j = sum_b E_b f_b: for every model of Sec. 2, om rho E_a.u^eq / c +
    C rho dt E_a.a / c equals om E_a.j + rho dt E_a.a / c (u^eq = u + dt a/2
    with C = 1 - om/2 for [e], u^eq = u with C = 1 for [a]-[d]).  The GPU's
    FP32 node codes evaluate the odd part in this form; here the oracle's
    collision (Eqs. 1-3 as the paper writes them) is checked against it, with
    the Lorentz force (a from the implicit v), Smagorinsky LES (the node's own
    relaxation time) and the Maxwell term (even, so absent from the odd part)."""
    kw = {}
    if extra == "lorentz":
        kw = dict(lorentz=1, B=(0.02, 0.05, 0.03 if q == 19 else 0.0), sigma_e=0.7, E=(1e-3, 0.0, 2e-3))
    elif extra == "les":
        kw = dict(les=1, cs=0.2)
    elif extra == "maxwell":
        kw = dict(maxwell=1, B=(0.03, -0.02, 0.04 if q == 19 else 0.0), mu=1.3)
    cfg = _random_cfg(orc, q, model, **kw)
    c = cfg.dx / cfg.dt
    e, w, opp = orc.lattice(q)
    E = e.astype(float)
    for _ in range(4):
        f = _random_f(orc, cfg)
        nm = orc.node_macro(cfg, f)
        om = 1.0 / nm["tau"]
        fr = orc.collide_node(cfg, f)
        j = E.T @ f
        rho = f.sum()
        for a in range(1, q):
            b = opp[a]
            got = 0.5 * (fr[a] - fr[b])
            want = (1 - om) * 0.5 * (f[a] - f[b]) + 3 * w[a] * (om * (E[a] @ j) + rho * cfg.dt * (E[a] @ nm["a"]) / c)
            assert np.isclose(got, want, rtol=0, atol=1e-14 * max(abs(f).max(), 1.0)), (a, got, want)
