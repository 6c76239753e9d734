"""Pins of the oracle's steady-state residual (no GPU).

Sec. 6 states the global balance between the wall force and the body force
on the fluid (Eq. 32 and the steady form after it); it holds once the flow
no longer changes, and the residual r = sum |v(t) - v(t - k)| / sum |v(t)|
over fluid nodes (v the flow velocity of the text after Eq. 1) is the
measure of that.  The pins fix it by results that do not use its formula:

* uniform body force in a periodic box: every model adds exactly rho a dt of
  momentum per node and step, so the state stays uniform and the flow
  velocity is v(t) = g dt (t + 1/2) at every node; hence
  r = (t2 - t1)/(t2 + 1/2) (the 1/2 is the half force of v = u + dt a/2);
* a decaying shear wave u_x = U sin(K y): the wave decays as exp(-nu K^2 t),
  so r over k steps is exp(nu K^2 k dt) - 1 (to the lattice's O(K^2)
  correction of the decay rate);
* a uniform stream at equilibrium is a fixed point of the step: r = 0;
* against a zero or a reversed reference field r is 1 or 2.
"""
import math

import numpy as np
import pytest


def _uniform(orc, cfg, shape, u=(0.0, 0.0, 0.0)):
    nz, ny, nx = shape
    uu = np.zeros((3, nz, ny, nx))
    for k in range(3):
        uu[k] = u[k]
    return orc.init(cfg, np.zeros(shape, np.uint8), np.full(shape, cfg.rho0), uu)


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("model", list("abcde"))
def test_uniform_force_velocity_and_residual(orc, q, model):
    shape = (1, 5, 6) if q == 9 else (4, 3, 5)
    g = (2e-4, -7e-5, 0.0) if q == 9 else (2e-4, -7e-5, 4e-5)
    dx, dt = 0.5, 0.25
    cfg = orc.make_cfg(q=q, nx=shape[2], ny=shape[1], nz=shape[0], periodic=(1, 1, 1), dx=dx, dt=dt,
                       tau=0.8, force_model=model, g=g)
    mask = np.zeros(shape, np.uint8)
    f = _uniform(orc, cfg, shape)
    t1, t2 = 7, 19
    f1 = orc.run(cfg, mask, f, t1)
    _, _, _, v1 = orc.residual(cfg, mask, f1)
    for k in range(3):
        assert np.allclose(v1[k], g[k] * dt * (t1 + 0.5), rtol=0, atol=1e-15)
    f2 = orc.run(cfg, mask, f1, t2 - t1)
    dsum, vsum, r, v2 = orc.residual(cfg, mask, f2, v1)
    for k in range(3):
        assert np.allclose(v2[k], g[k] * dt * (t2 + 0.5), rtol=0, atol=1e-15)
    gn = math.sqrt(sum(x * x for x in g))
    n = int(np.prod(shape))
    # (the momentum sums cancel O(w rho) terms down to O(g dt t): ~1e-12 relative)
    assert vsum == pytest.approx(n * gn * dt * (t2 + 0.5), rel=1e-10)
    assert dsum == pytest.approx(n * gn * dt * (t2 - t1), rel=1e-10)
    assert r == pytest.approx((t2 - t1) / (t2 + 0.5), rel=1e-10)


@pytest.mark.parametrize("q", [9, 19])
def test_shear_wave_residual_closed_form(orc, q):
    L, U, tau = 64, 1e-4, 0.8
    if q == 9:
        shape = (1, L, 2)
    else:
        shape = (L, 2, 2)          # wave along z, flow along x
    nz, ny, nx = shape
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=tau, force_model="e")
    mask = np.zeros(shape, np.uint8)
    z, y, _ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = y if q == 9 else z
    K = 2 * math.pi / L
    u = np.zeros((3,) + shape)
    u[0] = U * np.sin(K * s)
    f = orc.init(cfg, mask, np.ones(shape), u)
    nu = (tau - 0.5) / 3
    f = orc.run(cfg, mask, f, 100)            # let the non-equilibrium part settle
    _, _, _, v1 = orc.residual(cfg, mask, f)
    k = 400
    f = orc.run(cfg, mask, f, k)
    _, _, r, v2 = orc.residual(cfg, mask, f, v1)
    expect = math.exp(nu * K * K * k) - 1
    assert r == pytest.approx(expect, rel=5e-3)
    # against its own velocity field the residual vanishes
    _, _, r_self, _ = orc.residual(cfg, mask, f, v2)
    assert r_self == 0.0
    # the decayed amplitude itself
    assert np.abs(v2[0]).max() / np.abs(v1[0]).max() == pytest.approx(math.exp(-nu * K * K * k), rel=5e-3)


@pytest.mark.parametrize("q", [9, 19])
def test_equilibrium_stream_is_steady(orc, q):
    shape = (1, 7, 9) if q == 9 else (5, 4, 6)
    u0 = (0.03, -0.02, 0.0) if q == 9 else (0.03, -0.02, 0.01)
    cfg = orc.make_cfg(q=q, nx=shape[2], ny=shape[1], nz=shape[0], periodic=(1, 1, 1), tau=0.7,
                       force_model="e")
    mask = np.zeros(shape, np.uint8)
    f = _uniform(orc, cfg, shape, u0)
    _, _, _, v0 = orc.residual(cfg, mask, f)
    f = orc.run(cfg, mask, f, 50)
    dsum, vsum, r, _ = orc.residual(cfg, mask, f, v0)
    assert r < 1e-13
    assert vsum == pytest.approx(int(np.prod(shape)) * math.sqrt(sum(x * x for x in u0)), rel=1e-13)


def test_reference_fields_zero_and_reversed(orc):
    from paper_2512_12213_gb300 import inputs
    nx, ny = 11, 8
    mask = inputs.random_solids(nx, ny, 1, 0.15, n_walls=1, seed=4)
    cfg = orc.make_cfg(q=9, nx=nx, ny=ny, nz=1, periodic=(1, 1, 1), tau=0.9, force_model="d",
                       g=(1e-4, 0, 0), wall_u=((0, 0, 0),))
    rho, u = inputs.smooth_fields(nx, ny, 1, dims=2, u_amplitude=0.03, seed=2)
    f = orc.init(cfg, mask, rho, u)
    _, vsum, r0, v = orc.residual(cfg, mask, f)
    assert r0 == pytest.approx(1.0, rel=1e-15)
    assert np.all(v[:, mask == 1] == 0.0)
    _, _, r2, _ = orc.residual(cfg, mask, f, -v)
    assert r2 == pytest.approx(2.0, rel=1e-14)
    _, _, rs, _ = orc.residual(cfg, mask, f, v)
    assert rs == 0.0


def test_openmp_timing_build_gives_the_same_state(orc):
    """The OpenMP timing copy of the oracle (parallel node loops only) steps
    to exactly the state of the single-threaded parity build."""
    from paper_2512_12213_gb300 import inputs
    nx, ny, nz = 17, 9, 6
    mask = inputs.sphere_mask(nx, ny, nz, (8.2, 4.1, 3.0), 2.4, wall=1)
    cfg = orc.make_cfg(q=19, nx=nx, ny=ny, nz=nz, periodic=(1, 0, 1), tau=0.7, force_model="e",
                       g=(1e-4, 0, 2e-5), wall_u=((0, 0, 0), (0.02, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=3, u_amplitude=0.03, seed=5)
    f = orc.init(cfg, mask, rho, u)
    a = orc.run(cfg, mask, f, 5)
    b = orc.run(cfg, mask, f, 5, omp=True)
    assert np.array_equal(a, b)
