"""Pins of the oracle's discrete adjoint of the time-averaged wall drag (no GPU).

J = (1/T) sum_{t<T} d . F_wall(t), F_wall the uncorrected momentum exchange of
Eq. (25) on one wall, differentiated with respect to the uniform body force g
and that wall's velocity u_w.  The adjoint (transpose of propagation and of
each node's complex-step collision Jacobian) must agree with central finite
differences of the forward oracle, and J itself with the time-summed exact
momentum balance (the discrete form of Eq. 32).
"""
import numpy as np
import pytest

from paper_2512_12213_gb300 import inputs


def _setup(orc, q, model, les=0, lorentz=0):
    if q == 9:
        nx, ny, nz, per = 10, 8, 1, (1, 0, 1)
        mask = inputs.block_mask(nx, ny, nz, (3, 3, 0), (5, 5, 1), wall=1)
    else:
        nx, ny, nz, per = 6, 6, 5, (1, 1, 0)
        mask = inputs.block_mask(nx, ny, nz, (2, 2, 1), (4, 4, 3), wall=1)
    kw = dict(q=q, nx=nx, ny=ny, nz=nz, periodic=per, tau=0.7, dx=0.5, dt=0.25, force_model=model,
              g=(2e-2, -7e-3, 3e-3), wall_u=((0.03, -0.02, 0.01), (0.0, 0.0, 0.0)),
              face_wall=(2, 2, 2, 2, 2, 2), les=les, cs=0.15, lorentz=lorentz,
              B=(0.1, 0.2, 0.05), sigma_e=0.5)
    cfg = orc.make_cfg(**kw)
    f0 = orc.init(cfg, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    return kw, cfg, mask, f0


def _fd(orc, kw, mask, f0, T, d):
    fd = np.zeros(6)
    for k in range(6):
        for sgn in (1, -1):
            kw2 = dict(kw)
            if k < 3:
                g = list(kw["g"])
                h = 1e-4 * max(abs(g[k]), 1e-3)
                g[k] += sgn * h
                kw2["g"] = tuple(g)
            else:
                wu = [list(x) for x in kw["wall_u"]]
                h = 1e-4 * max(abs(wu[0][k - 3]), 1e-2)
                wu[0][k - 3] += sgn * h
                kw2["wall_u"] = tuple(map(tuple, wu))
            fd[k] += sgn * orc.drag_average(orc.make_cfg(**kw2), mask, f0, T, 1, d) / (2 * h)
    return fd


CASES = [(9, m, 0, 0) for m in "abcde"] + [(19, m, 0, 0) for m in "abcde"] + [
    (9, "e", 1, 0), (9, "d", 0, 1), (19, "c", 1, 1)]


@pytest.mark.parametrize("q,model,les,lorentz", CASES)
def test_adjoint_matches_central_differences(orc, q, model, les, lorentz):
    kw, cfg, mask, f0 = _setup(orc, q, model, les, lorentz)
    T, d = 12, (1.0, 0.3, -0.2)
    J, grad = orc.adjoint_drag(cfg, mask, f0, T, 1, d)
    assert np.isclose(J, orc.drag_average(cfg, mask, f0, T, 1, d), rtol=1e-14)
    fd = _fd(orc, kw, mask, f0, T, d)
    idx = [0, 1, 3, 4] if q == 9 else list(range(6))
    # central differences with h = 1e-4 |theta|: truncation ~1e-8 |grad|
    assert np.allclose(grad[idx], fd[idx], rtol=0, atol=1e-8 * np.abs(fd[idx]).max())
    if q == 9:
        assert grad[2] == 0 and grad[5] == 0


def test_drag_average_equals_time_summed_balance(orc):
    """sum_t F_all(t) = sum_t sum rho a(t) - [M(T) - M(0)]/dt, so with a single
    wall J = d . (mean body force) - d . (M(T) - M(0))/(T dt)."""
    q = 9
    nx, ny, nz = 12, 10, 1
    mask = inputs.cylinder_mask(nx, ny, (5.5, 4.8), 2.3)
    cfg = orc.make_cfg(q=q, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.65, dx=1.0, dt=1.0,
                       force_model="d", g=(1e-3, 2e-4, 0), wall_u=((0.0, 0.0, 0.0),))
    f0 = orc.init(cfg, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    T, d = 15, np.array([1.0, 0.0, 0.0])
    J = orc.drag_average(cfg, mask, f0, T, 1, d)
    f = f0.copy()
    _, M0, _ = orc.balance(cfg, mask, f0)
    body = np.zeros(3)
    for _ in range(T):
        _, _, rhoa = orc.balance(cfg, mask, f)
        body += rhoa / T
        f, _ = orc.step(cfg, mask, f)
    _, MT, _ = orc.balance(cfg, mask, f)
    ref = d @ body - d @ (MT - M0) / (T * cfg.dt)
    assert np.isclose(J, ref, rtol=1e-12)
