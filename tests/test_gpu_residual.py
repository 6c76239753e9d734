"""Steady-state residual through the C ABI against the oracle, and the
statuses built on it.

Sec. 6 balances the wall force against the body force on the fluid
(Eq. 32); the steady form holds once the flow stops changing, which the
residual r = sum |v - v_ref| / sum |v| over fluid nodes measures (v the flow
velocity of the text after Eq. 1).  Checked here:

* the sums, r and the stored velocity field against ``orc_residual`` after a
  few steps from a noisy state (FP64 within 1e-12; the FP32-compute formats
  within bounds set by their storage rounding: the velocity of a node is a
  sum of Q stored deviations of relative half-ulp u, so its error is about
  u |d| / |u| relative, FP32 2e-6, binary16 5e-4, bfloat16 5e-3 of max |v|);
* device, page-locked host and host outputs agree bit for bit;
* ``lbm_run_steady`` on the Poiseuille channel (64 x 32, tau 0.8, g 1e-6)
  stops with r below its tolerance at the exact discrete solution
  v = (g/2nu)[(y + 1/2)(H - 1/2 - y) + (16 Lambda - 3)/12], Lambda = (tau - 1/2)^2,
  where the walls carry the whole body force (the steady balance after
  Eq. 32), and with too few steps allowed it reports LBM_ERR_NOT_CONVERGED;
* a state holding a NaN makes the host-output reductions return LBM_ERR_NAN.
"""
import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import inputs, lbm, workloads

pytestmark = pytest.mark.gpu

VTOL = {"f64": 1e-12, "f32": 2e-6, "f16s": 5e-4, "bf16s": 5e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()
    assert torch.cuda.is_available()


def _case(name, storage):
    if name == "d2q9_lorentz":
        nx, ny = 70, 37
        mask = inputs.cylinder_mask(nx, ny, (20.5, 14.2), 5.3, wall=3)
        cfg = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=(1, 0, 1), dx=0.5, dt=0.2, tau=0.81, force_model="d",
                   g=(1e-3, 0, 0), lorentz=1, B=(0.05, 0.2, 0.0), E=(0, 0, 1e-3), sigma_e=0.3, maxwell=1, mu=0.9,
                   storage=storage, wall_u=((0, 0, 0), (0.03, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    elif name == "d3q19_sphere":
        nx, ny, nz = 50, 13, 11
        mask = inputs.sphere_mask(nx, ny, nz, (21.3, 6.2, 5.4), 3.3, wall=1)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.66, force_model="e",
                   g=(2e-4, -1e-4, 5e-5), storage=storage, wall_u=((0, 0, 0),))
    elif name == "cavity_les":
        n = 19
        mask = inputs.empty_mask(n, n, n)
        cfg = dict(lattice=19, nx=n, ny=n, nz=n, periodic=(0, 0, 0), tau=0.55, force_model="e", les=1, cs=0.1,
                   storage=storage, wall_u=((0, 0, 0), (0.1, 0, 0)), face_wall=(1, 1, 1, 1, 1, 2))
    else:
        raise KeyError(name)
    return cfg, mask


def _start(orc, cfg, mask):
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    nz, ny, nx = mask.shape
    D = 2 if cfg["lattice"] == 9 else 3
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, u_amplitude=0.04, seed=8)
    c = cfg.get("dx", 1.0) / cfg.get("dt", 1.0)
    f0 = orc.init(ocfg, mask, rho, u * c, inputs.noise(cfg["lattice"], nx, ny, nz, 1e-3, seed=9))
    return ocfg, f0


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("name", ["d2q9_lorentz", "d3q19_sphere", "cavity_les"])
def test_residual_against_oracle(orc, name, storage):
    cfg, mask = _case(name, storage)
    ocfg, f0 = _start(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    vref = sim.velocity_buffer()
    tol = VTOL[storage]
    f = orc.run(ocfg, mask, f0, 3)
    sim.step(3)
    got = sim.residual(vref)                           # against zero: r = 1
    d0, s0, r0, v3 = orc.residual(ocfg, mask, f)
    vmax = np.abs(v3).max()
    assert np.abs(vref.cpu().numpy() - v3).max() <= tol * vmax
    assert got[1] == pytest.approx(s0, rel=tol)
    assert got[0] == pytest.approx(d0, rel=tol)
    assert got[2] == pytest.approx(1.0, rel=1e-14)
    f = orc.run(ocfg, mask, f, 4)
    sim.step(4)
    got = sim.residual(vref)
    d1, s1, r1, v7 = orc.residual(ocfg, mask, f, v3)
    assert np.abs(vref.cpu().numpy() - v7).max() <= tol * vmax
    assert got[1] == pytest.approx(s1, rel=tol)
    # the change over 4 steps is a difference of velocities: its error is
    # the velocity error of both states, relative to sum |v|
    assert abs(got[0] - d1) <= 4 * tol * s1
    assert abs(got[2] - r1) <= 4 * tol
    if storage == "f64":
        assert got[0] == pytest.approx(d1, rel=1e-11)
        assert got[2] == pytest.approx(r1, rel=1e-11)
    sim.close()


def test_residual_outputs_agree():
    cfg, mask = _case("d3q19_sphere", "f32")
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(20)
    st = sim.stream
    v1, v2, v3 = (sim.velocity_buffer() for _ in range(3))
    host = np.zeros(3)
    lbm.lbm_residual(sim.ctx, v1, 1, host, lbm.OUT_HOST, st)
    dev = torch.zeros(3, dtype=torch.float64, device=sim.device)
    lbm.lbm_residual(sim.ctx, v2, 1, dev, lbm.OUT_DEVICE, st)
    pinned = torch.zeros(3, dtype=torch.float64, pin_memory=True)
    lbm.lbm_residual(sim.ctx, v3, 1, pinned, lbm.OUT_HOST_ASYNC, st)
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())
    assert np.array_equal(host, pinned.numpy())
    assert torch.equal(v1, v2) and torch.equal(v1, v3)
    # without update the reference stays as it was
    sim.step(5)
    keep = v1.clone()
    lbm.lbm_residual(sim.ctx, v1, 0, host, lbm.OUT_HOST, st)
    assert torch.equal(v1, keep) and host[2] > 0
    sim.close()


def test_run_steady_poiseuille_reaches_the_discrete_solution():
    cfg, mask = workloads.poiseuille(storage="f64")       # 64 x 32, tau 0.8, g 1e-6, model [d]
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    r, steps = sim.run_steady(every=500, tol=1e-11, max_steps=200_000)
    assert r <= 1e-11 and steps % 500 == 0 and steps < 200_000
    H, tau, g = cfg["ny"], cfg["tau"], cfg["g"][0]
    nu = (tau - 0.5) / 3
    lam = (tau - 0.5) ** 2
    y = np.arange(H)
    exact = g / (2 * nu) * ((y + 0.5) * (H - 0.5 - y) + (16 * lam - 3) / 12)
    _, _, _, v = sim.stress(lbm.S2)
    vx = v[0, 0].cpu().numpy()                          # (ny, nx)
    assert np.abs(vx - exact[:, None]).max() <= 1e-8 * exact.max()
    # steady balance: the two walls carry the body force of the fluid
    mass, _, rho_a = sim.balance()
    F = sim.wall_force(-1)
    assert F[0] == pytest.approx(rho_a[0], rel=1e-8)
    assert F[0] == pytest.approx(g * mass, rel=1e-8)
    # too few steps allowed
    sim.rest()
    with pytest.raises(lbm.LbmError) as e:
        sim.run_steady(every=500, tol=1e-11, max_steps=2000)
    assert e.value.status == lbm.ERR_NOT_CONVERGED
    sim.close()


def test_nan_state_is_reported():
    cfg, mask = workloads.poiseuille(nx=40, ny=12, storage="f32")
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    f = sim.export_f().cpu().numpy()
    f[3, 0, 5, 17] = np.nan
    sim.import_f(f)
    sim.step(1)
    out = np.zeros(7)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_balance(sim.ctx, out, lbm.OUT_HOST, sim.stream)
    assert e.value.status == lbm.ERR_NAN and not np.isfinite(out[0])
    with pytest.raises(lbm.LbmError) as e:
        sim.residual(sim.velocity_buffer())
    assert e.value.status == lbm.ERR_NAN
    # a device output is written without a check
    dev = torch.zeros(7, dtype=torch.float64, device=sim.device)
    lbm.lbm_balance(sim.ctx, dev, lbm.OUT_DEVICE, sim.stream)
    assert not bool(torch.isfinite(dev[0]))
    sim.close()
