"""GPU runs at the full sizes of the five synthetic configurations, checked
against the FP64 oracle where it can follow (full fields for a few steps),
the stored golden case, closed forms, and exact properties at any size."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import adjoint, inputs, lbm, workloads

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poiseuille_c1.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max())


def test_poiseuille_64x32_against_golden_and_closed_form():
    """64 x 32 channel, tau 0.8, g 1e-6, model [d], 10000 steps (FP64)."""
    cfg, mask = workloads.poiseuille()
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(10000)
    g = json.load(open(GOLDEN))
    o = g["oracle_after_10000_steps"]
    _, _, _, v = sim.stress(lbm.S2)
    vx = v[0, 0, :, 3].cpu().numpy()
    assert _rel(vx, o["v_x_profile"]) < 1e-11
    sig, _, _, _ = sim.stress(lbm.S2)
    assert _rel(sig[2, 0, :, 3].cpu().numpy(), o["sigma_xy_profile"]) < 1e-10
    # the x force is what is left of ~128 link terms of the size of the
    # pressure force (F_y = 21.3); compare on that scale
    for wall, key in ((1, "wall_force_bottom"), (2, "wall_force_top")):
        F, Fo = sim.wall_force(wall), np.array(o[key])
        assert np.abs(F - Fo).max() < 1e-11 * np.abs(Fo).max()
    # the profile is uniform in x
    v_all = v[0, 0].cpu().numpy()
    assert np.abs(v_all - v_all[:, :1]).max() < 1e-15


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_hartmann_256x128_closed_form(storage, tau):
    """Ha 10, moving lid 0.05, 50000 steps: cosh profile and wall shear within
    the halfway-bounce-back error at H = 64 (second order, see the oracle
    pins), and the exact steady balance of wall forces and body forces."""
    cfg, mask = workloads.hartmann(tau=tau, storage=storage)
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(50000)
    H, Ha, Uw = 64, 10.0, 0.05
    nu = (tau - 0.5) / 3
    K = nu * Ha ** 2 / H ** 2
    g = cfg["g"][0]
    m = Ha / H
    y = np.arange(128) - H + 0.5
    u = (g / K) * (1 - np.cosh(m * y) / np.cosh(m * H)) + Uw * np.sinh(m * (y + H)) / np.sinh(2 * m * H)
    dudy = lambda yy: (g / K) * (-m * np.sinh(m * yy) / np.cosh(m * H)) + Uw * m * np.cosh(m * (yy + H)) / np.sinh(2 * m * H)
    _, _, rho, v = sim.stress(lbm.S2)
    vx = v[0, 0, :, 100].cpu().numpy()
    assert _rel(vx, u) < 3e-3
    Fb, Ft = sim.wall_force(1), sim.wall_force(2)
    L = 256
    # the top wall's shear nearly cancels (Couette against pressure-driven
    # flow), so both walls are compared on the bottom wall's scale
    scale = abs(L * nu * dudy(-H))
    assert abs(Fb[0] - L * nu * dudy(-H)) < 3e-3 * scale
    assert abs(Ft[0] + L * nu * dudy(H)) < 3e-3 * scale
    _, _, body = sim.balance()
    imbalance = abs(Fb[0] + Ft[0] - body[0])
    if storage == "f64":
        assert imbalance < 1e-9 * abs(body[0])
    else:
        # a rounded fixed point conserves momentum per step only up to the
        # rounding of every stored deviation, N Q 2^-24 max|d|; the flow is
        # uniform in x, so the columns' rounding errors add coherently
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        d = sim.export_f().cpu().numpy()[:, 0] - w[:, None, None] * cfg.get("rho0", 1.0)
        bound = 256 * 128 * 9 * 2.0 ** -24 * np.abs(d).max()
        assert imbalance < bound


def test_hartmann_full_size_parity_and_maxwell_removal(orc):
    """256 x 128, 200 steps: FP64 fields match the oracle; with the Maxwell
    equilibrium (uniform B) the removed force equals the force without it."""
    cfg, mask = workloads.hartmann(tau=0.8, storage="f64")
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    f0 = orc.init(ocfg, mask, np.ones((1, 128, 256)), np.zeros((3, 1, 128, 256)))
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    sim.step(200)
    f_ref = orc.run(ocfg, mask, f0, 200)
    assert _rel(sim.export_f().cpu().numpy(), f_ref) < 1e-12
    cm = dict(cfg, maxwell=1)
    sm = lbm.Sim(cm, mask)
    sm.rest()
    sim.rest()
    sm.step(200)
    sim.step(200)
    for wall in (1, 2):
        F0, FR = sim.wall_force(wall), sm.wall_force(wall, lbm.MAXWELL_REMOVE)
        assert np.abs(FR - F0).max() < 1e-12 * np.abs(F0).max()


@pytest.mark.parametrize("storage,rounding,tol", [
    ("f64", "nearest", 1e-12), ("f32", "nearest", 2e-6), ("f16s", "nearest", 1e-4),
    ("f16s", "stochastic", 1e-4), ("bf16s", "stochastic", 1e-3)])
def test_sphere_256x128x128_against_oracle(orc, storage, rounding, tol):
    """The benchmark's workload and launch configuration: two full steps from a
    perturbed state against the oracle's full field, and the wall force."""
    cfg, mask = workloads.sphere(storage=storage)
    cfg = dict(cfg, rounding=rounding, seed=2024)
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    rho, u = inputs.smooth_fields(256, 128, 128, dims=3, u_amplitude=0.03, seed=4)
    f0 = orc.init(ocfg, mask, rho, u, inputs.noise(19, 256, 128, 128, 1e-3, seed=5))
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    sim.step(2)
    f1 = orc.run(ocfg, mask, f0, 1)
    f2, frel = orc.step(ocfg, mask, f1)
    assert _rel(sim.export_f().cpu().numpy(), f2) < tol
    F = sim.wall_force(1)
    Fo = orc.wall_force(ocfg, mask, frel, f2, 1, 0)
    scale = np.abs(orc.wall_force(ocfg, mask, frel, f2, -1, 0)).max() + np.abs(Fo).max()
    assert np.abs(F - Fo).max() < max(1e-12, 50 * tol) * scale
    assert sim.device_status() == 0


def test_sphere_full_size_momentum_balance():
    """Exact per-step balance F = sum rho a - dM/dt at 256 x 128 x 128 (FP64)."""
    cfg, mask = workloads.sphere(storage="f64")
    sim = lbm.Sim(cfg, mask)
    rho, u = inputs.smooth_fields(256, 128, 128, dims=3, u_amplitude=0.03, seed=4)
    sim.init_equilibrium(rho, u)
    for _ in range(3):
        _, M0, body = sim.balance()
        sim.step(1)
        _, M1, _ = sim.balance()
        F = sim.wall_force(-1)
        assert np.abs(F - (body - (M1 - M0))).max() < 1e-11 * (np.abs(M0).max() + np.abs(F).max())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 2e-6), ("f16s", 1e-4)])
def test_cavity_128_les_against_oracle(orc, storage, tol):
    """LES cavity 128^3 (lid 0.1, tau 0.55, Cs 0.1): two steps from a perturbed
    state against the oracle's full field."""
    cfg, mask = workloads.cavity(n=128, storage=storage)
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    rho, u = inputs.smooth_fields(128, 128, 128, dims=3, u_amplitude=0.05, seed=6)
    f0 = orc.init(ocfg, mask, rho, u, inputs.noise(19, 128, 128, 128, 1e-3, seed=7))
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    sim.step(2)
    assert _rel(sim.export_f().cpu().numpy(), orc.run(ocfg, mask, f0, 2)) < tol


def test_cavity_512_properties():
    """512^3 LES cavity with binary16 storage and stochastic rounding, 50 steps:
    finite, mass conserved to the storage rounding, lid force along the lid."""
    cfg, mask = workloads.cavity(n=512, storage="f16s")
    cfg = dict(cfg, rounding="stochastic", seed=3)
    sim = lbm.Sim(cfg, mask, stage=False)
    sim.init_equilibrium(torch.ones((512, 512, 512), dtype=torch.float64, device="cuda"),
                         torch.zeros((3, 512, 512, 512), dtype=torch.float64, device="cuda"))
    m0, _, _ = sim.balance()
    sim.step(50)
    m1, M, _ = sim.balance()
    assert np.isfinite(m1) and np.all(np.isfinite(M))
    assert abs(m1 / m0 - 1) < 1e-6
    F = sim.wall_force(2)
    assert np.all(np.isfinite(F)) and F[0] < 0     # the fluid holds the lid back
    assert sim.device_status() == 0


def test_sphere_128_adjoint_vs_central_differences():
    """D3Q19 128^3 sphere r 10, T 2000, FP32 forward and adjoint with FP64
    reductions, against central differences of the FP64 forward."""
    T = 2000
    c32, mask = workloads.sphere_small(storage="f32")
    c64 = dict(c32, storage="f64")
    theta = np.array(list(c32["g"]) + [0.0, 0.0, 0.0])
    p32 = adjoint.DragProblem(lbm.Sim(c32, mask), T, 1)
    p32.forward(theta)
    g32 = p32.backward()
    del p32
    torch.cuda.empty_cache()
    p64 = adjoint.DragProblem(lbm.Sim(c64, mask), T, 1, stride=T // 4)
    fd = np.zeros(6)
    for k in (0, 1, 3):
        h = 1e-3 * (abs(theta[k]) if theta[k] else 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (p64.forward(tp) - p64.forward(tm)) / (2 * h)
    for k in (0, 1, 3):
        assert abs(g32[k] - fd[k]) <= 1e-4 * np.abs(fd).max(), (k, g32, fd)
