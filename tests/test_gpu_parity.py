"""CUDA path against the FP64 CPU oracle, element by element, through the C ABI.

Sizes span several 64-node rows and vector chunks with a ragged tail; every
force model, moving walls, scattered solids, the Lorentz force, the Maxwell
equilibrium and LES are covered; non-unit dx and dt.

Tolerances: FP64 populations within 1e-12 of max|f| (the FP64 requirement);
the FP32 compute paths within bounds derived from the storage rounding
(relative half-ulp u of the stored deviation d ~ 1e-2 f, accumulated over
the steps): FP32 u = 6e-8, binary16 (scaled) u = 4.9e-4, bfloat16 u = 3.9e-3.
"""
import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import inputs, lbm, workloads

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6, "f16s": 1e-4, "bf16s": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()
    assert torch.cuda.is_available()


def _case(name, model="e", storage="f64"):
    if name == "d2q9":
        nx, ny, nz = 70, 37, 1
        mask = inputs.random_solids(nx, ny, nz, 0.06, n_walls=1, seed=21)
        mask[mask > 0] = 3
        cfg = dict(lattice=9, nx=nx, ny=ny, nz=nz, periodic=(1, 0, 1), dx=0.5, dt=0.2, tau=0.74,
                   force_model=model, g=(2e-3, -1e-3, 0), storage=storage,
                   wall_u=((0.01, 0, 0), (-0.02, 0.0, 0), (0.0, 0.0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    elif name == "d2q9_mhd":
        nx, ny, nz = 66, 29, 1
        mask = inputs.cylinder_mask(nx, ny, (20.5, 14.2), 5.3, wall=3)
        cfg = dict(lattice=9, nx=nx, ny=ny, nz=nz, periodic=(1, 0, 1), dx=1.0, dt=1.0, tau=0.81,
                   force_model=model, g=(1e-4, 0, 0), lorentz=1, B=(0.05, 0.2, 0.0), E=(0, 0, 1e-3),
                   sigma_e=0.3, maxwell=1, mu=0.9, storage=storage,
                   wall_u=((0, 0, 0), (0.03, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    elif name == "d3q19":
        nx, ny, nz = 21, 13, 11
        mask = inputs.sphere_mask(nx, ny, nz, (9.3, 6.1, 5.2), 3.1, wall=3)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 0, 0), dx=0.5, dt=0.25, tau=0.7,
                   force_model=model, g=(1e-2, 2e-3, -1e-3), storage=storage,
                   wall_u=((0.0, 0.01, 0.0), (0.02, 0.0, -0.01), (0, 0, 0)), face_wall=(1, 1, 1, 2, 2, 1))
    elif name == "d3q19_ext":
        nx, ny, nz = 67, 9, 8
        mask = inputs.random_solids(nx, ny, nz, 0.05, n_walls=1, seed=5)
        mask[mask > 0] = 2
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), dx=1.0, dt=1.0, tau=0.6,
                   force_model=model, g=(5e-5, 0, 1e-5), lorentz=1, B=(0.1, -0.05, 0.2), E=(1e-3, 0, 0),
                   sigma_e=0.4, maxwell=1, mu=1.2, les=1, cs=0.16, storage=storage,
                   wall_u=((0.02, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 1, 1, 1))
    elif name == "cavity":
        n = 19
        mask = inputs.empty_mask(n, n, n)
        cfg = dict(lattice=19, nx=n, ny=n, nz=n, periodic=(0, 0, 0), tau=0.55, force_model=model, les=1, cs=0.1,
                   storage=storage, wall_u=((0, 0, 0), (0.1, 0, 0)), face_wall=(1, 1, 1, 1, 1, 2))
    elif name == "closed_x":   # every face closed, moving x faces, no LES: the vector path's x-face bounce
        nx, ny, nz = 37, 9, 7
        mask = inputs.random_solids(nx, ny, nz, 0.03, n_walls=1, seed=17)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(0, 0, 0), tau=0.62, force_model=model,
                   g=(1e-4, -5e-5, 2e-5), storage=storage,
                   wall_u=((0, 0, 0), (0.0, 0.03, 0.01), (0.0, -0.02, 0.02)), face_wall=(2, 3, 1, 1, 1, 1))
    elif name == "periodic_ragged":   # fully periodic D3Q19, ragged x, last warp of chunks half full
        nx, ny, nz = 50, 13, 11
        mask = inputs.sphere_mask(nx, ny, nz, (21.3, 6.2, 5.4), 3.3, wall=1)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.66, force_model=model,
                   g=(2e-4, -1e-4, 5e-5), storage=storage, wall_u=((0, 0, 0),))
    elif name == "periodic_multi":    # a box of 3072 blocks of chunks
        nx, ny, nz = 128, 64, 48
        mask = inputs.sphere_mask(nx, ny, nz, (40.5, 30.2, 20.7), 8.4, wall=1)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.7, force_model=model,
                   g=(1e-4, 0, 0), storage=storage, wall_u=((0, 0, 0),))
    elif name == "periodic_2d":       # fully periodic D2Q9 with a cylinder, ragged x
        nx, ny = 203, 37
        mask = inputs.cylinder_mask(nx, ny, (60.4, 18.3), 7.1, wall=1)
        cfg = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=(1, 1, 1), tau=0.74, force_model=model,
                   g=(3e-4, 1e-4, 0), storage=storage, wall_u=((0, 0, 0),))
    elif name == "column":     # nx = 1: every chunk is mostly padding
        mask = inputs.empty_mask(1, 24)
        cfg = dict(lattice=9, nx=1, ny=24, nz=1, periodic=(1, 0, 1), tau=0.9, force_model=model, g=(1e-4, 0, 0),
                   storage=storage, wall_u=((0, 0, 0), (0.05, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    elif name == "single":     # one periodic node
        mask = inputs.empty_mask(1, 1, 1)
        cfg = dict(lattice=19, nx=1, ny=1, nz=1, periodic=(1, 1, 1), tau=0.9, force_model=model,
                   g=(1e-3, 2e-3, 3e-3), storage=storage)
    elif name == "wide":       # several warps per row, exact multiple of 64
        mask = inputs.empty_mask(256, 6)
        cfg = dict(lattice=9, nx=256, ny=6, nz=1, periodic=(1, 1, 1), tau=0.6, force_model=model,
                   g=(1e-4, 3e-5, 0), storage=storage)
    elif name == "ultrawide":  # rows too long for shared-memory staging: register-tiled kernel
        nx, ny, nz = 4100, 3, 2
        mask = inputs.random_solids(nx, ny, nz, 0.02, n_walls=1, seed=13)
        cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), tau=0.8, force_model=model,
                   g=(1e-4, 0, 0), storage=storage, wall_u=((0.01, 0, 0),), face_wall=(1, 1, 1, 1, 1, 1))
    else:
        raise KeyError(name)
    return cfg, mask


def _initial(orc, cfg, mask, amp=1e-3):
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    nz, ny, nx = mask.shape
    D = 2 if cfg["lattice"] == 9 else 3
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, u_amplitude=0.04, seed=8)
    c = cfg.get("dx", 1.0) / cfg.get("dt", 1.0)
    f0 = orc.init(ocfg, mask, rho, u * c, inputs.noise(cfg["lattice"], nx, ny, nz, amp, seed=9))
    return ocfg, f0, rho, u * c


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


CASES = [("d2q9", m) for m in "abcde"] + [("d3q19", m) for m in "abcde"] + [
    ("d2q9_mhd", "d"), ("d2q9_mhd", "e"), ("d3q19_ext", "c"), ("d3q19_ext", "e"), ("cavity", "e"), ("closed_x", "e"),
    ("column", "b"), ("single", "c"), ("wide", "a"), ("ultrawide", "d")]


@pytest.mark.parametrize("name,model", CASES)
def test_populations_fp64(orc, name, model):
    cfg, mask = _case(name, model)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    # the round trip import -> export is exact up to the Ladd term's rounding
    assert _rel(sim.export_f().cpu().numpy(), f0) < 1e-15
    steps = 25
    sim.step(steps)
    f_ref = orc.run(ocfg, mask, f0, steps)
    assert sim.time == steps
    assert _rel(sim.export_f().cpu().numpy(), f_ref) < TOL["f64"]
    assert sim.device_status() == 0


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("name,model", [("d2q9", "d"), ("d3q19", "e"), ("d3q19_ext", "c"), ("cavity", "e"),
                                        ("ultrawide", "b")])
def test_populations_reduced_precision(orc, name, model, storage):
    cfg, mask = _case(name, model, storage)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    steps = 10
    sim.step(steps)
    f_ref = orc.run(ocfg, mask, f0, steps)
    err = _rel(sim.export_f().cpu().numpy(), f_ref)
    assert err < TOL[storage], err


@pytest.mark.parametrize("storage", ["f32", "f16s"])
@pytest.mark.parametrize("model", "abcde")
@pytest.mark.parametrize("name", ["d2q9", "d3q19", "closed_x"])
def test_force_models_fp32_paths(orc, name, model, storage):
    """Every force model through the FP32 node-pair path (uniform body force,
    moving closed faces on y/z, and on x for closed_x)."""
    cfg, mask = _case(name, model, storage)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    steps = 10
    sim.step(steps)
    f_ref = orc.run(ocfg, mask, f0, steps)
    err = _rel(sim.export_f().cpu().numpy(), f_ref)
    assert err < TOL[storage], err


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("model", "abcde")
@pytest.mark.parametrize("name", ["d2q9", "d3q19", "periodic_ragged"])
def test_les_with_body_force_every_model(orc, name, model, storage):
    """Smagorinsky LES with a uniform body force and no other EXT term, every
    force model: 16-bit storage takes the FP32x2 pair code specialised for
    LES (per-node relaxation rate, C and, for model [c], u^F), FP32 storage
    the EXT node code (in pairs where a box face is closed), FP64 the scalar
    EXT code; each against the oracle."""
    cfg, mask = _case(name, model, storage)
    cfg = dict(cfg, les=1, cs=0.18)
    ocfg, f0, _, _ = _initial(orc, cfg, mask, amp=3e-3)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    steps = 10
    sim.step(steps)
    f_ref = orc.run(ocfg, mask, f0, steps)
    err = _rel(sim.export_f().cpu().numpy(), f_ref)
    assert err < TOL[storage], err
    assert sim.device_status() == 0


@pytest.mark.parametrize("name,model", [("d2q9", "e"), ("d2q9_mhd", "d"), ("d3q19", "c"), ("d3q19_ext", "e")])
def test_init_equilibrium_matches_oracle(orc, name, model):
    cfg, mask = _case(name, model)
    ocfg, f0, rho, u = _initial(orc, cfg, mask)
    nz, ny, nx = mask.shape
    xi = inputs.noise(cfg["lattice"], nx, ny, nz, 1e-3, seed=9)
    sim = lbm.Sim(cfg, mask)
    sim.init_equilibrium(rho, u, xi)                       # host arrays
    assert _rel(sim.export_f().cpu().numpy(), f0) < 1e-14
    sim.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(),
                         torch.from_numpy(xi).cuda())      # device arrays
    assert _rel(sim.export_f().cpu().numpy(), f0) < 1e-14


@pytest.mark.parametrize("name,model", [("d2q9", "b"), ("d2q9_mhd", "e"), ("d3q19", "d"), ("d3q19_ext", "c"),
                                        ("cavity", "e")])
def test_wall_force_stress_balance_fp64(orc, name, model):
    cfg, mask = _case(name, model)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    K = 7
    sim.step(K)
    f_prev = orc.run(ocfg, mask, f0, K - 1)                # f(K-1)
    f_K, frel = orc.step(ocfg, mask, f_prev)               # f(K), f^rel(K-1)
    walls = sorted(set(range(1, len(cfg.get("wall_u", ())) + 1)))
    for wall in walls + [-1]:
        for flags in (0, 1, 2, 3):
            Fg = sim.wall_force(wall, flags)
            Fo = orc.wall_force(ocfg, mask, frel, f_K, wall, flags)
            scale = max(np.abs(orc.wall_force(ocfg, mask, frel, f_K, -1, 0)).max(), 1e-30)
            assert np.abs(Fg - Fo).max() < 1e-12 * scale, (wall, flags, Fg, Fo)
    for variant in (1, 2, 3, 4):
        sg, Sg, rg, vg = [x.cpu().numpy() for x in sim.stress(variant)]
        so, So, ro, vo = orc.stress(ocfg, mask, f_K if variant <= 2 else f_prev, frel, f_K, variant)
        assert _rel(sg, so) < 1e-10, variant
        assert _rel(Sg, So) < 1e-10, variant
        assert _rel(rg, ro) < 1e-14, variant
        assert _rel(vg, vo) < 1e-11, variant
    mg, Mg, bg = sim.balance()
    mo, Mo, bo = orc.balance(ocfg, mask, f_K)
    assert abs(mg - mo) < 1e-13 * mo
    assert np.abs(Mg - Mo).max() < 1e-12 * mo * ocfg.dx / ocfg.dt
    assert np.abs(bg - bo).max() < 1e-12 * max(np.abs(bo).max(), 1e-30)


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("name,model", [("d2q9", "b"), ("d2q9_mhd", "e"), ("d3q19", "d"), ("d3q19_ext", "c"),
                                        ("cavity", "e"), ("periodic_ragged", "e")])
def test_stress_reduced_precision(orc, name, model, storage):
    """Stress variants S1-S4 of the FP32-compute paths against the FP64
    oracle, node by node.  The stored populations differ from the oracle's
    by at most TOL[storage] max|f| (the population bound above); the second
    moment sums Q of them times c^2, so each stress component is within
    Q TOL max|f| c^2, the strain rate S = sigma/(2 rho nu) within that over
    2 rho_min nu, the density within Q TOL max|f| and the velocity within
    Q TOL max|f| c / rho_min.  (The FP32 arithmetic itself adds ~1e-7 of
    the moment scale, far below these bounds.)"""
    cfg, mask = _case(name, model, storage)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    K = 7
    sim.step(K)
    f_prev = orc.run(ocfg, mask, f0, K - 1)
    f_K, frel = orc.step(ocfg, mask, f_prev)
    Q = cfg["lattice"]
    c = cfg.get("dx", 1.0) / cfg.get("dt", 1.0)
    fmax = np.abs(f_K).max()
    tol = Q * TOL[storage] * fmax
    nu = cfg.get("dt", 1.0) * c * c * (cfg["tau"] - 0.5) / 3
    fluid = mask == 0
    worst = {}
    for variant in (1, 2, 3, 4):
        sg, Sg, rg, vg = [x.cpu().numpy().astype(np.float64) for x in sim.stress(variant)]
        so, So, ro, vo = orc.stress(ocfg, mask, f_K if variant <= 2 else f_prev, frel, f_K, variant)
        rmin = ro[fluid].min()
        e_sig = np.abs(sg - so).max() / (c * c)
        e_S = np.abs(Sg - So).max() * 2 * rmin * nu / (c * c)
        e_rho = np.abs(rg - ro).max()
        e_v = np.abs(vg - vo).max() * rmin / c
        worst[variant] = e_sig / fmax
        assert e_sig <= tol, (variant, e_sig, tol)
        assert e_S <= tol * (1 + 1e-6) + 1e-7 * fmax, (variant, e_S, tol)
        assert e_rho <= tol, (variant, e_rho, tol)
        assert e_v <= tol, (variant, e_v, tol)
        assert np.all(sg[:, ~fluid] == 0) and np.all(Sg[:, ~fluid] == 0)
    print(f"stress error / (c^2 max|f|), {name} {storage}:", {k: f"{v:.2e}" for k, v in worst.items()})


@pytest.mark.parametrize("name,model", [("d2q9", "a"), ("d3q19", "e"), ("d3q19_ext", "d")])
def test_exact_momentum_balance_on_gpu(orc, name, model):
    """Every step: F_wall = sum rho a - [M(t+dt) - M(t)]/dt (FP64 path)."""
    cfg, mask = _case(name, model)
    _, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    dt = cfg.get("dt", 1.0)
    for _ in range(5):
        _, M0, ba = sim.balance()
        sim.step(1)
        _, M1, _ = sim.balance()
        F = sim.wall_force(-1, 0)
        ref = ba - (M1 - M0) / dt
        scale = np.abs(M0).max() / dt + np.abs(F).max()
        assert np.abs(F - ref).max() < 1e-13 * scale


def test_state_errors(orc):
    cfg, mask = _case("d2q9", "e")
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    with pytest.raises(lbm.LbmError) as e:
        sim.wall_force(1)
    assert e.value.status == 6
    with pytest.raises(lbm.LbmError) as e:
        sim.stress(3)
    assert e.value.status == 6
    sim.step(1)
    sim.stress(3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(sim.ctx, -1, sim.stream)
    assert e.value.status == 1


def test_all_solid_domain():
    mask = np.ones((1, 8, 70), np.uint8)
    cfg = dict(lattice=9, nx=70, ny=8, nz=1, periodic=(1, 1, 1), tau=0.8, force_model="e", g=(1e-3, 0, 0),
               wall_u=((0, 0, 0),))
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(3)
    assert np.all(sim.export_f().cpu().numpy() == 0)
    assert np.all(sim.wall_force(-1) == 0)
    m, M, b = sim.balance()
    assert m == 0 and np.all(M == 0) and np.all(b == 0)


@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("name,model", [("periodic_ragged", "e"), ("periodic_ragged", "c"), ("periodic_multi", "e"),
                                        ("periodic_2d", "d"), ("periodic_2d", "a")])
def test_periodic_16bit_against_oracle(orc, name, model, storage, rounding):
    """16-bit storage in fully periodic boxes (the benchmark's kind of box):
    rows whose length is not a multiple of the vector width, a last warp of
    chunks half full, and a box of many thousand blocks."""
    cfg, mask = _case(name, model, storage)
    cfg = dict(cfg, rounding=rounding, seed=77)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    steps = 6
    sim.step(steps)
    f_ref = orc.run(ocfg, mask, f0, steps)
    err = _rel(sim.export_f().cpu().numpy(), f_ref)
    assert err < TOL[storage], err


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_stochastic_rounding(orc, storage):
    """Stochastic rounding of 16-bit stores: within the same bound of the
    oracle as rounding to nearest, replayed bit for bit by lbm_step_from with
    the same step index, and dependent on the seed."""
    cfg, mask = _case("d3q19", "e", storage)
    cfg = dict(cfg, rounding="stochastic", seed=1234)
    ocfg, f0, _, _ = _initial(orc, cfg, mask)
    sim = lbm.Sim(cfg, mask)
    sim.import_f(f0)
    sim.step(3)
    saved = torch.empty(sim.sizes[lbm.BUF_POP_A], dtype=torch.uint8, device=sim.device)
    lbm.lbm_save_state(sim.ctx, saved, sim.stream)
    sim.step(7)
    f_ref = orc.run(ocfg, mask, f0, 10)
    assert _rel(sim.export_f().cpu().numpy(), f_ref) < TOL[storage]
    # replay step 3 from the saved state
    a = torch.empty_like(saved)
    lbm.lbm_step_from(sim.ctx, saved, a, 3, sim.stream)
    sim2 = lbm.Sim(cfg, mask)
    sim2.import_f(f0)
    sim2.step(4)
    b = torch.empty_like(saved)
    lbm.lbm_save_state(sim2.ctx, b, sim2.stream)
    torch.cuda.synchronize()
    # populations only (the buffer size is rounded up to 256 bytes)
    nxp = (cfg["nx"] + 63) // 64 * 64
    n = cfg["lattice"] * nxp * cfg["ny"] * cfg["nz"] * 2
    a, b = a[:n], b[:n]
    assert torch.equal(a, b)
    # another step index or seed gives other bits
    c = torch.empty_like(saved)
    lbm.lbm_step_from(sim.ctx, saved, c, 4, sim.stream)
    sim3 = lbm.Sim(dict(cfg, seed=99), mask)
    sim3.import_f(f0)
    sim3.step(4)
    e = torch.empty_like(saved)
    lbm.lbm_save_state(sim3.ctx, e, sim3.stream)
    torch.cuda.synchronize()
    assert not torch.equal(a, c[:n]) and not torch.equal(a, e[:n])
