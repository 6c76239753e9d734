"""The staged step kernel (bulk asynchronous copies of each tile's source
rows into shared memory) against the register-tiled kernel: both run the
same node arithmetic and the same stochastic-rounding stream, so after any
number of steps their stored states must be identical bit for bit.  Cases:
16-bit (nearest and stochastic rounding) and FP32 storage, D3Q19 and D2Q9,
rows whose length is not a multiple of the pair, vector or 64-node pitch,
y extents that are not a multiple of the tile rows, solids that send chunks
to the node-by-node path, a single-node box and a box of thousands of tiles.
The oracle parity of the staged kernel is covered by every periodic 16-bit
and FP32 case of the parity tests (it is the default kernel there)."""
import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import inputs, lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()


def _box(name):
    if name == "sphere3d":       # several tiles per plane, scattered boundary chunks
        nx, ny, nz = 256, 24, 20
        mask = inputs.sphere_mask(nx, ny, nz, (60.3, 11.2, 9.6), 6.7, wall=1)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, tau=0.68, g=(3e-5, 1e-6, -2e-6)), mask
    if name == "ragged3d":       # nx = 50: padded rows; ny = 13 not a multiple of the 8 tile rows
        nx, ny, nz = 50, 13, 11
        mask = inputs.sphere_mask(nx, ny, nz, (21.3, 6.2, 5.4), 3.3, wall=1)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, tau=0.66, g=(2e-4, -1e-4, 5e-5)), mask
    if name == "many_tiles":     # 3,072 tiles
        nx, ny, nz = 128, 64, 48
        mask = inputs.sphere_mask(nx, ny, nz, (40.5, 30.2, 20.7), 8.4, wall=1)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, tau=0.7, g=(1e-4, 0, 0)), mask
    if name == "odd2d":          # D2Q9, nx = 203 (odd), random solids
        nx, ny = 203, 37
        mask = inputs.random_solids(nx, ny, 1, 0.05, n_walls=1, seed=19)
        return dict(lattice=9, nx=nx, ny=ny, nz=1, tau=0.74, g=(3e-4, 1e-4, 0)), mask
    if name == "long2d":         # one tile row of 1,024 nodes: two tasks per consumer warp
        nx, ny = 1024, 9
        mask = inputs.cylinder_mask(nx, ny, (300.2, 4.1), 2.6, wall=1)
        return dict(lattice=9, nx=nx, ny=ny, nz=1, tau=0.9, g=(1e-4, 0, 0)), mask
    if name == "single":         # one node
        mask = inputs.empty_mask(1, 1, 1)
        return dict(lattice=19, nx=1, ny=1, nz=1, tau=0.9, g=(1e-3, 2e-3, 3e-3)), mask
    raise KeyError(name)


def _raw_after(cfg, mask, f0, steps, kernel):
    sim = lbm.Sim(dict(cfg, step_kernel=kernel), mask)
    sim.import_f(f0)
    sim.step(steps)
    raw = torch.empty(sim.sizes[lbm.BUF_POP_A], dtype=torch.uint8, device=sim.device)
    lbm.lbm_save_state(sim.ctx, raw, sim.stream)
    status = sim.device_status()
    f = sim.export_f().cpu().numpy()
    sim.close()
    return raw.cpu(), f, status


@pytest.mark.parametrize("storage,rounding", [("f16s", "nearest"), ("f16s", "stochastic"), ("bf16s", "stochastic"),
                                              ("bf16s", "nearest"), ("f32", "nearest")])
@pytest.mark.parametrize("name", ["sphere3d", "ragged3d", "many_tiles", "odd2d", "long2d", "single"])
def test_staged_equals_register_kernel(orc, name, storage, rounding):
    base, mask = _box(name)
    cfg = dict(base, periodic=(1, 1, 1), force_model="e", storage=storage, rounding=rounding, seed=31,
               wall_u=((0, 0, 0),))
    nz, ny, nx = mask.shape
    D = 2 if cfg["lattice"] == 9 else 3
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, u_amplitude=0.04, seed=4)
    f0 = orc.init(ocfg, mask, rho, u, inputs.noise(cfg["lattice"], nx, ny, nz, 1e-3, seed=6))
    a, fa, sa = _raw_after(cfg, mask, f0, 9, "staged")
    b, fb, sb = _raw_after(cfg, mask, f0, 9, "register")
    assert sa == 0 and sb == 0
    nxp = (nx + 63) // 64 * 64
    n = cfg["lattice"] * nxp * ny * nz * (4 if storage == "f32" else 2)
    assert torch.equal(a[:n], b[:n])
    assert np.array_equal(fa, fb)
    assert np.all(np.isfinite(fa))


@pytest.mark.parametrize("storage,rounding", [("f16s", "stochastic"), ("bf16s", "nearest"), ("f32", "nearest")])
def test_step_force_fused_in_the_staged_step(orc, storage, rounding):
    """lbm_step_force on the staged kernel: the wall force of the step before
    it, summed inside the step kernel, equals lbm_wall_force called before
    lbm_step to rounding (FP64 sums in another fixed order), for one wall,
    another and every wall, with and without the moving-wall correction, to
    host and device outputs; the populations stepped are bit for bit those of
    the plain step."""
    nx, ny, nz = 96, 40, 24
    mask = inputs.sphere_mask(nx, ny, nz, (30.2, 19.6, 11.3), 5.2, wall=1)
    mask = np.where(inputs.sphere_mask(nx, ny, nz, (70.7, 12.1, 13.0), 4.1, wall=2) > 0, 2, mask).astype(np.uint8)
    cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.7, force_model="e", g=(2e-5, 0, 0),
               storage=storage, rounding=rounding, seed=11, wall_u=((0, 0, 0), (0.01, -0.02, 0.005)),
               step_kernel="staged")
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=3, u_amplitude=0.03, seed=3)
    f0 = orc.init(ocfg, mask, rho, u, inputs.noise(19, nx, ny, nz, 1e-3, seed=2))
    a = lbm.Sim(cfg, mask)
    b = lbm.Sim(cfg, mask)
    a.import_f(f0)
    b.import_f(f0)
    assert a.step_kernel == "staged"
    a.step(1)
    b.step(1)
    scale = np.abs(a.wall_force(-1)).max()
    for wall, flags in [(1, 0), (2, lbm.MOVING_CORR), (-1, 0), (-1, lbm.MOVING_CORR), (2, 0)]:
        ref = a.wall_force(wall, flags)
        a.step(1)
        got = np.zeros(3)
        lbm.lbm_step_force(b.ctx, wall, flags, 1.0, got, lbm.OUT_HOST, b.stream)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (wall, flags, got, ref)
    # device output with accumulation, over three steps
    acc = torch.zeros(3, dtype=torch.float64, device=b.device)
    ref = np.zeros(3)
    for _ in range(3):
        ref += 0.5 * a.wall_force(-1)
        a.step(1)
        lbm.lbm_step_force(b.ctx, -1, lbm.ACCUMULATE, 0.5, acc, lbm.OUT_DEVICE, b.stream)
    assert np.abs(acc.cpu().numpy() - ref).max() <= 1e-12 * scale
    assert b.time == a.time
    assert np.array_equal(a.export_f().cpu().numpy(), b.export_f().cpu().numpy())
    assert a.device_status() == 0 and b.device_status() == 0


def test_step_force_on_the_register_kernel(orc):
    """Without the staged kernel lbm_step_force is lbm_wall_force then
    lbm_step: the same values and the same state."""
    cfg, mask = workloads.poiseuille(nx=70, ny=20, storage="f32")
    a, b = lbm.Sim(cfg, mask), lbm.Sim(cfg, mask)
    for s in (a, b):
        s.rest()
        s.step(2)
    assert b.step_kernel == "register"
    for _ in range(3):
        ref = a.wall_force(1)
        a.step(1)
        got = np.zeros(3)
        lbm.lbm_step_force(b.ctx, 1, 0, 1.0, got, lbm.OUT_HOST, b.stream)
        assert np.array_equal(got, ref)
    assert np.array_equal(a.export_f().cpu().numpy(), b.export_f().cpu().numpy())


def _closed_box(name):
    if name == "cavity_les":       # every face closed, lid moving, Smagorinsky LES
        n = 40
        return dict(lattice=19, nx=n, ny=n, nz=n, periodic=(0, 0, 0), tau=0.55, force_model="e", les=1, cs=0.1,
                    wall_u=((0, 0, 0), (0.1, 0, 0)), face_wall=(1, 1, 1, 1, 1, 2)), inputs.empty_mask(n, n, n)
    if name == "closed_x_moving":  # every face closed, moving x and y faces, solids, body force, no EXT
        nx, ny, nz = 70, 13, 11
        mask = inputs.random_solids(nx, ny, nz, 0.01, n_walls=1, seed=17)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(0, 0, 0), tau=0.62, force_model="e",
                    g=(1e-4, -5e-5, 2e-5), wall_u=((0, 0, 0), (0.0, 0.03, 0.01), (0.0, -0.02, 0.02)),
                    face_wall=(2, 3, 1, 2, 3, 1)), mask
    if name == "mhd_channel":      # periodic x and y, closed z, Lorentz + Maxwell + LES
        nx, ny, nz = 64, 9, 12
        mask = inputs.random_solids(nx, ny, nz, 0.01, n_walls=1, seed=5)
        mask[mask > 0] = 2
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), tau=0.6, force_model="c",
                    g=(5e-5, 0, 1e-5), lorentz=1, B=(0.1, -0.05, 0.2), E=(1e-3, 0, 0), sigma_e=0.4, maxwell=1,
                    mu=1.2, les=1, cs=0.16, wall_u=((0.02, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 1, 1, 1)), mask
    if name == "channel_2d":       # D2Q9, closed y with a moving top wall, periodic x, odd nx
        nx, ny = 131, 24
        return dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=(1, 0, 1), tau=0.8, force_model="d", g=(1e-4, 0, 0),
                    wall_u=((0, 0, 0), (0.05, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1)), inputs.empty_mask(nx, ny)
    if name == "les_periodic_c":   # periodic box with a sphere, LES alone with model [c] and a body force
        nx, ny, nz = 64, 12, 10
        mask = inputs.sphere_mask(nx, ny, nz, (30.6, 5.9, 4.7), 2.9, wall=1)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.56, force_model="c",
                    g=(2e-4, -1e-4, 5e-5), les=1, cs=0.14, wall_u=((0, 0, 0),)), mask
    if name == "brinkman_periodic":  # periodic box, linear equilibrium and Darcy resistance (EXT)
        nx, ny, nz = 64, 12, 10
        mask = inputs.sphere_mask(nx, ny, nz, (20.3, 6.1, 5.2), 3.1, wall=1)
        return dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=0.7, force_model="e",
                    g=(1e-4, 0, 0), stokes=1, darcy=1e-3, wall_u=((0, 0, 0),)), mask
    raise KeyError(name)


@pytest.mark.parametrize("storage,rounding", [("f16s", "stochastic"), ("bf16s", "nearest"), ("f32", "nearest")])
@pytest.mark.parametrize("name", ["cavity_les", "closed_x_moving", "mhd_channel", "channel_2d", "brinkman_periodic",
                                  "les_periodic_c"])
def test_staged_closed_faces_and_ext_equal_register(orc, name, storage, rounding):
    """The staged kernel with closed box faces (rows outside a closed face
    replaced by the node's own opposite populations, the x-face values staged
    by the producer, Ladd's term of moving faces) and with the EXT node code
    (LES, Lorentz force, Maxwell term, linear equilibrium, Darcy) stores the
    register-tiled kernel's bits (LES alone with 16-bit storage runs the
    FP32x2 LES pair code in both)."""
    base, mask = _closed_box(name)
    cfg = dict(base, storage=storage, rounding=rounding, seed=23)
    nz, ny, nx = mask.shape
    D = 2 if cfg["lattice"] == 9 else 3
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    rho, u = inputs.smooth_fields(nx, ny, nz, dims=D, u_amplitude=0.04, seed=4)
    f0 = orc.init(ocfg, mask, rho, u, inputs.noise(cfg["lattice"], nx, ny, nz, 1e-3, seed=6))
    a, fa, sa = _raw_after(cfg, mask, f0, 7, "staged")
    b, fb, sb = _raw_after(cfg, mask, f0, 7, "register")
    assert sa == 0 and sb == 0
    nxp = (nx + 63) // 64 * 64
    n = cfg["lattice"] * nxp * ny * nz * (4 if storage == "f32" else 2)
    assert torch.equal(a[:n], b[:n])
    assert np.array_equal(fa, fb)
    # and the oracle's state within the storage bound of the parity tests
    tol = {"f32": 2e-6, "f16s": 1e-4, "bf16s": 1e-3}[storage]
    ref = orc.run(ocfg, mask, f0, 7)
    assert np.abs(fa - ref).max() / np.abs(ref).max() < tol
