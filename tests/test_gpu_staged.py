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
