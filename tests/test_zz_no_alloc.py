"""lbm_wall_force_noalloc, through the C ABI, against lbm_wall_force.

The entry point serves callers that cannot allocate device memory when they
need a force: its partial sums live in a static array inside the library
instead of a caller buffer.  Its results must equal those of lbm_wall_force
(same launch shape and reduction order) on consecutive calls, for host and
device outputs, every wall and every flag, at link counts that fit one pass
of the reduction grid and at counts where every thread sums several links,
and it must refuse requests beyond its fixed capacity.  This file is collected last on purpose.
"""
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


def _compare(sim, walls, flag_sets):
    st = sim.stream
    for wall in walls:
        for flags in flag_sets:
            ref = np.zeros(3)
            lbm.lbm_wall_force(sim.ctx, wall, flags, 1.0, ref, 1, st)
            for _ in range(2):                          # two calls in a row
                got = np.zeros(3)
                lbm.lbm_wall_force_noalloc(sim.ctx, wall, flags, 1.0, got, 1, st)
                assert np.array_equal(got, ref), (wall, flags, got, ref)
            dev = torch.zeros(3, dtype=torch.float64, device=sim.device)
            lbm.lbm_wall_force_noalloc(sim.ctx, wall, flags | lbm.ACCUMULATE, 0.5, dev, 0, st)
            lbm.lbm_wall_force_noalloc(sim.ctx, wall, flags | lbm.ACCUMULATE, 0.5, dev, 0, st)
            assert np.allclose(dev.cpu().numpy(), ref, rtol=1e-15, atol=1e-300)


@pytest.mark.parametrize("storage", ["f64", "f16s"])
def test_noalloc_matches_wall_force(storage):
    cfg, mask = workloads.sphere(nx=48, ny=40, nz=36, radius=7, center=(20.3, 19.6, 18.1), storage=storage)
    cfg = dict(cfg, periodic=(1, 0, 1), face_wall=(1, 1, 2, 3, 1, 1),
               wall_u=((0, 0, 0), (0.02, 0, 0), (0, 0, 0.01)), maxwell=1, B=(0.02, 0.05, 0.0))
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(5)
    _compare(sim, [1, 2, 3, -1], [0, lbm.MOVING_CORR, lbm.MAXWELL_REMOVE, 3])
    sim.step(3)
    _compare(sim, [1, -1], [0])


def test_noalloc_matches_wall_force_on_a_capped_grid():
    # 3 * 100,000 = 300,000 links on the bottom wall: more links than one
    # pass of the 1024-block grid covers, so every thread of both entry
    # points sums several links; the results must still agree bit for bit
    nx = 100_000
    cfg, mask = workloads.poiseuille(nx=nx, ny=4, storage="f32")
    cfg = dict(cfg, wall_u=((0.01, 0, 0), (0, 0, 0)))
    sim = lbm.Sim(cfg, mask)
    rho, u = inputs.smooth_fields(nx, 4, 1, dims=2, u_amplitude=0.03, seed=3)
    sim.init_equilibrium(rho, u)
    sim.step(2)
    n1 = sim.link_count(1)
    assert 262_144 < n1 <= 1_048_576
    st = sim.stream
    for flags in (0, lbm.MOVING_CORR):
        ref = np.zeros(3)
        lbm.lbm_wall_force(sim.ctx, 1, flags, 1.0, ref, 1, st)
        for _ in range(2):
            got = np.zeros(3)
            lbm.lbm_wall_force_noalloc(sim.ctx, 1, flags, 1.0, got, 1, st)
            assert np.array_equal(got, ref), (flags, got, ref)
        ref_dev = torch.zeros(3, dtype=torch.float64, device=sim.device)
        got_dev = torch.zeros(3, dtype=torch.float64, device=sim.device)
        lbm.lbm_wall_force(sim.ctx, 1, flags, 0.25, ref_dev, 0, st)
        lbm.lbm_wall_force_noalloc(sim.ctx, 1, flags, 0.25, got_dev, 0, st)
        assert torch.equal(got_dev, ref_dev)
        for _ in range(2):
            lbm.lbm_wall_force(sim.ctx, 1, flags | lbm.ACCUMULATE, 0.5, ref_dev, 0, st)
            lbm.lbm_wall_force_noalloc(sim.ctx, 1, flags | lbm.ACCUMULATE, 0.5, got_dev, 0, st)
        assert torch.equal(got_dev, ref_dev)


def test_noalloc_refuses_more_links_than_it_holds():
    # a 2-D channel whose bottom wall has 3 * 400,000 > 1,048,576 links
    nx = 400_000
    cfg, mask = workloads.poiseuille(nx=nx, ny=4, storage="f16s")
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(1)
    assert sim.link_count(1) > 1_048_576
    out = np.zeros(3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_wall_force_noalloc(sim.ctx, 1, 0, 1.0, out, 1, sim.stream)
    assert e.value.status == 1 and "1048576" in str(e.value)
    # the regular entry point still serves it
    lbm.lbm_wall_force(sim.ctx, 1, 0, 1.0, out, 1, sim.stream)
    assert np.all(np.isfinite(out))
