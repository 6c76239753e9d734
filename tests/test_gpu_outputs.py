"""Output placement of the reductions (device, host, asynchronous pinned host)
and the wall force computed on a second stream beside the step that reads
the same stored state: both give exactly the values of the plain sequential
calls."""
import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()
    assert torch.cuda.is_available()


def _sim(storage="f32", rounding="nearest"):
    nx, ny, nz = 72, 20, 18
    mask = inputs.sphere_mask(nx, ny, nz, (30.2, 9.7, 8.6), 5.3, wall=1)
    cfg = dict(lattice=19, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), tau=0.66, force_model="e",
               g=(3e-5, 0, 0), storage=storage, rounding=rounding, seed=7,
               wall_u=((0, 0, 0), (0.02, 0, 0)), face_wall=(1, 1, 1, 1, 1, 2))
    sim = lbm.Sim(cfg, mask)
    sim.rest()
    sim.step(5)
    return sim


def test_async_host_output_matches_blocking():
    sim = _sim()
    st = sim.stream
    for fn, width, extra in ((lbm.lbm_wall_force, 3, (1, lbm.MOVING_CORR, 0.5)),
                             (lbm.lbm_wall_force_noalloc, 3, (-1, 0, 1.0)),
                             (lbm.lbm_balance, 7, ())):
        ref = np.zeros(width)
        fn(sim.ctx, *extra, ref, lbm.OUT_HOST, st)
        pinned = torch.full((width,), -1.0, dtype=torch.float64, pin_memory=True)
        fn(sim.ctx, *extra, pinned, lbm.OUT_HOST_ASYNC, st)
        torch.cuda.synchronize()
        assert np.array_equal(pinned.numpy(), ref)
        dev = torch.zeros(width, dtype=torch.float64, device=sim.device)
        fn(sim.ctx, *extra, dev, lbm.OUT_DEVICE, st)
        assert np.array_equal(dev.cpu().numpy(), ref)


def test_async_host_output_refusals():
    sim = _sim()
    st = sim.stream
    pageable = np.zeros(3)
    with pytest.raises(lbm.LbmError, match="page-locked"):
        lbm.lbm_wall_force(sim.ctx, 1, 0, 1.0, pageable, lbm.OUT_HOST_ASYNC, st)
    with pytest.raises(lbm.LbmError, match="page-locked"):
        lbm.lbm_wall_force_noalloc(sim.ctx, 1, 0, 1.0, pageable, lbm.OUT_HOST_ASYNC, st)
    pinned = torch.zeros(3, dtype=torch.float64, pin_memory=True)
    with pytest.raises(lbm.LbmError, match="ACCUMULATE"):
        lbm.lbm_wall_force(sim.ctx, 1, lbm.ACCUMULATE, 1.0, pinned, lbm.OUT_HOST_ASYNC, st)
    with pytest.raises(lbm.LbmError, match="out_on_host"):
        lbm.lbm_wall_force(sim.ctx, 1, 0, 1.0, pageable, 3, st)
    with pytest.raises(lbm.LbmError, match="out_on_host"):
        lbm.lbm_balance(sim.ctx, np.zeros(7), -1, st)
    # a refused call leaves the context usable
    F = np.zeros(3)
    lbm.lbm_wall_force(sim.ctx, 1, 0, 1.0, F, lbm.OUT_HOST, st)
    assert np.all(np.isfinite(F)) and F[0] != 0.0


@pytest.mark.parametrize("storage,rounding", [("f32", "nearest"), ("f16s", "stochastic")])
def test_force_beside_step_on_second_stream(storage, rounding):
    """Force of step T-1 -> T on a side stream while the step T -> T+1 runs
    on the main stream (ordered as the benchmark orders them) equals the
    force of the sequential run, bit for bit, and so do the states."""
    steps = 12
    a = _sim(storage, rounding)
    ref = np.zeros((steps, 3))
    for i in range(steps):
        lbm.lbm_wall_force(a.ctx, 2, 0, 1.0, ref[i], lbm.OUT_HOST, a.stream)
        a.step(1)
    f_ref = a.export_f()

    b = _sim(storage, rounding)
    cs = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=cs.device)
    got = torch.zeros((steps, 3), dtype=torch.float64, device=b.device)
    for i in range(steps):
        side.wait_stream(cs)
        lbm.lbm_wall_force(b.ctx, 2, 0, 1.0, got[i], lbm.OUT_DEVICE, side.cuda_stream)
        lbm.lbm_step(b.ctx, 1, b.stream)
        cs.wait_stream(side)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)
    assert torch.equal(b.export_f(), f_ref)
