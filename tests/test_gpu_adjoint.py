"""The CUDA adjoint of time-averaged drag against the oracle's complex-step
adjoint (tiny grids, FP64) and against central finite differences of the
GPU FP64 forward at the full cylinder size (512 x 256, T = 2000), through
the sqrt(T) checkpoint driver and the autograd function."""
import numpy as np
import pytest
import torch

from paper_2512_12213_gb300 import adjoint, inputs, lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_12213_gb300 import build
    build.build()
    lbm.load()


def _tiny(q, model, storage="f64"):
    if q == 9:
        nx, ny, nz = 10, 8, 1
        mask = inputs.block_mask(nx, ny, nz, (3, 3, 0), (5, 5, 1), wall=1)
        per = (1, 0, 1)
    else:
        nx, ny, nz = 6, 6, 5
        mask = inputs.block_mask(nx, ny, nz, (2, 2, 1), (4, 4, 3), wall=1)
        per = (1, 1, 0)
    cfg = dict(lattice=q, nx=nx, ny=ny, nz=nz, periodic=per, tau=0.7, dx=0.5, dt=0.25, force_model=model,
               g=(2e-2, -7e-3, 3e-3), wall_u=((0.03, -0.02, 0.01), (0.0, 0.0, 0.0)),
               face_wall=(2, 2, 2, 2, 2, 2), storage=storage)
    return cfg, mask


@pytest.mark.parametrize("q,model", [(9, m) for m in "abcde"] + [(19, m) for m in "abcde"])
def test_adjoint_matches_oracle_fp64(orc, q, model):
    cfg, mask = _tiny(q, model)
    T, d = 12, (1.0, 0.3, -0.2)
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    nz, ny, nx = mask.shape
    f0 = orc.init(ocfg, mask, np.full((nz, ny, nx), 1.0), np.zeros((3, nz, ny, nx)))
    J_o, g_o = orc.adjoint_drag(ocfg, mask, f0, T, 1, d)
    sim = lbm.Sim(cfg, mask)
    prob = adjoint.DragProblem(sim, T, 1, d, stride=5)     # 3 segments, ragged last
    theta = list(cfg["g"]) + list(cfg["wall_u"][0])
    J = prob.forward(theta)
    g = prob.backward()
    assert abs(J - J_o) < 1e-13 * abs(J_o)
    idx = [0, 1, 3, 4] if q == 9 else list(range(6))
    assert np.abs(g[idx] - g_o[idx]).max() < 1e-10 * np.abs(g_o[idx]).max(), (g, g_o)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_adjoint_reduced_precision(orc, storage, tol):
    cfg, mask = _tiny(19, "e", storage)
    T, d = 12, (1.0, 0.0, 0.0)
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    nz, ny, nx = mask.shape
    f0 = orc.init(ocfg, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    J_o, g_o = orc.adjoint_drag(ocfg, mask, f0, T, 1, d)
    prob = adjoint.DragProblem(lbm.Sim(cfg, mask), T, 1, d)
    theta = list(cfg["g"]) + list(cfg["wall_u"][0])
    J = prob.forward(theta)
    g = prob.backward()
    assert abs(J - J_o) < tol * abs(J_o)
    assert np.abs(g - g_o).max() < tol * np.abs(g_o).max(), (g, g_o)


def test_autograd_function(orc):
    cfg, mask = _tiny(9, "d")
    prob = adjoint.DragProblem(lbm.Sim(cfg, mask), 9, 1, (1.0, 0.0, 0.0))
    theta = torch.tensor(list(cfg["g"]) + list(cfg["wall_u"][0]), dtype=torch.float64, requires_grad=True)
    J = adjoint.DragFn.apply(theta, prob)
    (3.0 * J).backward()
    g = prob.backward()
    assert torch.allclose(theta.grad, 3.0 * torch.as_tensor(g), rtol=1e-14, atol=0)


def test_cylinder_gradient_vs_central_differences():
    """D2Q9 512 x 256 cylinder, r = 20, T = 2000, FP32 forward and adjoint with
    FP64 reductions, against central differences of the FP64 forward."""
    T = 2000
    cfg32, mask = workloads.cylinder(storage="f32")
    cfg64 = dict(cfg32, storage="f64")
    theta = np.array(list(cfg32["g"]) + [0.0, 0.0, 0.0])
    p32 = adjoint.DragProblem(lbm.Sim(cfg32, mask), T, 1)
    J32 = p32.forward(theta)
    g32 = p32.backward()
    p64 = adjoint.DragProblem(lbm.Sim(cfg64, mask), T, 1)
    J64 = p64.forward(theta)
    assert abs(J32 / J64 - 1) < 1e-4
    fd = np.zeros(6)
    for k in (0, 1, 3, 4):
        h = 1e-3 * (abs(theta[k]) if theta[k] else 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (p64.forward(tp) - p64.forward(tm)) / (2 * h)
    for k in (0, 1, 3, 4):
        assert abs(g32[k] - fd[k]) <= 1e-4 * np.abs(fd).max(), (k, g32, fd)
