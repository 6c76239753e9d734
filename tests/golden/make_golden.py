"""Write the stored expected values under tests/golden/ from the oracle alone.

The paper (arXiv 2512.12213) prints no worked numbers, so every stored value
here is either a closed form (cited in the file) or an output of the FP64 CPU
oracle, written by this script and nothing else.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_2512_12213_gb300 import inputs  # noqa: E402


def poiseuille_c1():
    """D2Q9 Poiseuille channel, 64 x 32 nodes, periodic x, halfway walls at
    y = -1/2 and 31.5, tau = 0.8, g = 1e-6, exact-difference forcing, rho0 = 1,
    started at rest, 10000 steps."""
    nx, ny, tau, g = 64, 32, 0.8, 1e-6
    cfg = orc.make_cfg(q=9, nx=nx, ny=ny, nz=1, periodic=(1, 0, 1), tau=tau, force_model="d",
                       g=(g, 0, 0), wall_u=((0, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    mask = inputs.empty_mask(nx, ny)
    f = orc.init(cfg, mask, np.ones((1, ny, nx)), np.zeros((3, 1, ny, nx)))
    f = orc.run(cfg, mask, f, 10000)
    fn, fr = orc.step(cfg, mask, f)
    sig, _, rho, v = orc.stress(cfg, mask, f, fr, fn, 2)
    nu = (tau - 0.5) / 3
    H = ny
    return {
        "case": "D2Q9 Poiseuille 64x32, tau 0.8, g 1e-6, model [d], 10000 steps from rest",
        "closed_form": {
            "citation": "recovered momentum equation, Eq. (7) (Sec. 3), for a body-force "
                        "driven channel with walls half a node outside the first fluid rows; "
                        "wall force balance, Eq. (33)",
            "nu": nu,
            "u_max_continuum": g * H * H / (8 * nu),
            "wall_shear_per_wall_per_unit_length": g * H / 2,
            "total_wall_force_x": g * H * nx,
        },
        "oracle_after_10000_steps": {
            "v_x_profile": v[0, 0, :, 0].tolist(),
            "sigma_xy_profile": sig[2, 0, :, 0].tolist(),
            "wall_force_bottom": orc.wall_force(cfg, mask, fr, fn, 1).tolist(),
            "wall_force_top": orc.wall_force(cfg, mask, fr, fn, 2).tolist(),
        },
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "poiseuille_c1.json")
    with open(out, "w") as fh:
        json.dump(poiseuille_c1(), fh, indent=1)
    print("wrote", out)
