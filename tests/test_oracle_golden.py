"""The stored Poiseuille case (written by tests/golden/make_golden.py from the
oracle) against its closed forms and against a fresh oracle run (no GPU)."""
import json
import os

import numpy as np

from paper_2512_12213_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poiseuille_c1.json")


def test_golden_poiseuille_closed_form_and_rerun(orc):
    data = json.load(open(GOLDEN))
    cf = data["closed_form"]
    # closed forms for H = 32, g = 1e-6, nu = (0.8 - 0.5)/3
    assert np.isclose(cf["u_max_continuum"], 1.28e-3, rtol=1e-12)
    assert np.isclose(cf["wall_shear_per_wall_per_unit_length"], 1.6e-5, rtol=1e-12)
    assert np.isclose(cf["total_wall_force_x"], 2.048e-3, rtol=1e-12)
    o = data["oracle_after_10000_steps"]
    v = np.array(o["v_x_profile"])
    H, g, nu, tau = 32, 1e-6, 0.1, 0.8
    y = np.arange(H)
    v_exact = g / (2 * nu) * ((y + 0.5) * (H - 0.5 - y) + (16 * (tau - 0.5) ** 2 - 3) / 12)
    # after 10000 steps the slowest mode exp(-nu pi^2 t / H^2) leaves ~6.5e-5
    assert np.abs(v - v_exact).max() / v_exact.max() < 1e-4
    # each wall carries about half of the 2.048e-3 total (transient included)
    assert np.isclose(o["wall_force_bottom"][0], o["wall_force_top"][0], rtol=1e-12)
    assert abs(o["wall_force_bottom"][0] / (0.5 * cf["total_wall_force_x"]) - 1) < 1e-3
    # a fresh oracle run reproduces the stored profile
    cfg = orc.make_cfg(q=9, nx=64, ny=32, nz=1, periodic=(1, 0, 1), tau=0.8, force_model="d",
                       g=(1e-6, 0, 0), wall_u=((0, 0, 0), (0, 0, 0)), face_wall=(1, 1, 1, 2, 1, 1))
    mask = inputs.empty_mask(64, 32)
    f = orc.init(cfg, mask, np.ones((1, 32, 64)), np.zeros((3, 1, 32, 64)))
    f = orc.run(cfg, mask, f, 10000)
    fn, fr = orc.step(cfg, mask, f)
    _, _, _, vv = orc.stress(cfg, mask, f, fr, fn, 2)
    assert np.allclose(vv[0, 0, :, 0], v, rtol=1e-12, atol=0)
