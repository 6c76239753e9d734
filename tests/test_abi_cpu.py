"""The C ABI library on a machine without a GPU: it loads, exports every
symbol declared in include/lbm.h, and validates configurations (lbm_buffer_sizes
touches no CUDA state)."""
import os
import re

import numpy as np
import pytest

from paper_2512_12213_gb300 import inputs, lbm, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_12213_gb300 import build
    build.build()
    return lbm.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm.EXPORTED)


def test_buffer_sizes(lib):
    cfg, mask = workloads.sphere(nx=32, ny=16, nz=16, radius=4, center=(8, 8, 8), storage="f16s")
    c = lbm.make_config(**cfg)
    s = lbm.lbm_buffer_sizes(c, mask)
    nxp = 64
    assert s[lbm.BUF_POP_A] == s[lbm.BUF_POP_B] >= 19 * nxp * 16 * 16 * 2
    assert s[lbm.BUF_NODE] >= nxp * 16 * 16
    assert s[lbm.BUF_LINKS] > 0 and s[lbm.BUF_LINKS] % 256 == 0
    assert all(v % 256 == 0 for v in s)
    # the same geometry with FP64 storage needs four times the population bytes
    c64 = lbm.make_config(**dict(cfg, storage="f64"))
    s64 = lbm.lbm_buffer_sizes(c64, mask)
    assert s64[lbm.BUF_POP_A] >= 4 * 19 * nxp * 16 * 16 * 2


@pytest.mark.parametrize("field,value,msg", [
    ("lattice", 7, "lattice"), ("nx", 0, "nx"), ("tau", 0.5, "tau"), ("force_model", 5, "force_model"),
    ("storage", 4, "storage"), ("dx", 0.0, "dx"), ("nz", 2, "D2Q9"), ("insulating", 1, "Lorentz"),
    ("insulating", 2, "insulating"),
])
def test_invalid_configs_rejected(lib, field, value, msg):
    cfg, mask = workloads.poiseuille(nx=8, ny=6)
    c = lbm.make_config(**cfg)
    setattr(c, field, value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_buffer_sizes(c, mask if field != "nz" else np.zeros((2, 6, 8), np.uint8))
    assert e.value.status == 1 and msg in str(e.value)


def test_face_wall_and_mask_ids_checked(lib):
    cfg, mask = workloads.poiseuille(nx=8, ny=6)
    c = lbm.make_config(**dict(cfg, face_wall=(1, 1, 1, 3, 1, 1)))
    with pytest.raises(lbm.LbmError, match="face_wall"):
        lbm.lbm_buffer_sizes(c, mask)
    c = lbm.make_config(**cfg)
    bad = mask.copy()
    bad[0, 2, 3] = 5
    with pytest.raises(lbm.LbmError, match="exceeds n_walls"):
        lbm.lbm_buffer_sizes(c, bad)


def test_maximum_size_rejected(lib):
    # padded node count must stay below 2^31
    c = lbm.make_config(lattice=19, nx=1300, ny=1300, nz=1300, periodic=(1, 1, 1))
    with pytest.raises(lbm.LbmError, match="too large"):
        lbm.lbm_buffer_sizes(c, np.zeros(1, np.uint8))


def test_link_count_matches_oracle(lib, orc):
    """The library's link list has exactly the oracle's boundary links."""
    for q in (9, 19):
        if q == 9:
            mask = inputs.random_solids(23, 11, 1, 0.15, n_walls=3, seed=3)
            cfg = dict(lattice=9, nx=23, ny=11, nz=1, periodic=(1, 0, 1), wall_u=((0, 0, 0),) * 3,
                       face_wall=(1, 1, 2, 3, 1, 1))
        else:
            mask = inputs.random_solids(9, 8, 7, 0.1, n_walls=2, seed=4)
            cfg = dict(lattice=19, nx=9, ny=8, nz=7, periodic=(0, 1, 0), wall_u=((0, 0, 0),) * 2,
                       face_wall=(1, 2, 1, 1, 2, 1))
        c = lbm.make_config(**cfg)
        s = lbm.lbm_buffer_sizes(c, mask)
        n_links = orc.count_links(orc.make_cfg(**workloads.oracle_kwargs(cfg)), mask)
        assert s[lbm.BUF_LINKS] == (n_links * 8 + 255) // 256 * 256


def test_2d_maxwell_needs_in_plane_field(lib):
    cfg, mask = workloads.hartmann(nx=8, ny=6, maxwell=1)
    c = lbm.make_config(**dict(cfg, B=(0.0, 0.05, 0.01)))
    with pytest.raises(lbm.LbmError, match="in-plane"):
        lbm.lbm_buffer_sizes(c, mask)


def test_stochastic_rounding_only_for_16_bit(lib):
    cfg, mask = workloads.poiseuille(nx=8, ny=6, storage="f32")
    with pytest.raises(lbm.LbmError, match="16-bit"):
        lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, rounding="stochastic")), mask)
    lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, storage="f16s", rounding="stochastic")), mask)


def test_insulating_walls_scratch(lib):
    """Insulating walls add a field block and one row of 3 doubles per warp
    of the step grid (blocks of 128 threads; a thread takes 2 nodes in FP64,
    else 4) to the scratch buffer."""
    cfg, mask = workloads.hartmann_insulating(nx=100, ny=400)
    plain = lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, insulating=0)), mask)
    ins = lbm.lbm_buffer_sizes(lbm.make_config(**cfg), mask)
    warps = -(-(128 // 2) * 400 // 128) * 4
    assert ins[lbm.BUF_SCRATCH] >= plain[lbm.BUF_SCRATCH] + 3 * 8 * warps
    assert ins[lbm.BUF_SCRATCH] < plain[lbm.BUF_SCRATCH] + 3 * 8 * (warps + 1024 + 16) + 512
    assert ins[lbm.BUF_POP_A] == plain[lbm.BUF_POP_A]
    ins32 = lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, storage="f32")), mask)
    warps32 = -(-(128 // 4) * 400 // 128) * 4
    assert ins[lbm.BUF_SCRATCH] - ins32[lbm.BUF_SCRATCH] >= 3 * 8 * (warps - warps32) - 256


def test_curved_walls_buffer(lib):
    """Curved walls need a float per padded node for the wall distance."""
    cfg, mask = workloads.poiseuille(nx=100, ny=12)
    plain = lbm.lbm_buffer_sizes(lbm.make_config(**cfg), mask)
    cur = lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, curved=1)), mask)
    assert plain[lbm.BUF_PHI] == 0
    assert cur[lbm.BUF_PHI] >= 128 * 12 * 4 and cur[lbm.BUF_PHI] % 256 == 0
    c = lbm.make_config(**dict(cfg, curved=2))
    with pytest.raises(lbm.LbmError, match="curved"):
        lbm.lbm_buffer_sizes(c, mask)


def test_induced_field_buffers(lib):
    """The induced field needs two buffers of 3 x (5 or 7) distributions per
    padded node in compute precision (FP64, else FP32), and is refused
    without the Maxwell equilibrium, with the low-Rm Lorentz force, LES,
    curved or insulating walls, and for eta <= 0."""
    cfg, mask = workloads.hartmann_induced(nx=100, ny=12)
    plain = lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, induced=0)), mask)
    ind = lbm.lbm_buffer_sizes(lbm.make_config(**cfg), mask)
    assert plain[lbm.BUF_MAG_A] == plain[lbm.BUF_MAG_B] == 0
    assert ind[lbm.BUF_MAG_A] == ind[lbm.BUF_MAG_B] >= 3 * 5 * 128 * 12 * 8
    assert ind[lbm.BUF_MAG_A] % 256 == 0
    f32 = lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, storage="f16s")), mask)
    assert f32[lbm.BUF_MAG_A] == (3 * 5 * 128 * 12 * 4 + 255) // 256 * 256
    c3 = dict(lattice=19, nx=10, ny=6, nz=5, periodic=(1, 1, 1), maxwell=1, induced=1, eta=0.1, wall_u=((0, 0, 0),))
    m3 = np.zeros((5, 6, 10), np.uint8)
    s3 = lbm.lbm_buffer_sizes(lbm.make_config(**c3), m3)
    assert s3[lbm.BUF_MAG_A] == (3 * 7 * 64 * 6 * 5 * 8 + 255) // 256 * 256
    for bad, msg in ((dict(maxwell=0), "maxwell"), (dict(lorentz=1, sigma_e=0.1), "lorentz"),
                     (dict(les=1), "les"), (dict(curved=1), "curved"), (dict(eta=0.0), "eta"),
                     (dict(eta=float("nan")), "eta"), (dict(induced=2), "induced"),
                     (dict(mag_conducting=3), "mag_conducting")):
        with pytest.raises(lbm.LbmError, match=msg):
            lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, **bad)), mask)


def test_bench_workloads_are_valid_configurations(lib):
    """Every workload bench.py times (the headline sphere, the LES cavity and
    the four extension rows) passes the library's configuration checks, and
    the algorithmic bytes per node it reports match the buffers: two
    population buffers per step, plus the two field buffers of the induced
    field."""
    import bench
    for name in ["sphere", "cavity"] + list(bench.EXTENSIONS):
        cfg, mask, phi = bench.make_workload(workloads, name, "f32")
        sizes = lbm.lbm_buffer_sizes(lbm.make_config(**cfg), mask)
        if phi is not None:
            assert phi.shape == mask.shape and np.array_equal(phi < 0, mask > 0)
        nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
        pitch = -(-cfg["nx"] // 64) * 64
        padded = pitch * cfg["ny"] * cfg["nz"]
        bpn = bench.bytes_per_node(19, "f32", induced=bool(cfg.get("induced")))
        stream = 2 * 19 * 4 + 1 + (2 * 3 * 7 * 4 if cfg.get("induced") else 0)
        assert bpn == stream, name
        moved = sizes[lbm.BUF_POP_A] + sizes[lbm.BUF_POP_B] + sizes[lbm.BUF_MAG_A] + sizes[lbm.BUF_MAG_B]
        assert moved >= (bpn - 1) * padded
        assert nodes <= padded


def test_header_is_plain_c(tmp_path):
    """include/lbm.h is a C header: a C99 translation unit that takes the
    address of every declared entry point and fills a configuration compiles
    with gcc -std=c99 -Wall -Wextra -pedantic -Werror, and links against liblbm.so (no GPU is
    touched: nothing is called)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = open(os.path.join(root, "include", "lbm.h")).read()
    names = sorted(set(re.findall(r"^(?:lbm_status|const char\*)\s+(lbm_\w+)\(", hdr, re.M)))
    assert "lbm_step" in names and "lbm_export_field" in names
    src = ['#include <stdio.h>', '#include "lbm.h"', 'int main(void) {',
           '    lbm_config c = {0};', '    c.lattice = LBM_D3Q19; c.nx = c.ny = c.nz = 4; c.tau = 0.8;',
           '    c.induced = 0; c.eta = 0.0; c.storage = LBM_STORE_F16S;',
           '    size_t sizes[LBM_NUM_BUFFERS]; (void)sizes;',
           '    void (*fns[])(void) = {']
    src += ['        (void (*)(void))&%s,' % n for n in names]
    src += ['    };', '    printf("%d %d\\n", (int)(sizeof fns / sizeof fns[0]), c.lattice);', '    return 0;', '}']
    cfile = tmp_path / "abi.c"
    cfile.write_text("\n".join(src) + "\n")
    obj = tmp_path / "abi.o"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(root, "include"), "-c", str(cfile), "-o", str(obj)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    so = lbm.LIB_PATH
    if not os.path.exists(so):
        pytest.skip("liblbm.so not built")
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, str(obj), so, "-o", str(exe), "-Wl,-rpath," + os.path.dirname(so)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("change", [dict(storage="f64"), dict(curved=1),
                                    dict(lorentz=1, sigma_e=0.1, insulating=1, B=(0, 0.01, 0)),
                                    dict(induced=1, maxwell=1, eta=0.05, B=(0, 0.01, 0))])
def test_staged_kernel_refused_where_it_does_not_apply(lib, change):
    cfg, mask = workloads.sphere(nx=32, ny=16, nz=16, radius=4, center=(8, 8, 8), storage="f16s")
    c = lbm.make_config(**dict(cfg, step_kernel="staged", face_wall=(1, 1, 1, 1, 1, 1), **change))
    with pytest.raises(lbm.LbmError, match="staged"):
        lbm.lbm_buffer_sizes(c, mask)
    # the same configuration with the automatic choice is accepted
    lbm.lbm_buffer_sizes(lbm.make_config(**dict(cfg, face_wall=(1, 1, 1, 1, 1, 1), **change)), mask)
