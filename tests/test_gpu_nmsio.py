"""End to end through the file front end: a data tree of the paper's uniform
sphere in micromagnetic units -> GPU -> SANS1D.csv in cm^-1, checked against
the paper's Table I; loop mode writes one SANS_i folder per state."""
import csv
import os

import numpy as np
import pytest

from conftest import read_golden
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nmsio

pytestmark = pytest.mark.gpu

R_SPH = 20.0


def write(path, rows):
    path.parent.mkdir(parents=True, exist_ok=True)
    np.savetxt(path, rows, fmt="%.9g")


def read_csv(path):
    with open(path) as f:
        rows = list(csv.reader(f))
    hdr = rows[0]
    data = np.array([[float(x) for x in r] for r in rows[1:]])
    return {h: data[:, i] for i, h in enumerate(hdr)}, data.shape[0]


def sphere_tree(root, states):
    pos = I.lattice_ball(R_SPH, 1.0)
    n = len(pos)
    for i, m in enumerate(states):
        write(root / "MagData" / "Object_1" / f"m_{i + 1}.csv", np.hstack([pos, np.tile(m, (n, 1))]))
    write(root / "NucData" / "Object_1" / "n_1.csv", np.hstack([pos, np.ones((n, 1))]))
    return n


def config(path, data, out, loop=0):
    vs = 4.0 / 3.0 * np.pi * (R_SPH * 1e-9) ** 3
    path.write_text(f"""NucData_activate = 1; MagData_activate = 1; StructData_activate = 0;
DataPath = "{data}"; OutputPath = "{out}"; Mode = "micromagnetic";
Ms = 1.7e6; Ns = 8.0e14; Scale = 1; CellSize = {{1, 1, 1}}; Volume = {vs!r};
q_max = 1.2; r_max = 45; N_q = 97; N_theta = 16; N_r = 33; N_alpha = 8; k_max = 4;
alpha = 0; beta = 0; Polarization = {{0, 0, 1}}; Loop = {loop};
""")
    return vs


def test_table1_through_files(tmp_path):
    n = sphere_tree(tmp_path / "data", [(0.0, 0.0, 1.0)])
    vs = config(tmp_path / "run.conf", tmp_path / "data", tmp_path / "out")
    out = nmsio.run(str(tmp_path / "run.conf"))
    s1, rows = read_csv(os.path.join(out, "SANS1D.csv"))
    assert rows == 97 and s1["q"][0] == 0.0
    # at q = 0 the lattice sum is exactly the continuum integral over the
    # lattice's own volume n a^3: I(0) scales by (n a^3 / V_s)^2
    r2 = (n * 1e-27 / vs) ** 2
    checked = 0
    for kind, qty, val, tol in read_golden("table1_uniform_sphere.txt"):
        if kind != "I0" or qty not in s1:
            continue
        assert abs(s1[qty][0] - val * r2) <= tol * r2 + 1e-9 * abs(val), (qty, s1[qty][0], val * r2)
        checked += 1
    assert checked >= 10
    _, rows2 = read_csv(os.path.join(out, "SANS2D.csv"))
    assert rows2 == 97 * 16
    c1, rowsc = read_csv(os.path.join(out, "Corr1D.csv"))
    assert rowsc == 33 and "p_N" in c1 and c1["p_N"][0] == 0.0
    _, rowsc2 = read_csv(os.path.join(out, "Corr2D.csv"))
    assert rowsc2 == 33 * 8
    amp, _ = read_csv(os.path.join(out, "AngularSpectrum", "SF_amplitudes.csv"))
    # the spin-flip pattern of a saturated sphere is sin^2 cos^2: A0/A4 = -1
    # (up to the cubic lattice's small anisotropy in the detector plane)
    np.testing.assert_allclose(amp["A_c"][0] / amp["A_c"][4], -1.0, rtol=1e-4)


def test_loop_mode_writes_each_state(tmp_path):
    sphere_tree(tmp_path / "data", [(0.0, 0.0, 1.0), (0.0, 1.0, 0.0)])
    config(tmp_path / "run.conf", tmp_path / "data", tmp_path / "out", loop=1)
    out = nmsio.run(str(tmp_path / "run.conf"))
    a, _ = read_csv(os.path.join(out, "SANS_1", "SANS1D.csv"))
    b, _ = read_csv(os.path.join(out, "SANS_2", "SANS1D.csv"))
    # M along z -> |P.Q|^2 = M^2 sin^4 (mean 3/8); along y -> M^2 sin^2 cos^2 (mean 1/8)
    np.testing.assert_allclose(b["P"][0], a["P"][0] / 3.0, rtol=1e-6)
    np.testing.assert_allclose(b["M"][0], a["M"][0], rtol=1e-6)
    np.testing.assert_allclose(b["N"], a["N"], rtol=1e-12)
