"""Host logic of the file front end: configuration parsing, the real-space
data tree (objects, loop indices, structure file), unit conversion and the
sample rotation.  No GPU."""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import nmsio


def write(path, rows, header=None):
    path.parent.mkdir(parents=True, exist_ok=True)
    with open(path, "w") as f:
        if header:
            f.write(header + "\n")
        for r in rows:
            f.write(" ".join(f"{v:.9g}" for v in r) + "\n")


def test_read_config_values_and_comments(tmp_path):
    p = tmp_path / "NuMagSANSInput.conf"
    p.write_text("""// comment line
NucData_activate    = 1;   // activate nuclear data
MagData_activate    = 0;
DataPath = "my data";  Mode = "atomistic";
q_max = 2.5; N_q = 200;
Polarization = {0, 1, 0};  // perpendicular
Unknown_Key = hello;
""")
    cfg = nmsio.read_config(p)
    assert cfg["NucData_activate"] == 1 and cfg["MagData_activate"] == 0
    assert cfg["DataPath"] == "my data" and cfg["Mode"] == "atomistic"
    assert cfg["q_max"] == 2.5 and cfg["N_q"] == 200 and isinstance(cfg["N_q"], int)
    assert cfg["Polarization"] == [0.0, 1.0, 0.0]
    assert cfg["Unknown_Key"] == "hello"
    assert cfg["N_theta"] == nmsio.DEFAULTS["N_theta"]


def make_tree(root, n_fields=2):
    rng = np.random.default_rng(0)
    objs = []
    for k in range(3):
        n = 5 + k
        pos = rng.uniform(-3, 3, size=(n, 3))
        nu = rng.uniform(0.5, 1.5, n)
        ms = [rng.normal(size=(n, 3)) for _ in range(n_fields)]
        for i, m in enumerate(ms):
            write(root / "MagData" / f"Object_{k + 1}" / f"m_{i + 1}.csv", np.hstack([pos, m]), header="x y z mx my mz")
        write(root / "NucData" / f"Object_{k + 1}" / "n_1.txt", np.hstack([pos, nu[:, None]]))
        objs.append((pos, nu, ms))
    centres = rng.uniform(-20, 20, size=(3, 3))
    write(root / "StructData.csv", centres)
    return objs, centres


def test_data_tree_micromagnetic_units_and_loop(tmp_path):
    objs, centres = make_tree(tmp_path / "data")
    cfg = dict(nmsio.DEFAULTS, DataPath=str(tmp_path / "data"), NucData_activate=1, MagData_activate=1,
               StructData_activate=1, Loop=1, Ms=1.7e6, Ns=8e14, Scale=0.5, CellSize=[1.0, 2.0, 0.5])
    f, S_ = nmsio.read_data(cfg)
    assert S_ == 2
    assert list(f.offsets) == [0, 5, 11, 18]
    np.testing.assert_allclose(f.pos, 0.5 * np.concatenate([o[0] for o in objs]))
    np.testing.assert_allclose(f.centers, 0.5 * centres)
    np.testing.assert_allclose(f.vol, 1.0)                    # 1 x 2 x 0.5 nm^3
    assert f.mag.shape == (2, 18, 3) and f.nuc.shape == (2, 18)
    for i in range(2):
        np.testing.assert_allclose(f.mag[i], 1.7e6 * 1e-9 * np.concatenate([o[2][i] for o in objs]))
        np.testing.assert_allclose(f.nuc[i], 8e14 * 1e-18 * np.concatenate([o[1] for o in objs]))
    # without the loop mode only the first index is read
    f1, S1 = nmsio.read_data(dict(cfg, Loop=0))
    assert S1 == 1 and f1.mag.shape == (18, 3)
    np.testing.assert_allclose(f1.mag, f.mag[0])


def test_data_tree_atomistic_units(tmp_path):
    objs, _ = make_tree(tmp_path / "data", n_fields=1)
    cfg = dict(nmsio.DEFAULTS, DataPath=str(tmp_path / "data"), NucData_activate=1, MagData_activate=1,
               Mode="atomistic")
    f, _ = nmsio.read_data(cfg)
    np.testing.assert_allclose(f.vol, 1.0)
    # Bohr magneton in A nm^2 and 1e-15 m in nm
    np.testing.assert_allclose(f.mag, 9.274e-24 * 1e18 * np.concatenate([o[2][0] for o in objs]))
    np.testing.assert_allclose(f.nuc, 1e-6 * np.concatenate([o[1] for o in objs]))
    assert f.centers is None


def test_data_tree_errors(tmp_path):
    make_tree(tmp_path / "data")
    (tmp_path / "data" / "MagData" / "Object_2" / "m_2.csv").rename(tmp_path / "data" / "MagData" / "Object_2" / "m_3.csv")
    cfg = dict(nmsio.DEFAULTS, DataPath=str(tmp_path / "data"))
    with pytest.raises(ValueError):
        nmsio.read_data(cfg)
    with pytest.raises(ValueError):
        nmsio.read_data(dict(cfg, MagData_activate=0, NucData_activate=0))


def test_rotation_convention():
    # alpha = 90 deg turns e_z into e_x (the parallel geometry of the paper)
    np.testing.assert_allclose(nmsio.rotation(90.0, 0.0) @ [0, 0, 1], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(nmsio.rotation(33.0, -71.0), S.sample_rotation(33.0, -71.0), atol=1e-15)
