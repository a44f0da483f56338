"""File front end in the layout of the paper's program: a configuration file,
the real-space data tree, and the CSV outputs (paper, Sec. "Configuration
file", Sec. "Real-space input data", Sec. "Fourier and real-space output
data").  Host-side only: it reads and writes files, converts units, and calls
the C ABI for every computed quantity.

Configuration file: ``key = value;`` lines, ``//`` comments; values are
numbers, quoted strings, or ``{a, b, c}`` vectors.  The activation keys are
the paper's (``NucData_activate``, ``MagData_activate``,
``StructData_activate``); the paper lists the other parameters without their
spelling, so these names are this library's:

  DataPath        directory holding NucData/, MagData/, StructData.csv
  OutputPath      output directory (created)
  Mode            "micromagnetic" (cells a_x a_y a_z, M = Ms m, N = Ns nu) or
                  "atomistic" (points; moments in Bohr magnetons, nuclear
                  scattering lengths in 1e-15 m)
  Ms              saturation magnetization [A/m] (micromagnetic)
  Ns              nuclear scattering-length density factor [m^-2]
                  (micromagnetic)
  Scale           lattice length scale s: input length x s = nm
  CellSize        {a_x, a_y, a_z} [nm] (micromagnetic)
  Volume          scattering volume V [m^3]
  q_max, r_max    [nm^-1], [nm]; q_min = 0
  N_q, N_theta    polar detector grid
  N_r, N_alpha    correlation distances and angles
  k_max           highest order of the angular spectrum
  alpha, beta     sample rotation R = R_z(beta) R_y(alpha) [deg]
  Polarization    {P_x, P_y, P_z}
  Loop            1: every m_i.csv (n_i.csv) index is one weight set
  Export_G        1: add the cross spectra G_ab (Re, Im) to SANS2D.csv

Data tree (1-based, continuous numbering): ``MagData/Object_k/m_i.csv``
(x y z mx my mz), ``NucData/Object_k/n_i.csv`` (x y z nu; one file n_1 serves
every loop index), ``StructData.csv`` (r_x r_y r_z per object); space- or
comma-separated columns, extensions .csv/.txt/.obj.

Units (library internals: lengths in nm).  Micromagnetic: M_j V_j =
Ms m V_cell with Ms in A/nm, N_j V_j = Ns nu V_cell with Ns in nm^-2.
Atomistic: moment mu_B mu in A nm^2, scattering length nu 1e-15 m in nm.
b_H = 2.91e8 A^-1 m^-1 in A^-1 nm^-1, V in nm^3; the library's cross
sections then come in nm^-1 and are exported x 1e7 in cm^-1 (the correlation
functions in nm^-4 and p(r) in nm^-2 as the paper states).
"""
from __future__ import annotations

import glob
import os
import re
import sys

import numpy as np

from . import inputs as I
from . import nms

MU_B = 9.274e-24              # J/T = A m^2
B_H = 2.91e8                  # A^-1 m^-1
NM_PER_M = 1e9
CM_PER_NM_INV = 1e7           # nm^-1 -> cm^-1

DEFAULTS = {
    "NucData_activate": 0, "MagData_activate": 1, "StructData_activate": 0,
    "DataPath": ".", "OutputPath": "NuMagSANS_out", "Mode": "micromagnetic",
    "Ms": 1.0, "Ns": 1.0, "Scale": 1.0, "CellSize": [1.0, 1.0, 1.0], "Volume": 0.0,
    "q_max": 1.0, "r_max": 50.0, "N_q": 128, "N_theta": 64, "N_r": 64, "N_alpha": 32, "k_max": 8,
    "alpha": 0.0, "beta": 0.0, "Polarization": [0.0, 0.0, 1.0], "Loop": 0, "Export_G": 0,
}


# ----------------------------------------------------------------- config
def _value(text):
    t = text.strip()
    if t.startswith("{") and t.endswith("}"):
        return [float(x) for x in t[1:-1].split(",") if x.strip()]
    if len(t) >= 2 and t[0] == t[-1] and t[0] in "\"'":
        return t[1:-1]
    try:
        return int(t)
    except ValueError:
        pass
    try:
        return float(t)
    except ValueError:
        return t


def read_config(path):
    """Parse a configuration file into a dict over DEFAULTS."""
    cfg = dict(DEFAULTS)
    with open(path) as f:
        text = f.read()
    text = re.sub(r"//[^\n]*", "", text)
    for stmt in text.split(";"):
        if "=" not in stmt:
            continue
        key, val = stmt.split("=", 1)
        key = key.strip()
        if key:
            cfg[key] = _value(val)
    return cfg


# ----------------------------------------------------------------- data tree
def _load_columns(path, ncol):
    with open(path) as f:
        rows = [r for r in (line.replace(",", " ").split() for line in f) if r]
    data = []
    for r in rows:
        try:
            data.append([float(x) for x in r[:ncol]])
        except ValueError:
            continue                      # header line
    a = np.asarray(data, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != ncol:
        raise ValueError(f"{path}: expected {ncol} numeric columns")
    return a


def _numbered(folder, prefix):
    """Files prefix_1, prefix_2, ... (any of .csv/.txt/.obj), continuous from 1."""
    found = {}
    for p in glob.glob(os.path.join(folder, prefix + "_*")):
        m = re.match(re.escape(prefix) + r"_(\d+)\.(csv|txt|obj)$", os.path.basename(p))
        if m:
            found[int(m.group(1))] = p
    n = len(found)
    if sorted(found) != list(range(1, n + 1)):
        raise ValueError(f"{folder}: {prefix}_i files must be numbered 1..{n} without gaps")
    return [found[i] for i in range(1, n + 1)]


def _objects(root):
    found = {}
    for p in glob.glob(os.path.join(root, "Object_*")):
        m = re.match(r"Object_(\d+)$", os.path.basename(p))
        if m and os.path.isdir(p):
            found[int(m.group(1))] = p
    n = len(found)
    if n == 0 or sorted(found) != list(range(1, n + 1)):
        raise ValueError(f"{root}: Object_k directories must be numbered 1..K without gaps")
    return [found[i] for i in range(1, n + 1)]


def read_data(cfg):
    """Real-space data of the configuration in library units (nm).

    Returns (field, n_sets): field.nuc [S][n] and field.mag [S][n][3] when the
    loop mode gives S > 1 weight sets, else plain [n] / [n][3]; offsets and
    centres describe the objects."""
    root = cfg["DataPath"]
    s = float(cfg["Scale"])
    atomistic = str(cfg["Mode"]).lower().startswith("atom")
    use_nuc, use_mag = int(cfg["NucData_activate"]), int(cfg["MagData_activate"])
    if not (use_nuc or use_mag):
        raise ValueError("activate NucData and/or MagData")
    loop = int(cfg["Loop"])
    mag_files, nuc_files = [], []
    if use_mag:
        mag_files = [_numbered(o, "m") for o in _objects(os.path.join(root, "MagData"))]
    if use_nuc:
        nuc_files = [_numbered(o, "n") for o in _objects(os.path.join(root, "NucData"))]
    K = len(mag_files) if use_mag else len(nuc_files)
    if use_mag and use_nuc and len(nuc_files) != K:
        raise ValueError("NucData and MagData must hold the same objects")
    n_idx = 1
    if loop:
        n_idx = max(len(f) for f in (mag_files or nuc_files))
    # per object: positions from the first file, then every set
    pos, nuc_sets, mag_sets, off = [], [[] for _ in range(n_idx)], [[] for _ in range(n_idx)], [0]
    for k in range(K):
        ref = None
        for i in range(n_idx):
            if use_mag:
                files = mag_files[k]
                a = _load_columns(files[min(i, len(files) - 1)], 6)
                if ref is None:
                    ref = a[:, :3]
                elif not np.allclose(a[:, :3], ref):
                    raise ValueError(f"object {k + 1}: positions differ between loop files")
                mag_sets[i].append(a[:, 3:6])
            if use_nuc:
                files = nuc_files[k]
                a = _load_columns(files[min(i, len(files) - 1)], 4)
                if ref is None:
                    ref = a[:, :3]
                elif not np.allclose(a[:, :3], ref):
                    raise ValueError(f"object {k + 1}: nuclear and magnetic positions differ")
                nuc_sets[i].append(a[:, 3])
        pos.append(ref * s)
        off.append(off[-1] + len(ref))
    pos = np.concatenate(pos)
    n = len(pos)
    if atomistic:
        vol = np.ones(n)
        mag_f = MU_B * NM_PER_M ** 2          # A m^2 -> A nm^2 per Bohr magneton
        nuc_f = 1e-15 * NM_PER_M               # 1e-15 m -> nm
    else:
        ax, ay, az = (float(v) for v in cfg["CellSize"])
        vol = np.full(n, ax * ay * az)
        mag_f = float(cfg["Ms"]) / NM_PER_M     # A/m -> A/nm
        nuc_f = float(cfg["Ns"]) / NM_PER_M ** 2   # m^-2 -> nm^-2
    nuc = np.stack([np.concatenate(v) * nuc_f for v in nuc_sets]) if use_nuc else None
    mag = np.stack([np.concatenate(v) * mag_f for v in mag_sets]) if use_mag else None
    if n_idx == 1:
        nuc = None if nuc is None else nuc[0]
        mag = None if mag is None else mag[0]
    centers = None
    if int(cfg["StructData_activate"]):
        centers = _load_columns(os.path.join(root, "StructData.csv"), 3) * s
        if len(centers) != K:
            raise ValueError("StructData.csv needs one row per object")
    offsets = np.asarray(off, dtype=np.int64) if K > 1 else None
    return I.Field(pos, vol, nuc, mag, offsets=offsets, centers=centers, name="data_tree"), n_idx


def rotation(alpha_deg, beta_deg):
    """R = R_z(beta) R_y(alpha) (Sec. "Configuration file")."""
    a, b = np.deg2rad(alpha_deg), np.deg2rad(beta_deg)
    Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    Rz = np.array([[np.cos(b), -np.sin(b), 0], [np.sin(b), np.cos(b), 0], [0, 0, 1]])
    return Rz @ Ry


# ----------------------------------------------------------------- outputs
def _responses(has_nuc, has_mag):
    names = []
    if has_nuc:
        names.append("N")
    if has_mag:
        names += ["M", "P", "CHI", "SF", "PM", "MP"]
    if has_nuc and has_mag:
        names += ["NM"]
    names += ["PP", "MM", "SANSPOL_P", "SANSPOL_M", "UNPOL"]
    return names


def _write_csv(path, header, cols):
    a = np.column_stack([np.asarray(c, dtype=np.float64).ravel() for c in cols])
    np.savetxt(path, a, delimiter=",", header=",".join(header), comments="", fmt="%.10e")


def write_outputs(plan, cfg, outdir, has_nuc, has_mag, part=nms.PART_TOTAL):
    """SANS1D/SANS2D/Corr1D/Corr2D CSVs and AngularSpectrum/ of the plan's
    selected weight set; cross sections in cm^-1, q in nm^-1, theta in rad,
    r in nm, c(r) in nm^-4, p(r) in nm^-2.  part: TOTAL (objects at their
    StructData positions) or DILUTE (no StructData: the sum over objects of
    each object's own cross section, Sec. "Summation approach")."""
    os.makedirs(os.path.join(outdir, "AngularSpectrum"), exist_ok=True)
    nq, nth = int(cfg["N_q"]), int(cfg["N_theta"])
    q = np.linspace(0.0, float(cfg["q_max"]), nq)
    th = 2 * np.pi * np.arange(nth) / nth
    Q, TH = np.meshgrid(q, th, indexing="ij")
    r = np.linspace(0.0, float(cfg["r_max"]), int(cfg["N_r"]))
    alpha = 2 * np.pi * np.arange(int(cfg["N_alpha"])) / int(cfg["N_alpha"])
    kmax = int(cfg["k_max"])
    names = _responses(has_nuc, has_mag)
    img = {k: nms.nms_response(plan, k, part) * CM_PER_NM_INV for k in names}
    cols2 = [Q, TH] + [img[k] for k in names]
    hdr2 = ["q", "theta"] + names
    if int(cfg["Export_G"]) and has_mag:
        for k in ("G_XX", "G_XY", "G_XZ", "G_YY", "G_YZ", "G_ZZ"):
            for part in ("RE", "IM"):
                name = f"{k}_{part}"
                if name in nms.RESPONSE_NAMES:
                    cols2.append(nms.nms_response(plan, name, part) * CM_PER_NM_INV)
                    hdr2.append(name)
    _write_csv(os.path.join(outdir, "SANS2D.csv"), hdr2, cols2)
    I1 = {}
    for k in names:
        Iq, _, _ = nms.nms_azimuthal_average(plan, img[k], nbins=nq)
        I1[k] = Iq
    _write_csv(os.path.join(outdir, "SANS1D.csv"), ["q"] + names, [q] + [I1[k] for k in names])
    cols, hdr = [r], ["r"]
    for k in names:
        # Eq. crrad on I in nm^-1 (c in nm^-4), Eq. prrad (nm^-2)
        c, p = nms.nms_correlation(q, I1[k] / CM_PER_NM_INV, r)
        cols += [c, p]
        hdr += [f"c_{k}", f"p_{k}"]
    _write_csv(os.path.join(outdir, "Corr1D.csv"), hdr, cols)
    R, A = np.meshgrid(r, alpha, indexing="ij")
    cols, hdr = [R, A], ["r", "alpha"]
    for k in names:
        C, _ = nms.nms_correlation_2d(plan, img[k] / CM_PER_NM_INV, r, alpha)
        cols += [C.real, C.imag]
        hdr += [f"C_{k}_re", f"C_{k}_im"]
    _write_csv(os.path.join(outdir, "Corr2D.csv"), hdr, cols)
    for k in names:
        out = nms.nms_angular_spectrum(plan, img[k], kmax, nbins=nq)
        _write_csv(os.path.join(outdir, "AngularSpectrum", f"{k}_modes.csv"),
                   ["q"] + [f"Ic_{j}" for j in range(kmax + 1)] + [f"Is_{j}" for j in range(kmax + 1)],
                   [q] + list(out["Ic"]) + list(out["Is"]))
        _write_csv(os.path.join(outdir, "AngularSpectrum", f"{k}_amplitudes.csv"), ["k", "A_c", "A_s"],
                   [np.arange(kmax + 1), out["Ac"], out["As"]])


def run(config_path, stream=None):
    """Read the configuration and data tree, compute on the GPU, write the
    outputs (one SANS_i folder per loop index in loop mode).  Returns the
    output directory."""
    cfg = read_config(config_path)
    base = os.path.dirname(os.path.abspath(config_path))
    for key in ("DataPath", "OutputPath"):
        if not os.path.isabs(str(cfg[key])):
            cfg[key] = os.path.join(base, str(cfg[key]))
    field, n_sets = read_data(cfg)
    grid = nms.make_grid("polar", int(cfg["N_q"]), int(cfg["N_theta"]), 0.0, float(cfg["q_max"]))
    V = float(cfg["Volume"]) * NM_PER_M ** 3
    opt = nms.nms_options_default(volume_V=V if V > 0 else 1.0, b_H=B_H / NM_PER_M, n_sets=n_sets,
                                  want_dilute=1 if field.offsets is not None else 0, P=cfg["Polarization"])
    R = rotation(float(cfg["alpha"]), float(cfg["beta"]))
    plan = nms.plan_from_field(field, grid, opt, rot=R.reshape(1, 9), stream=stream)
    nms.nms_amplitudes(plan)
    out = cfg["OutputPath"]
    os.makedirs(out, exist_ok=True)
    has_nuc, has_mag = field.nuc is not None, field.mag is not None
    # several objects without StructData: the dilute (noninteracting) sum
    part = nms.PART_DILUTE if field.offsets is not None and field.centers is None else nms.PART_TOTAL
    if n_sets == 1:
        write_outputs(plan, cfg, out, has_nuc, has_mag, part)
    else:
        for i in range(n_sets):
            nms.nms_select_set(plan, i)
            write_outputs(plan, cfg, os.path.join(out, f"SANS_{i + 1}"), has_nuc, has_mag, part)
    plan.close()
    return out


if __name__ == "__main__":
    if len(sys.argv) != 2:
        raise SystemExit("usage: python -m paper_2601_18444_gb300.nmsio CONFIG")
    print(run(sys.argv[1]))
