"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against an independent fact: values printed in
the paper's Tables I and II, closed forms (Dirichlet kernel, sphere form
factor, two scatterers), symmetries (translation, 90-degree rotations,
Hermitian symmetry), the paper's expanded POLARIS/SANSPOL expressions, and
brute force on tiny inputs.  None of these needs a GPU.
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from conftest import read_golden

# SI-ish units in nm: N0 [nm^-2], M0 [A nm^-1], b_H [A^-1 nm^-1]
R_SPH = 20.0
N0 = 8.0e14 * 1e-18
M0 = 1.7e6 * 1e-9
BH = 2.91e8 * 1e-9
VS = 4.0 / 3.0 * np.pi * R_SPH ** 3
TO_CM = 1e7               # nm^-1 -> cm^-1


def _polar(nq, nth, qmax, q0=0.0):
    q = np.linspace(q0, qmax, nq)
    th = 2 * np.pi * np.arange(nth) / nth
    Q, T = np.meshgrid(q, th, indexing="ij")
    return q, np.sin(T).ravel(), np.cos(T).ravel(), Q.ravel(), T.ravel()


def _avg(img, nq, nth):
    return S.azimuthal_average_polar(img, nq, nth)


# ---------------------------------------------------------------- Table I/II
@pytest.mark.parametrize("table", ["table1_uniform_sphere.txt", "table2_linear_vortex.txt"])
def test_tables_q0_and_max(table):
    nq, nth = 3001, 16
    q, hy, hz, qa, _ = _polar(nq, nth, 1.2)
    if table.startswith("table1"):
        F = S.uniform_sphere_amplitudes(qa, R_SPH, N0, M0, (0.0, 0.0, 1.0))
    else:
        F = S.linear_vortex_amplitudes(qa, hy, hz, R_SPH, N0, M0, 5.0 * M0 / R_SPH)
    res = S.responses(F, hy, hz, (0, 0, 1), BH, VS)
    checked = 0
    for kind, qty, val, tol in read_golden(table):
        if kind not in ("I0", "IMAX"):
            continue
        Iq = _avg(res[qty], nq, nth) * TO_CM
        got = Iq[0] if kind == "I0" else Iq.max()
        assert abs(got - val) <= tol + 1e-12 * abs(val), (kind, qty, got, val)
        checked += 1
    assert checked >= 9


@pytest.mark.parametrize("table", ["table1_uniform_sphere.txt", "table2_linear_vortex.txt"])
def test_tables_pmax(table):
    # Table p values = r^2 * integral I j0 q^2 dq (prefactor 1): reading of Eq. crrad
    nq, nth = 8001, 16
    q, hy, hz, qa, _ = _polar(nq, nth, 40.0)
    if table.startswith("table1"):
        F = S.uniform_sphere_amplitudes(qa, R_SPH, N0, M0, (0.0, 0.0, 1.0))
    else:
        F = S.linear_vortex_amplitudes(qa, hy, hz, R_SPH, N0, M0, 5.0 * M0 / R_SPH)
    res = S.responses(F, hy, hz, (0, 0, 1), BH, VS)
    r = np.linspace(0.0, 45.0, 901)
    for kind, qty, val, tol in read_golden(table):
        if kind != "PMAX":
            continue
        Iq = _avg(res[qty], nq, nth)
        _, p = S.correlation(q, Iq, r, prefactor=1.0)
        assert abs(p.max() - val) <= tol + 2e-9, (qty, p.max(), val)


def test_sphere_pddf_closed_form():
    # f(xi) = xi^2 (xi-2)^2 (xi+4)/4, xi_max = sqrt(105)/5 - 1, f(xi_max) = 1.2562;
    # p_N = 3 pi V N0^2/(8R) f(r/R) x 1/(2 pi^2) with the printed Eq. crrad prefactor
    nq = 16001
    q = np.linspace(0.0, 60.0, nq)
    Iq = 9.0 * N0 ** 2 * VS * S.sphere_g(q * R_SPH) ** 2
    xi = np.array([0.25, 0.5, 1.0, np.sqrt(105) / 5 - 1, 1.5, 1.9])
    _, p = S.correlation(q, Iq, xi * R_SPH)
    f = 0.25 * xi ** 2 * (xi - 2) ** 2 * (xi + 4)
    exact = 3 * np.pi * VS * N0 ** 2 / (8 * R_SPH) * f / (2 * np.pi ** 2)
    np.testing.assert_allclose(p, exact, rtol=2e-4, atol=1e-12)
    xm = np.sqrt(105) / 5 - 1
    assert abs(0.25 * xm ** 2 * (xm - 2) ** 2 * (xm + 4) - 1.2562) < 5e-5
    # beyond the largest distance 2R the PDDF vanishes (consistency check of the paper)
    _, pz = S.correlation(q, Iq, np.array([41.0, 50.0, 60.0]))
    assert np.all(np.abs(pz) < 1e-5 * exact.max())


# ------------------------------------------------------ 2D closed forms
def test_uniform_sphere_2d_forms_general_n():
    rng = np.random.default_rng(11)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    nq, nth = 7, 32
    q, hy, hz, qa, T = _polar(nq, nth, 0.5, q0=0.01)
    F = S.uniform_sphere_amplitudes(qa, R_SPH, N0, M0, n)
    res = S.responses(F, hy, hz, (0, 0, 1), BH, VS)
    g2 = S.sphere_g(qa * R_SPH) ** 2
    s, c = np.sin(T), np.cos(T)
    nx, ny, nz = n
    np.testing.assert_allclose(res["N"], 9 * N0 ** 2 * VS * g2, rtol=1e-12)
    np.testing.assert_allclose(res["M"], 9 * BH ** 2 * M0 ** 2 * VS * g2 *
                               (nx ** 2 + ny ** 2 * c ** 2 + nz ** 2 * s ** 2 - 2 * ny * nz * s * c),
                               rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(res["NM"], 18 * BH * M0 * N0 * VS * g2 * (ny * s * c - nz * s ** 2),
                               rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(res["P"], 9 * BH ** 2 * M0 ** 2 * VS * g2 *
                               (ny ** 2 * s ** 2 * c ** 2 + nz ** 2 * s ** 4 - 2 * ny * nz * s ** 3 * c),
                               rtol=1e-10, atol=1e-14)
    assert np.max(np.abs(res["CHI"])) < 1e-12 * np.max(res["M"])
    # azimuthal averages (trapezoid exact for these trig polynomials)
    gq = S.sphere_g(q * R_SPH) ** 2
    np.testing.assert_allclose(_avg(res["M"], nq, nth),
                               9 * BH ** 2 * M0 ** 2 * VS * gq * (2 * nx ** 2 + ny ** 2 + nz ** 2) / 2, rtol=1e-10)
    np.testing.assert_allclose(_avg(res["NM"], nq, nth), -9 * BH * M0 * N0 * VS * gq * nz, rtol=1e-9)
    np.testing.assert_allclose(_avg(res["P"], nq, nth),
                               9 * BH ** 2 * M0 ** 2 * VS * gq * (ny ** 2 + 3 * nz ** 2) / 8, rtol=1e-10)


def test_linear_vortex_2d_forms():
    nq, nth = 9, 24
    q, hy, hz, qa, T = _polar(nq, nth, 0.6, q0=0.02)
    M1 = 5 * M0 / R_SPH
    F = S.linear_vortex_amplitudes(qa, hy, hz, R_SPH, N0, M0, M1)
    res = S.responses(F, hy, hz, (0, 0, 1), BH, VS)
    g = S.sphere_g(qa * R_SPH)
    gp = S.sphere_gprime(qa * R_SPH)
    s, c = np.sin(T), np.cos(T)
    np.testing.assert_allclose(res["M"], 9 * BH ** 2 * VS * (M0 ** 2 * g ** 2 + M1 ** 2 * R_SPH ** 2 * gp ** 2) * s ** 2,
                               rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(res["NM"], -18 * BH * M0 * N0 * VS * g ** 2 * s ** 2, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(res["P"], 9 * BH ** 2 * M0 ** 2 * VS * g ** 2 * s ** 4, rtol=1e-10, atol=1e-14)
    # chiral term: printed as 18 V b^2 M0 M1 g g' sin^2 cos; dimensional reading adds R
    np.testing.assert_allclose(res["CHI"], 18 * VS * BH ** 2 * M0 * M1 * R_SPH * g * gp * s ** 2 * c,
                               rtol=1e-10, atol=1e-14)
    # the chiral term averages to zero (Eq. iqazi remark)
    assert np.max(np.abs(_avg(res["CHI"], nq, nth))) < 1e-12 * np.max(res["M"])


def _paper_polaris_perp(F, s, c, b, V):
    """The paper's expanded POLARIS/SANSPOL/unpolarized forms for P = e_z."""
    N, Mx, My, Mz = F
    sc = 1.0 / V
    cc = lambda a, bb: a * np.conj(bb) + np.conj(a) * bb
    yz = np.real(cc(My, Mz))
    nz_ = np.real(cc(N, Mz))
    ny_ = np.real(cc(N, My))
    chi = Mx * np.conj(My) * c ** 2 - np.conj(Mx) * My * c ** 2 - (Mx * np.conj(Mz) - np.conj(Mx) * Mz) * s * c
    ichi = np.real(1j * chi)
    base = abs(N) ** 2 / b ** 2 + abs(My) ** 2 * s ** 2 * c ** 2 + abs(Mz) ** 2 * s ** 4 - yz * s ** 3 * c
    pp = sc * b ** 2 * (base - nz_ * s ** 2 / b + ny_ * s * c / b)
    mm = sc * b ** 2 * (base + nz_ * s ** 2 / b - ny_ * s * c / b)
    sf0 = abs(Mx) ** 2 + abs(My) ** 2 * c ** 4 + abs(Mz) ** 2 * s ** 2 * c ** 2 - yz * s * c ** 3
    pm = sc * b ** 2 * (sf0 - ichi)
    mp = sc * b ** 2 * (sf0 + ichi)
    u0 = abs(N) ** 2 / b ** 2 + abs(Mx) ** 2 + abs(My) ** 2 * c ** 2 + abs(Mz) ** 2 * s ** 2 - yz * s * c
    sp = sc * b ** 2 * (u0 - nz_ * s ** 2 / b + ny_ * s * c / b - ichi)
    sm = sc * b ** 2 * (u0 + nz_ * s ** 2 / b - ny_ * s * c / b + ichi)
    un = sc * b ** 2 * u0
    return dict(PP=pp, MM=mm, PM=pm, MP=mp, SANSPOL_P=sp, SANSPOL_M=sm, UNPOL=un)


def _paper_polaris_para(F, s, c, b, V):
    """The paper's expanded forms for P = e_x (parallel geometry)."""
    N, Mx, My, Mz = F
    sc = 1.0 / V
    cc = lambda a, bb: np.real(a * np.conj(bb) + np.conj(a) * bb)
    pp = sc * b ** 2 * (abs(N) ** 2 / b ** 2 + abs(Mx) ** 2 - cc(N, Mx) / b)
    mm = sc * b ** 2 * (abs(N) ** 2 / b ** 2 + abs(Mx) ** 2 + cc(N, Mx) / b)
    sf = sc * b ** 2 * (abs(My) ** 2 * c ** 2 + abs(Mz) ** 2 * s ** 2 - cc(My, Mz) * s * c)
    u0 = abs(N) ** 2 / b ** 2 + abs(Mx) ** 2 + abs(My) ** 2 * c ** 2 + abs(Mz) ** 2 * s ** 2 - cc(My, Mz) * s * c
    sp = sc * b ** 2 * (u0 - cc(N, Mx) / b)
    sm = sc * b ** 2 * (u0 + cc(N, Mx) / b)
    return dict(PP=pp, MM=mm, PM=sf, MP=sf, SANSPOL_P=sp, SANSPOL_M=sm, UNPOL=sc * b ** 2 * u0)


@pytest.mark.parametrize("geometry", ["perp", "para"])
def test_expanded_polaris_forms_random_amplitudes(geometry):
    rng = np.random.default_rng(5)
    npix = 200
    th = rng.uniform(0, 2 * np.pi, npix)
    F = rng.normal(size=(4, npix)) + 1j * rng.normal(size=(4, npix))
    b, V = 1.7, 2.3
    P = (0, 0, 1) if geometry == "perp" else (1, 0, 0)
    res = S.responses(F, np.sin(th), np.cos(th), P, b, V)
    ref = (_paper_polaris_perp if geometry == "perp" else _paper_polaris_para)(F, np.sin(th), np.cos(th), b, V)
    for k, v in ref.items():
        np.testing.assert_allclose(res[k], v, rtol=1e-11, atol=1e-11, err_msg=k)
    if geometry == "para":
        assert np.max(np.abs(res["CHI"])) < 1e-12 * np.max(np.abs(res["M"]))


def test_cross_spectra_and_qsq():
    rng = np.random.default_rng(9)
    F = rng.normal(size=(4, 50)) + 1j * rng.normal(size=(4, 50))
    th = rng.uniform(0, 2 * np.pi, 50)
    res = S.responses(F, np.sin(th), np.cos(th))
    np.testing.assert_allclose(res["G_XY_RE"] + 1j * res["G_XY_IM"], F[1] * np.conj(F[2]))
    np.testing.assert_allclose(res["G_ZZ_IM"], 0.0, atol=1e-14)
    # Eq. HJdef1: Qx = -Mx, Qy = -My c^2 + Mz s c, Qz = My s c - Mz s^2
    s, c = np.sin(th), np.cos(th)
    np.testing.assert_allclose(res["QX2"], abs(F[1]) ** 2)
    np.testing.assert_allclose(res["QY2"], abs(-F[2] * c ** 2 + F[3] * s * c) ** 2, rtol=1e-12)
    np.testing.assert_allclose(res["QZ2"], abs(F[2] * s * c - F[3] * s ** 2) ** 2, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------- Fourier sum
def test_dsft_bruteforce_tiny():
    f = I.small_random_field(10, seed=3)
    R = S.sample_rotation(33.0, -71.0)
    rng = np.random.default_rng(1)
    qy, qz = rng.uniform(-2, 2, 37), rng.uniform(-2, 2, 37)
    pr = S.rotate_cells(f.pos, R)
    w = S.cell_weights(f.vol, f.nuc, f.mag, R)
    np.testing.assert_allclose(S.dsft(pr[:, 1], pr[:, 2], w, qy, qz),
                               S.dsft_bruteforce(pr, w, qy, qz), rtol=1e-12, atol=1e-12)


def test_dsft_hand_expanded_two_cells():
    # F = w1 e^{-i q.r1} + w2 e^{-i q.r2} written out by hand
    Y = np.array([1.5, -0.25])
    Z = np.array([0.5, 2.0])
    w = np.zeros((4, 2))
    w[0] = [2.0, -1.0]
    qy, qz = np.array([0.7]), np.array([-1.1])
    p1, p2 = 0.7 * 1.5 - 1.1 * 0.5, 0.7 * -0.25 - 1.1 * 2.0
    exp = 2.0 * (np.cos(p1) - 1j * np.sin(p1)) - 1.0 * (np.cos(p2) - 1j * np.sin(p2))
    assert abs(S.dsft(Y, Z, w, qy, qz)[0, 0] - exp) < 1e-14


def test_two_point_scatterers():
    d = np.array([0.0, 3.0, -1.25])
    Y = np.array([0.4, 0.4 + d[1]])
    Z = np.array([-0.2, -0.2 + d[2]])
    w = np.zeros((4, 2))
    w[0] = 1.0
    rng = np.random.default_rng(2)
    qy, qz = rng.uniform(-3, 3, 101), rng.uniform(-3, 3, 101)
    F = S.dsft(Y, Z, w, qy, qz)
    np.testing.assert_allclose(np.abs(F[0]) ** 2, 2 + 2 * np.cos(qy * d[1] + qz * d[2]), rtol=1e-12, atol=1e-12)


def test_q_zero_is_weight_sum():
    f = I.sphere_vortex(8.0, 1.0, seed=2)
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    F = S.dsft(f.pos[:, 1], f.pos[:, 2], w, np.array([0.0]), np.array([0.0]))
    np.testing.assert_allclose(F[:, 0].real, w.sum(1), rtol=1e-13, atol=1e-10)
    assert np.max(np.abs(F[:, 0].imag)) == 0.0


def test_dirichlet_box_closed_form():
    f = I.box_field(6, 11, 8, a=1.5, n_modes=4, seed=3, pores=False)
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    rng = np.random.default_rng(4)
    qy, qz = rng.uniform(-2, 2, 64), rng.uniform(-2, 2, 64)
    F = S.dsft(f.pos[:, 1], f.pos[:, 2], w, qy, qz)

    def D(k, n, a):
        x = k * a / 2
        return np.where(np.abs(x) < 1e-12, n, np.sin(n * x) / np.where(np.abs(x) < 1e-12, 1, np.sin(x)))

    exact = 1.5 ** 3 * 6 * D(qy, 11, 1.5) * D(qz, 8, 1.5)
    np.testing.assert_allclose(F[0], exact, rtol=1e-11, atol=1e-11 * 1.5 ** 3 * 6 * 11 * 8)


def test_translation_invariance_and_hermitian():
    f = I.small_random_field(40, seed=8)
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    rng = np.random.default_rng(3)
    qy, qz = rng.uniform(-2, 2, 50), rng.uniform(-2, 2, 50)
    F1 = S.dsft(f.pos[:, 1], f.pos[:, 2], w, qy, qz)
    F2 = S.dsft(f.pos[:, 1] + 7.3, f.pos[:, 2] - 2.9, w, qy, qz)
    np.testing.assert_allclose(np.abs(F1) ** 2, np.abs(F2) ** 2, rtol=1e-10)
    Fm = S.dsft(f.pos[:, 1], f.pos[:, 2], w, -qy, -qz)
    np.testing.assert_allclose(Fm, np.conj(F1), rtol=1e-12, atol=1e-12)


def test_rotation_90_is_permutation():
    f = I.small_random_field(30, seed=12)
    rng = np.random.default_rng(6)
    qy, qz = rng.uniform(-2, 2, 40), rng.uniform(-2, 2, 40)
    x, y, z = f.pos.T
    mx, my, mz = f.mag.T
    v = f.vol
    # about x by +90 deg: (x, y, z) -> (x, -z, y), same for M
    Rx = np.array([[1.0, 0, 0], [0, 0, -1.0], [0, 1.0, 0]])
    w_perm = np.stack([v * f.nuc, v * mx, -v * mz, v * my])
    got = S.amplitudes(f, Rx, qy, qz)
    np.testing.assert_allclose(got, S.dsft(-z, y, w_perm, qy, qz), rtol=1e-12, atol=1e-12)
    # the paper's R(alpha = 90, beta = 0) maps e_z to e_x: (x, y, z) -> (z, y, -x)
    R = S.sample_rotation(90.0, 0.0)
    np.testing.assert_allclose(R @ np.array([0, 0, 1.0]), [1, 0, 0], atol=1e-15)
    w_perm = np.stack([v * f.nuc, v * mz, v * my, -v * mx])
    np.testing.assert_allclose(S.amplitudes(f, R, qy, qz), S.dsft(y, -x, w_perm, qy, qz), rtol=1e-12, atol=1e-12)
    # R_z(90): (x, y, z) -> (-y, x, z)
    R = S.sample_rotation(0.0, 90.0)
    w_perm = np.stack([v * f.nuc, -v * my, v * mx, v * mz])
    np.testing.assert_allclose(S.amplitudes(f, R, qy, qz), S.dsft(x, z, w_perm, qy, qz), rtol=1e-12, atol=1e-12)


def test_lattice_sphere_converges_to_form_factor():
    q = np.linspace(0.0, 0.8, 41)
    qy, qz = q * np.sin(0.3), q * np.cos(0.3)
    errs = []
    for a in (1.0, 0.5):
        pos = I.lattice_ball(10.0, a)
        w = np.zeros((4, len(pos)))
        w[0] = a ** 3
        F = S.dsft(pos[:, 1], pos[:, 2], w, qy, qz)[0]
        Vs = 4 / 3 * np.pi * 1000.0
        errs.append(np.max(np.abs(F.real - 3 * Vs * S.sphere_g(q * 10.0))) / Vs)
    assert errs[1] < errs[0] and errs[1] < 2e-2


def test_even_field_has_no_chiral_term():
    # M(r) = M(-r) => M~ real => chi = 0 (paper, remark after Eq. ChiralSANS)
    pos = I.lattice_ball(6.0, 1.0)
    m = np.stack([pos[:, 0] * pos[:, 1], np.cos(pos[:, 2]), pos[:, 2] ** 2], axis=1)
    f = I.Field(pos, np.ones(len(pos)), np.ones(len(pos)), m)
    g = S.q_grid("cartesian", 9, 9, -1, 1, -1, 1)
    F = S.amplitudes(f, np.eye(3), g[0], g[1])
    res = S.responses(F, g[2], g[3])
    assert np.max(np.abs(res["CHI"])) < 1e-9 * np.max(res["M"])


def test_saturated_spin_flip_pattern():
    # saturated M || e_z: sf = M - P ~ sin^2 cos^2 (remark after Eq. sfperp)
    pos = I.lattice_ball(5.0, 1.0)
    f = I.Field(pos, np.ones(len(pos)), None, np.tile([0, 0, 1.0], (len(pos), 1)))
    g = S.q_grid("polar", 5, 36, 0.05, 0.5)
    F = S.amplitudes(f, np.eye(3), g[0], g[1])
    res = S.responses(F, g[2], g[3])
    th = 2 * np.pi * np.arange(36) / 36
    shape = (np.sin(th) * np.cos(th)) ** 2
    sf = res["SF"].reshape(5, 36)
    M2 = (np.abs(F[3]) ** 2).reshape(5, 36)
    np.testing.assert_allclose(sf, M2 * shape[None, :], rtol=1e-10, atol=1e-10 * M2.max())


# --------------------------------------------------------------- averages
def test_cartesian_ring_average_constant_and_counts():
    g = S.q_grid("cartesian", 64, 64, -1, 1, -1, 1)
    edges = np.linspace(0, 1, 17)
    Iq, cnt, qm = S.azimuthal_average_cartesian(np.full(64 * 64, 3.5), g[4], edges)
    np.testing.assert_allclose(Iq[cnt > 0], 3.5)
    assert cnt.sum() == int(np.sum(g[4] < 1.0))
    assert np.all((qm[cnt > 0] >= edges[:-1][cnt > 0]) & (qm[cnt > 0] < edges[1:][cnt > 0]))


def test_polar_average_is_exact_trapezoid():
    # (1/2pi) int sin^4 = 3/8, int cos^2 = 1/2 exactly for N_theta > 4
    g = S.q_grid("polar", 3, 12, 0.1, 0.3)
    th = 2 * np.pi * np.arange(12) / 12
    img = np.tile(np.sin(th) ** 4 + 2 * np.cos(th) ** 2, 3)
    np.testing.assert_allclose(S.azimuthal_average_polar(img, 3, 12), 3 / 8 + 1.0, rtol=1e-14)


def test_interference_split_two_objects():
    # |F1 + F2 e^{-iq.d}|^2 = |F1|^2 + |F2|^2 + 2 Re(F1 conj(F2) e^{iq.d}) for identical objects
    pos = I.lattice_ball(3.0, 1.0)
    n = len(pos)
    f = I.Field(np.vstack([pos, pos]), np.ones(2 * n), np.ones(2 * n), None,
                offsets=np.array([0, n, 2 * n]), centers=np.array([[0, 0, 0], [0, 9.0, -4.0]]))
    g = S.q_grid("cartesian", 7, 7, -1, 1, -1, 1)
    parts = S.response_parts(f, np.eye(3), g, ids=("N",))
    tot, dil, inter = parts["N"]
    F1 = S.amplitudes(I.Field(pos, np.ones(n), np.ones(n), None), np.eye(3), g[0], g[1])[0]
    np.testing.assert_allclose(dil, 2 * np.abs(F1) ** 2, rtol=1e-12)
    np.testing.assert_allclose(inter, 2 * np.abs(F1) ** 2 * np.cos(g[0] * 9.0 - g[1] * 4.0), rtol=1e-9,
                               atol=1e-9 * np.abs(F1).max() ** 2)


def test_interference_split_rotated_sample_moves_centres():
    # Sec. "Summation approach" with a sample orientation: the centres turn
    # with the sample, F_tot = F_1 + F_2 exp(-i q.(R d)).  For identical
    # objects every quadratic response then splits into 2 r_1 (dilute) and
    # 2 r_1 cos(q.(R d)) (interference), r_1 one rotated object's response;
    # nuclear, magnetic and spin-flip terms alike (Q is linear in F_M)
    rng = np.random.default_rng(5)
    pos = I.lattice_ball(3.0, 1.0)
    n = len(pos)
    mag = rng.normal(size=(n, 3))
    nuc = rng.uniform(0.5, 1.5, n)
    d = np.array([0.0, 9.0, -4.0]) + np.array([6.0, 0.0, 0.0])
    R = I.random_rotations(1, seed=12)[0]
    f = I.Field(np.vstack([pos, pos]), np.ones(2 * n), np.concatenate([nuc, nuc]), np.vstack([mag, mag]),
                offsets=np.array([0, n, 2 * n]), centers=np.array([[0.0, 0.0, 0.0], d]))
    g = S.q_grid("cartesian", 7, 9, -1, 1, -1.2, 0.8)
    ids = ("N", "M", "SF", "UNPOL")
    parts = S.response_parts(f, R, g, ids=ids)
    r1 = S.responses(S.amplitudes(I.Field(pos, np.ones(n), nuc, mag), R, g[0], g[1]), g[2], g[3])
    Rd = R @ d
    ph = np.cos(g[0] * Rd[1] + g[1] * Rd[2])
    for k in ids:
        tot, dil, inter = parts[k]
        scale = np.abs(r1[k]).max()
        np.testing.assert_allclose(dil, 2 * r1[k], rtol=1e-12, atol=1e-12 * scale)
        np.testing.assert_allclose(inter, 2 * r1[k] * ph, rtol=1e-9, atol=1e-9 * scale)

