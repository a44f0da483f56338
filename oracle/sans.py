"""FP64 CPU oracle of the SANS hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  It shares no code with the CUDA library: every
step is restated here from the paper in plain numpy (FP64), with the heavy
Fourier sum in ``dsft.c`` (plain FP64 loops, built by ``build_oracle``).

Steps and the passages they follow (paper section / equation):
  rotate_cells      Sec. "Real-space input data", X/Y/Z = R (x^{kl} + r^k),
                    R = R_z(beta) R_y(alpha) of Sec. "Configuration file".
  cell_weights      Sec. "Summation approach": n_j = N_j V_j, m_j = M_j V_j;
                    M is rotated with the sample (reading: M' = R M).
  dsft              Sec. "Summation approach" (DSFT, cos/sin split).
  q_grid            Detector plane q = (0, q_y, q_z), Eq. qdef; polar
                    (q, theta) grid of Sec. "Configuration file"; Cartesian
                    and list grids (reading: both supported).
  hj_vector         Eq. HJdef: Q = qhat x (qhat x M) = qhat (qhat . M) - M.
  responses         Eqs. NuclearSANS, MagneticSANS, PSANSdef, sfdef,
                    ChiralSANS, NMdef, POLARIS and SANSPOL definitions, the
                    unpolarized average (Sec. "Unpolarized SANS cross
                    sections") and the cross spectra G_ab of Sec. "Fourier and
                    real-space output data" (reported with the same 1/V
                    prefactor as the cross sections, like |Q_a|^2).  Prefactor 8 pi^3/V times the
                    (2 pi)^{-3} of the DSFT gives 1/V on the raw sums.
  dilute/total      Sec. "Summation approach", the interparticle
                    decomposition (form factor sum vs full amplitude).
  azimuthal_*       Eq. iqazi (trapezoidal rule; periodic in theta).
  correlation       Eqs. crrad and prrad (trapezoidal rule over the nodes).
  angular_spectrum_* Eq. CosineSinceIntensities (sine/cosine harmonics of
                    the 2D image over theta) and modal_amplitudes, Eq.
                    ModalAmplitudes.
  correlation_2d_*  Eq. crav2d (inverse 2D transform of the image; trapezoid
                    rule in q and theta, or in q_y and q_z).
  sphere_*/vortex_* Sec. "Spherical form factor model" and the linear vortex
                    section (analytic amplitudes used as pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

# Response names, in the paper's vocabulary.
RESPONSES = ["N", "M", "P", "NM", "CHI", "SF", "PM", "MP", "PP", "MM",
             "SANSPOL_P", "SANSPOL_M", "UNPOL"]
CROSS = [f"G_{a}{b}_{p}" for a in "XYZ" for b in "XYZ" for p in ("RE", "IM")]
QSQ = ["QX2", "QY2", "QZ2"]
ALL_IDS = RESPONSES + CROSS + QSQ


# --------------------------------------------------------------------------
# C direct sum
# --------------------------------------------------------------------------
def build_oracle(force=False):
    """Compile dsft.c with gcc (FP64, OpenMP) into oracle/_build."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    src = os.path.join(_HERE, "dsft.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        so = build_oracle()
        lib = ctypes.CDLL(so)
        d = ctypes.POINTER(ctypes.c_double)
        lib.oracle_dsft.argtypes = [ctypes.c_int64, d, d, d, ctypes.c_int64, d, d, d, d]
        lib.oracle_dsft.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def oracle_threads():
    return int(_lib().oracle_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dsft(Y, Z, w, qy, qz):
    """F[c, i] = sum_j w[c, j] exp(-i (qy_i Y_j + qz_i Z_j)), complex128 [4, nq]."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    qy = np.ascontiguousarray(qy, dtype=np.float64).ravel()
    qz = np.ascontiguousarray(qz, dtype=np.float64).ravel()
    n, nq = Y.shape[0], qy.shape[0]
    assert w.shape == (4, n)
    re = np.zeros((4, nq))
    im = np.zeros((4, nq))
    if n and nq:
        _lib().oracle_dsft(n, _p(Y), _p(Z), _p(w), nq, _p(qy), _p(qz), _p(re), _p(im))
    return re + 1j * im


def dsft_bruteforce(pos_rot, w, qy, qz):
    """Small-case DSFT as a complex matrix product, for pinning ``dsft``."""
    qvec = np.stack([np.zeros_like(qy), qy, qz], axis=1)          # [nq,3]
    ph = np.exp(-1j * (qvec @ pos_rot.T))                            # [nq,n]
    return (ph @ w.T.astype(np.complex128)).T                        # [4,nq]


# --------------------------------------------------------------------------
# rotation and weights
# --------------------------------------------------------------------------
def rot_y(alpha):
    c, s = np.cos(alpha), np.sin(alpha)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_z(beta):
    c, s = np.cos(beta), np.sin(beta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def sample_rotation(alpha_deg, beta_deg):
    """R(alpha, beta) = R_z(beta) R_y(alpha); alpha = 90 deg maps e_z to e_x."""
    return rot_z(np.deg2rad(beta_deg)) @ rot_y(np.deg2rad(alpha_deg))


def rotate_cells(pos, R, offsets=None, centers=None, use_centers=True):
    """Rotated global positions R (x^{kl} + r^k) -> [n,3]."""
    p = np.array(pos, dtype=np.float64, copy=True)
    if use_centers and centers is not None:
        for k in range(len(offsets) - 1):
            p[offsets[k]:offsets[k + 1]] += centers[k]
    return p @ np.asarray(R).T


def cell_weights(vol, nuc, mag, R):
    """w[4, n] = V_j (N_j, (R M_j)_x, (R M_j)_y, (R M_j)_z); absent channels are 0."""
    n = vol.shape[0]
    w = np.zeros((4, n))
    if nuc is not None:
        w[0] = vol * nuc
    if mag is not None:
        w[1:] = (mag @ np.asarray(R).T).T * vol[None, :]
    return w


# --------------------------------------------------------------------------
# detector grids
# --------------------------------------------------------------------------
def q_grid(kind, n0=0, n1=0, lo0=0.0, hi0=0.0, lo1=0.0, hi1=0.0, qlist=None):
    """Return (qy, qz, qhat_y, qhat_z, |q|) flattened row-major.

    cartesian: q_y[a] = lo0 + (hi0-lo0) a/(n0-1), q_z[b] likewise over n1
               (endpoints included; n = 1 gives lo); pixel (a, b) row-major.
    polar:     q_i = lo0 + (hi0-lo0) i/(n0-1), theta_j = 2 pi j/n1;
               q_y = q sin theta, q_z = q cos theta (Eq. qdef); qhat uses theta
               even at q = 0.
    list:      n0 (q_y, q_z) pairs.
    Where |q| = 0 on the cartesian and list grids, qhat = e_z.
    """
    def lin(n, lo, hi):
        if n == 1:
            return np.array([lo], dtype=np.float64)
        return lo + (hi - lo) * np.arange(n, dtype=np.float64) / (n - 1)

    if kind == "cartesian":
        qy1 = lin(n0, lo0, hi0)
        qz1 = lin(n1, lo1, hi1)
        qy = np.repeat(qy1, n1)
        qz = np.tile(qz1, n0)
    elif kind == "list":
        ql = np.asarray(qlist, dtype=np.float64).reshape(-1, 2)
        qy, qz = ql[:, 0].copy(), ql[:, 1].copy()
    elif kind == "polar":
        qm = lin(n0, lo0, hi0)
        th = 2.0 * np.pi * np.arange(n1) / n1
        Q, T = np.meshgrid(qm, th, indexing="ij")
        qy = (Q * np.sin(T)).ravel()
        qz = (Q * np.cos(T)).ravel()
        qa = Q.ravel()
        return qy, qz, np.sin(T).ravel(), np.cos(T).ravel(), qa
    else:
        raise ValueError(kind)
    qa = np.hypot(qy, qz)
    safe = np.where(qa > 0, qa, 1.0)
    hy = np.where(qa > 0, qy / safe, 0.0)
    hz = np.where(qa > 0, qz / safe, 1.0)
    return qy, qz, hy, hz, qa


# --------------------------------------------------------------------------
# Halpern-Johnson vector and responses
# --------------------------------------------------------------------------
def hj_vector(FM, hy, hz):
    """Q = qhat (qhat . M) - M with qhat = (0, hy, hz); FM complex [3, np]."""
    proj = hy * FM[1] + hz * FM[2]
    return np.stack([-FM[0], hy * proj - FM[1], hz * proj - FM[2]])


def responses(F, hy, hz, P=(0.0, 0.0, 1.0), b_H=1.0, V=1.0):
    """All response ids from raw amplitudes F (complex [4, np]) -> dict of real [np]."""
    s = 1.0 / V
    FN = F[0]
    FM = F[1:4]
    Q = hj_vector(FM, hy, hz)
    P = np.asarray(P, dtype=np.float64)
    PQ = P[0] * Q[0] + P[1] * Q[1] + P[2] * Q[2]
    QxQc = np.stack([Q[1] * np.conj(Q[2]) - Q[2] * np.conj(Q[1]),
                     Q[2] * np.conj(Q[0]) - Q[0] * np.conj(Q[2]),
                     Q[0] * np.conj(Q[1]) - Q[1] * np.conj(Q[0])])
    chi = P[0] * QxQc[0] + P[1] * QxQc[1] + P[2] * QxQc[2]
    out = {}
    out["N"] = s * np.abs(FN) ** 2
    out["M"] = s * b_H ** 2 * (np.abs(Q) ** 2).sum(0)
    out["P"] = s * b_H ** 2 * np.abs(PQ) ** 2
    out["NM"] = s * b_H * np.real(FN * np.conj(PQ) + np.conj(FN) * PQ)
    out["CHI"] = np.real(-1j * s * b_H ** 2 * chi)
    out["SF"] = out["M"] - out["P"]
    out["PM"] = out["SF"] + out["CHI"]
    out["MP"] = out["SF"] - out["CHI"]
    out["PP"] = out["N"] + out["NM"] + out["P"]
    out["MM"] = out["N"] - out["NM"] + out["P"]
    out["SANSPOL_P"] = out["PP"] + out["PM"]
    out["SANSPOL_M"] = out["MM"] + out["MP"]
    out["UNPOL"] = 0.5 * (out["PP"] + out["MM"] + out["PM"] + out["MP"])
    names = "XYZ"
    for a in range(3):
        for b in range(3):
            g = s * FM[a] * np.conj(FM[b])
            out[f"G_{names[a]}{names[b]}_RE"] = np.real(g)
            out[f"G_{names[a]}{names[b]}_IM"] = np.imag(g)
    for a in range(3):
        out[f"Q{names[a]}2"] = s * np.abs(Q[a]) ** 2
    return out


def amplitudes(field, R, qy, qz, use_centers=True, per_object=False):
    """Raw amplitudes of a field under rotation R.

    per_object=False: the full sum over all cells (with centres if given).
    per_object=True:  list of F_k of each object with local positions only.
    """
    w = cell_weights(field.vol, field.nuc, field.mag, R)
    if not per_object:
        pr = rotate_cells(field.pos, R, field.offsets, field.centers, use_centers)
        return dsft(pr[:, 1], pr[:, 2], w, qy, qz)
    pr = field.pos @ np.asarray(R).T
    off = field.offsets if field.offsets is not None else np.array([0, field.n])
    out = []
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        out.append(dsft(pr[a:b, 1], pr[a:b, 2], w[:, a:b], qy, qz))
    return out


def response_parts(field, R, grid, ids=("UNPOL",), P=(0, 0, 1), b_H=1.0, V=1.0):
    """(total, dilute, interference) per id for one rotation (interparticle split)."""
    qy, qz, hy, hz, _ = grid
    tot = responses(amplitudes(field, R, qy, qz, use_centers=True), hy, hz, P, b_H, V)
    dil = None
    for Fk in amplitudes(field, R, qy, qz, per_object=True):
        r = responses(Fk, hy, hz, P, b_H, V)
        dil = r if dil is None else {k: dil[k] + r[k] for k in dil}
    res = {}
    for i in ids:
        res[i] = (tot[i], dil[i], tot[i] - dil[i])
    return res


# --------------------------------------------------------------------------
# azimuthal average and correlation functions
# --------------------------------------------------------------------------
def azimuthal_average_polar(img, n_q, n_theta):
    """Eq. iqazi on the polar grid: the periodic trapezoid is the mean over theta."""
    return np.asarray(img).reshape(n_q, n_theta).mean(axis=1)


def azimuthal_average_cartesian(img, qabs, edges):
    """Ring-bin mean over pixels with edges[b] <= |q| < edges[b+1].

    Returns (I, counts, qmean); empty bins give I = nan, qmean = nan.
    """
    img = np.asarray(img).ravel()
    qabs = np.asarray(qabs).ravel()
    nb = len(edges) - 1
    I = np.full(nb, np.nan)
    qm = np.full(nb, np.nan)
    cnt = np.zeros(nb, dtype=np.int64)
    for b in range(nb):
        sel = (qabs >= edges[b]) & (qabs < edges[b + 1])
        cnt[b] = int(sel.sum())
        if cnt[b]:
            I[b] = img[sel].mean()
            qm[b] = qabs[sel].mean()
    return I, cnt, qm


def spherical_j0(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def correlation(q, Iq, r, prefactor=1.0 / (2.0 * np.pi ** 2)):
    """Eq. crrad by the trapezoidal rule over the given nodes, and Eq. prrad.

    Nodes with non-finite I are dropped (empty bins).  Returns (c, p).
    """
    q = np.asarray(q, dtype=np.float64)
    Iq = np.asarray(Iq, dtype=np.float64)
    ok = np.isfinite(q) & np.isfinite(Iq)
    q, Iq = q[ok], Iq[ok]
    r = np.asarray(r, dtype=np.float64)
    c = np.zeros_like(r)
    for m, rm in enumerate(r):
        f = Iq * spherical_j0(q * rm) * q * q
        c[m] = prefactor * np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(q))
    return c, r * r * c


# --------------------------------------------------------------------------
# angular spectrum and 2D correlation function
# --------------------------------------------------------------------------
def angular_spectrum_polar(img, n_q, n_theta, kmax):
    """Eq. CosineSinceIntensities on the polar grid, theta_j = 2 pi j / n_theta.

    The periodic trapezoid turns the theta integral into a mean over j:
        I_k^{c,s}(q_i) = (2 - delta_k0) / n_theta * sum_j f(q_i, theta_j) {cos, sin}(k theta_j).
    Returns (Ic, Is), each [kmax + 1][n_q].
    """
    f = np.asarray(img, dtype=np.float64).reshape(n_q, n_theta)
    theta = 2.0 * np.pi * np.arange(n_theta) / n_theta
    k = np.arange(kmax + 1)
    pref = (2.0 - (k == 0)) / n_theta
    Ic = pref[:, None] * (np.cos(np.outer(k, theta)) @ f.T)
    Is = pref[:, None] * (np.sin(np.outer(k, theta)) @ f.T)
    return Ic, Is


def angular_spectrum_cartesian(img, qy, qz, edges, kmax):
    """Eq. CosineSinceIntensities on ring bins of a Cartesian or list grid.

    Reading (as for the azimuthal average): the theta integral over the ring
    edges[b] <= |q| < edges[b+1] is the mean over its pixels, with the pixel
    angle theta = atan2(q_y, q_z) (qhat = (0, sin theta, cos theta); theta = 0
    at q = 0).  Returns (Ic, Is, counts, qmean); empty bins give NaN.
    """
    f = np.asarray(img, dtype=np.float64).ravel()
    qy = np.asarray(qy, dtype=np.float64).ravel()
    qz = np.asarray(qz, dtype=np.float64).ravel()
    qa = np.hypot(qy, qz)
    th = np.arctan2(qy, qz)
    nb = len(edges) - 1
    Ic = np.full((kmax + 1, nb), np.nan)
    Is = np.full((kmax + 1, nb), np.nan)
    qm = np.full(nb, np.nan)
    cnt = np.zeros(nb, dtype=np.int64)
    for b in range(nb):
        sel = (qa >= edges[b]) & (qa < edges[b + 1])
        cnt[b] = int(sel.sum())
        if not cnt[b]:
            continue
        qm[b] = qa[sel].mean()
        for k in range(kmax + 1):
            pref = 1.0 if k == 0 else 2.0
            Ic[k, b] = pref * np.mean(f[sel] * np.cos(k * th[sel]))
            Is[k, b] = pref * np.mean(f[sel] * np.sin(k * th[sel]))
    return Ic, Is, cnt, qm


def modal_amplitudes(Ic, Is):
    """Eq. ModalAmplitudes: a_k = sum_i I_k(q_i) over the finite nodes, and
    A_k^{s,c} = a_k^{s,c} / sum_{j <= kmax} sqrt(|a_j^s|^2 + |a_j^c|^2).
    Returns (Ac, As)."""
    Ic = np.asarray(Ic, dtype=np.float64)
    Is = np.asarray(Is, dtype=np.float64)
    ac = np.where(np.isfinite(Ic), Ic, 0.0).sum(axis=1)
    as_ = np.where(np.isfinite(Is), Is, 0.0).sum(axis=1)
    den = np.sum(np.sqrt(as_ ** 2 + ac ** 2))
    return ac / den, as_ / den


def trapezoid_weights(x):
    """Weights of the trapezoidal rule on the nodes x (increasing)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.zeros_like(x)
    if len(x) > 1:
        d = np.diff(x)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
    return w


def correlation_2d_polar(img, q, n_theta, rho, alpha):
    """Eq. crav2d on the polar grid:
        C(rho, alpha) = sum_i sum_j wq_i q_i (2 pi / n_theta) f(q_i, theta_j)
                        exp(i q_i rho cos(theta_j - alpha)),
    trapezoid weights wq in q, periodic trapezoid in theta.  Returns complex
    C[len(rho)][len(alpha)]."""
    q = np.asarray(q, dtype=np.float64)
    f = np.asarray(img, dtype=np.float64).reshape(len(q), n_theta)
    theta = 2.0 * np.pi * np.arange(n_theta) / n_theta
    w = (trapezoid_weights(q) * q)[:, None] * (2.0 * np.pi / n_theta) * f
    C = np.zeros((len(rho), len(alpha)), dtype=np.complex128)
    for m, rm in enumerate(rho):
        for n, an in enumerate(alpha):
            C[m, n] = np.sum(w * np.exp(1j * np.outer(q, np.cos(theta - an)) * rm))
    return C


def correlation_2d_cartesian(img, qy_nodes, qz_nodes, rho, alpha):
    """Eq. crav2d on a Cartesian grid: q dq dtheta = dq_y dq_z and
    q rho cos(theta - alpha) = q_y rho sin(alpha) + q_z rho cos(alpha)
    (qhat = (0, sin theta, cos theta)), trapezoid weights in q_y and q_z:
        C(rho, alpha) = sum_{a,b} wy_a wz_b f_ab exp(i (q_y,a rho sin alpha + q_z,b rho cos alpha)).
    img is [n_y][n_z] (pixel a * n_z + b).  Returns complex C[len(rho)][len(alpha)]."""
    qy = np.asarray(qy_nodes, dtype=np.float64)
    qz = np.asarray(qz_nodes, dtype=np.float64)
    f = np.asarray(img, dtype=np.float64).reshape(len(qy), len(qz))
    w = trapezoid_weights(qy)[:, None] * trapezoid_weights(qz)[None, :] * f
    C = np.zeros((len(rho), len(alpha)), dtype=np.complex128)
    for m, rm in enumerate(rho):
        for n, an in enumerate(alpha):
            ey = np.exp(1j * qy * rm * np.sin(an))
            ez = np.exp(1j * qz * rm * np.cos(an))
            C[m, n] = ey @ w @ ez
    return C


# --------------------------------------------------------------------------
# analytic amplitudes (pins)
# --------------------------------------------------------------------------
def sphere_g(v):
    """g(v) = j1(v)/v = (sin v - v cos v)/v^3, g(0) = 1/3."""
    v = np.asarray(v, dtype=np.float64)
    out = np.full_like(v, 1.0 / 3.0)
    big = np.abs(v) > 1e-3
    vb = v[big]
    out[big] = (np.sin(vb) - vb * np.cos(vb)) / vb ** 3
    vs = v[~big]
    out[~big] = 1.0 / 3.0 - vs ** 2 / 30.0 + vs ** 4 / 840.0
    return out


def sphere_gprime(v):
    """g'(v) = ((v^2 - 3) sin v + 3 v cos v)/v^4, g'(0) = 0."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    big = np.abs(v) > 1e-3
    vb = v[big]
    out[big] = ((vb ** 2 - 3.0) * np.sin(vb) + 3.0 * vb * np.cos(vb)) / vb ** 4
    vs = v[~big]
    out[~big] = -vs / 15.0 + vs ** 3 / 210.0
    return out


def linear_vortex_amplitudes(qabs, hy, hz, R, N0, M0, M1):
    """Raw amplitudes (no (2 pi)^{-3/2}) of the uniform sphere with a linear
    vortex, Eqs. for N~ and M~ of the linear-vortex section with q_x = 0:
    F_N = 3 V N0 g,  F_M = 3 V [M0 g e_z + i M1 R g' (qhat_x e_y - qhat_y e_x)]."""
    Vs = 4.0 / 3.0 * np.pi * R ** 3
    g = sphere_g(qabs * R)
    gp = sphere_gprime(qabs * R)
    F = np.zeros((4, qabs.size), dtype=np.complex128)
    F[0] = 3.0 * Vs * N0 * g
    F[1] = 3.0 * Vs * (-1j * M1 * R * gp * hy)
    F[2] = 0.0
    F[3] = 3.0 * Vs * M0 * g
    return F


def uniform_sphere_amplitudes(qabs, R, N0, M0, n):
    """Raw amplitudes of the uniform sphere: F_N = 3 V N0 g, F_M = 3 V M0 g n."""
    Vs = 4.0 / 3.0 * np.pi * R ** 3
    g = sphere_g(qabs * R)
    F = np.zeros((4, qabs.size), dtype=np.complex128)
    F[0] = 3.0 * Vs * N0 * g
    for a in range(3):
        F[1 + a] = 3.0 * Vs * M0 * g * n[a]
    return F
