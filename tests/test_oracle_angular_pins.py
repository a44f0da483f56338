"""Pins of the oracle's angular spectrum (Eqs. CosineSinceIntensities and
ModalAmplitudes) and 2D correlation function (Eq. crav2d).

Independent facts used: the anisotropy ratios the paper states for the
two-fold sin^2 and four-fold sin^2 cos^2 patterns, the discrete orthogonality
of sines and cosines on an equispaced periodic grid (exact recovery of a trig
polynomial), the k = 0 mode as the azimuthal average, the symmetry of a
square detector, the closed-form 2D Fourier transform of an anisotropic
Gaussian and the Hankel transform of an isotropic one, a library trapezoid
at rho = 0, and the conjugate symmetry of the transform of a real image.
"""
import numpy as np
from scipy.integrate import trapezoid

from oracle import sans as S


def _polar_image(fun, n_q=5, n_theta=64, q0=0.1, q1=1.0):
    q = np.linspace(q0, q1, n_q)
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    Q, T = np.meshgrid(q, th, indexing="ij")
    return q, th, fun(Q, T).ravel()


def test_twofold_and_fourfold_anisotropy_ratios():
    # the paper: sin^2 theta gives A_0^c / A_2^c = -1, sin^2 cos^2 gives A_0^c / A_4^c = -1
    for fun, k in ((lambda Q, T: np.exp(-Q) * np.sin(T) ** 2, 2),
                   (lambda Q, T: (1 + Q) * np.sin(T) ** 2 * np.cos(T) ** 2, 4)):
        q, th, img = _polar_image(fun)
        Ic, Is = S.angular_spectrum_polar(img, len(q), len(th), kmax=8)
        Ac, As = S.modal_amplitudes(Ic, Is)
        np.testing.assert_allclose(Ac[0] / Ac[k], -1.0, rtol=1e-12)
        others = [j for j in range(9) if j not in (0, k)]
        assert np.max(np.abs(Ac[others])) < 1e-14 and np.max(np.abs(As)) < 1e-14
        # normalisation: sum_k sqrt(As^2 + Ac^2) = 1
        np.testing.assert_allclose(np.sum(np.hypot(Ac, As)), 1.0, rtol=1e-14)


def test_trig_polynomial_recovered_exactly():
    rng = np.random.default_rng(3)
    n_q, n_theta, kmax = 4, 32, 10
    c = rng.normal(size=(7, n_q))
    s = rng.normal(size=(7, n_q))
    s[0] = 0.0
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    f = np.zeros((n_q, n_theta))
    for k in range(7):
        f += np.outer(c[k], np.cos(k * th)) + np.outer(s[k], np.sin(k * th))
    Ic, Is = S.angular_spectrum_polar(f.ravel(), n_q, n_theta, kmax)
    np.testing.assert_allclose(Ic[:7], c, atol=1e-13)
    np.testing.assert_allclose(Is[:7], s, atol=1e-13)
    assert np.max(np.abs(Ic[7:])) < 1e-13 and np.max(np.abs(Is[7:])) < 1e-13


def test_mode_zero_is_the_azimuthal_average():
    rng = np.random.default_rng(4)
    img = rng.normal(size=6 * 24)
    Ic, _ = S.angular_spectrum_polar(img, 6, 24, 3)
    np.testing.assert_allclose(Ic[0], S.azimuthal_average_polar(img, 6, 24), rtol=1e-14)
    g = S.q_grid("cartesian", 40, 40, -1, 1, -1, 1)
    img = rng.normal(size=40 * 40)
    edges = np.linspace(0, 1, 11)
    Ic, Is, cnt, qm = S.angular_spectrum_cartesian(img, g[0], g[1], edges, 4)
    I0, cnt0, qm0 = S.azimuthal_average_cartesian(img, g[4], edges)
    np.testing.assert_allclose(Ic[0], I0, rtol=1e-13)
    assert np.array_equal(cnt, cnt0)
    np.testing.assert_allclose(qm, qm0, rtol=1e-14)


def test_square_detector_symmetry():
    # a constant image on a square detector symmetric about q = 0: the pixel
    # set of every ring is invariant under 90-degree turns and under
    # q_y -> -q_y, so only cosine modes with k = 0 mod 4 survive
    g = S.q_grid("cartesian", 48, 48, -1, 1, -1, 1)
    edges = np.linspace(0.05, 1.0, 9)
    Ic, Is, cnt, _ = S.angular_spectrum_cartesian(np.ones(48 * 48), g[0], g[1], edges, 9)
    np.testing.assert_allclose(Ic[0], 1.0, rtol=1e-14)
    for k in range(1, 10):
        assert np.max(np.abs(Is[k])) < 1e-13
        if k % 4:
            assert np.max(np.abs(Ic[k])) < 1e-13, k
    assert np.max(np.abs(Ic[4])) > 1e-3     # the square's own fourfold harmonic
    # the angle convention: f = q_y^2/q^2 = sin^2(theta) has mean 1/2 and
    # I_2^c = 2 <sin^2 cos 2theta> = -(1 + <cos 4theta>)/2 = -(1 + I_4^c[1]/2)/2
    qa2 = g[0] ** 2 + g[1] ** 2
    f = np.where(qa2 > 0, g[0] ** 2 / np.where(qa2 > 0, qa2, 1.0), 0.0)
    Jc, Js, _, _ = S.angular_spectrum_cartesian(f, g[0], g[1], edges, 4)
    np.testing.assert_allclose(Jc[0], 0.5, rtol=1e-13)
    np.testing.assert_allclose(Jc[2], -(1 + Ic[4] / 2) / 2, rtol=1e-12)


def test_corr2d_cartesian_anisotropic_gaussian():
    # f = exp(-(a^2 q_y^2 + b^2 q_z^2)/2): C = 2 pi/(a b) exp(-(rho_y^2/a^2 + rho_z^2/b^2)/2),
    # rho_y = rho sin(alpha), rho_z = rho cos(alpha); the trapezoid rule is
    # spectrally accurate for a Gaussian on a wide range
    a, b = 2.0, 3.5
    qy = np.linspace(-14 / a, 14 / a, 401)
    qz = np.linspace(-14 / b, 14 / b, 401)
    QY, QZ = np.meshgrid(qy, qz, indexing="ij")
    img = np.exp(-(a * a * QY ** 2 + b * b * QZ ** 2) / 2).ravel()
    rho = np.array([0.0, 0.7, 2.0, 4.5])
    alpha = np.array([0.0, 0.4, np.pi / 2, 2.5, 4.0])
    C = S.correlation_2d_cartesian(img, qy, qz, rho, alpha)
    ry = np.outer(rho, np.sin(alpha))
    rz = np.outer(rho, np.cos(alpha))
    ref = 2 * np.pi / (a * b) * np.exp(-(ry ** 2 / a ** 2 + rz ** 2 / b ** 2) / 2)
    np.testing.assert_allclose(C.real, ref, rtol=1e-10, atol=1e-12)
    assert np.max(np.abs(C.imag)) < 1e-12


def test_corr2d_polar_isotropic_gaussian_hankel():
    # f = exp(-sigma^2 q^2 / 2): C = 2 pi int q f J0(q rho) dq = (2 pi / sigma^2) exp(-rho^2/(2 sigma^2)),
    # independent of alpha.  The trapezoid in q exceeds the integral by the
    # Euler-Maclaurin end term h^2/12 (g'(q_max) - g'(0)) of
    # g(q) = q f(q) J0(q rho), with g'(0) = 1 and g'(q_max) ~ 0
    sig = 1.3
    q = np.linspace(0.0, 10.0 / sig, 4001)
    n_theta = 128
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    img = np.repeat(np.exp(-(sig * q) ** 2 / 2), n_theta)
    rho = np.array([0.0, 0.6, 1.3, 2.6])
    alpha = np.array([0.0, 1.0, 3.0])
    C = S.correlation_2d_polar(img, q, n_theta, rho, alpha)
    h = q[1] - q[0]
    ref = 2 * np.pi / sig ** 2 * np.exp(-rho ** 2 / (2 * sig ** 2)) - 2 * np.pi * h * h / 12
    np.testing.assert_allclose(C.real, np.repeat(ref[:, None], 3, axis=1), rtol=1e-9)
    assert np.max(np.abs(C.imag)) < 1e-9


def test_corr2d_rho_zero_and_conjugate_symmetry():
    rng = np.random.default_rng(5)
    qy = np.linspace(-1.2, 1.2, 25)
    qz = np.linspace(-0.8, 1.0, 31)
    QY, QZ = np.meshgrid(qy, qz, indexing="ij")
    img = (1.0 + 0.7 * QY + 0.3 * QZ ** 3 + 0.1 * rng.normal(size=QY.shape)).ravel()
    C0 = S.correlation_2d_cartesian(img, qy, qz, [0.0], [0.3])
    np.testing.assert_allclose(C0[0, 0].real, trapezoid(trapezoid(img.reshape(25, 31), qz, axis=1), qy), rtol=1e-13)
    alpha = np.array([0.2, 1.1])
    C = S.correlation_2d_cartesian(img, qy, qz, [1.7, 3.0], np.concatenate([alpha, alpha + np.pi]))
    np.testing.assert_allclose(C[:, 2:], np.conj(C[:, :2]), rtol=1e-12, atol=1e-12)
    # a centrosymmetric image has a real transform
    g = (np.cos(QY) * np.exp(-QZ ** 2)).ravel()
    qyz = np.linspace(-1, 1, 21)
    QY2, QZ2 = np.meshgrid(qyz, qyz, indexing="ij")
    g = (np.cos(2 * QY2) * np.exp(-QZ2 ** 2) + QY2 * QZ2).ravel()
    Cs = S.correlation_2d_cartesian(g, qyz, qyz, [0.5, 2.0], [0.0, 0.9, 2.0])
    assert np.max(np.abs(Cs.imag)) < 1e-12 * np.max(np.abs(Cs.real))
