"""GPU parity of the angular spectrum (Eqs. CosineSinceIntensities,
ModalAmplitudes) and the 2D correlation function (Eq. crav2d) against the
oracle, on the polar grid and on Cartesian ring bins, through the C ABI.

Bars: the modal intensities are FP64 sums on both sides (relative 1e-11 of
the image scale; only the summation order differs); the 2D correlation uses
FP32 terms with two-float sums like the direct Fourier sum, so it is held to
|dC| <= 1e-6 sum_p |W_p f_p| (the amplitude bar), with the Gaussian's closed
form as an independent check.
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms

pytestmark = pytest.mark.gpu


def plan_for(grid_kw, n=40, prec=nms.PREC_FP32_DIRECT):
    f = I.small_random_field(n, seed=1, extent=3.0)
    g = nms.make_grid(**grid_kw)
    plan = nms.plan_from_field(f, g, nms.nms_options_default(precision=prec))
    nms.nms_amplitudes(plan)
    return plan


def og(grid_kw):
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    return S.q_grid(kind, **kw)


def test_angular_spectrum_polar_matches_oracle():
    kw = dict(kind="polar", n0=24, n1=72, lo0=0.0, hi0=1.5)
    plan = plan_for(kw)
    img = nms.nms_response(plan, "SF")
    out = nms.nms_angular_spectrum(plan, img, kmax=12, nbins=24)
    Ic, Is = S.angular_spectrum_polar(img, 24, 72, 12)
    sc = np.max(np.abs(img))
    np.testing.assert_allclose(out["Ic"], Ic, rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(out["Is"], Is, rtol=0, atol=1e-12 * sc)
    Ac, As = S.modal_amplitudes(Ic, Is)
    np.testing.assert_allclose(out["Ac"], Ac, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["As"], As, rtol=0, atol=1e-12)
    assert np.all(out["counts"] == 72)
    np.testing.assert_allclose(out["qmean"], np.linspace(0, 1.5, 24), rtol=1e-15)
    # device image in, same numbers
    import torch
    d = torch.tensor(img, device="cuda")
    out2 = nms.nms_angular_spectrum(plan, d, kmax=12, nbins=24)
    assert np.array_equal(out2["Ic"], out["Ic"]) and np.array_equal(out2["Is"], out["Is"])


def test_angular_spectrum_polar_anisotropy_ratios():
    # the paper's statements on the device: sin^2 -> A0/A2 = -1, sin^2 cos^2 -> A0/A4 = -1
    kw = dict(kind="polar", n0=8, n1=64, lo0=0.1, hi0=1.0)
    plan = plan_for(kw)
    g = og(kw)
    s2 = g[2] ** 2          # qhat_y = sin(theta)
    for img, k in ((s2 * np.exp(-g[4]), 2), (s2 * g[3] ** 2, 4)):
        out = nms.nms_angular_spectrum(plan, img, kmax=8, nbins=8)
        np.testing.assert_allclose(out["Ac"][0] / out["Ac"][k], -1.0, rtol=1e-12)


@pytest.mark.parametrize("nbins,kmax", [(17, 9), (1500, 8)])
def test_angular_spectrum_rings_match_oracle(nbins, kmax):
    # 17 bins: per-block shared-memory bins; 1500 x 19 rows: the global-bin path
    kw = dict(kind="cartesian", n0=96, n1=80, lo0=-1.1, hi0=1.3, lo1=-0.9, hi1=1.2)
    plan = plan_for(kw)
    g = og(kw)
    rng = np.random.default_rng(nbins)
    img = rng.normal(size=96 * 80) + 2.0 * g[2] ** 2
    edges = np.sort(np.concatenate([[0.0137], rng.uniform(0.02, 1.7, nbins - 1), [1.71]]))
    out = nms.nms_angular_spectrum(plan, img, kmax=kmax, bin_edges=edges)
    Ic, Is, cnt, qm = S.angular_spectrum_cartesian(img, g[0], g[1], edges, kmax)
    assert np.array_equal(out["counts"], cnt)
    ok = cnt > 0
    np.testing.assert_allclose(out["qmean"][ok], qm[ok], rtol=1e-13)
    assert np.all(np.isnan(out["Ic"][:, ~ok])) and np.all(np.isnan(out["qmean"][~ok]))
    sc = np.max(np.abs(img))
    np.testing.assert_allclose(out["Ic"][:, ok], Ic[:, ok], rtol=0, atol=1e-11 * sc)
    np.testing.assert_allclose(out["Is"][:, ok], Is[:, ok], rtol=0, atol=1e-11 * sc)
    Ac, As = S.modal_amplitudes(Ic, Is)
    np.testing.assert_allclose(out["Ac"], Ac, rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["As"], As, rtol=0, atol=1e-10)
    # the azimuthal average is the k = 0 mode
    Iq, c0, q0 = nms.nms_azimuthal_average(plan, img, edges)
    np.testing.assert_allclose(Iq[ok], out["Ic"][0, ok], rtol=1e-12)
    assert np.array_equal(c0, cnt)


def test_correlation_2d_cartesian_matches_oracle():
    kw = dict(kind="cartesian", n0=96, n1=80, lo0=-1.1, hi0=1.3, lo1=-0.9, hi1=1.2)
    plan = plan_for(kw)
    img = nms.nms_response(plan, "UNPOL")
    rho = np.linspace(0.0, 30.0, 13)
    alpha = np.linspace(0.0, 2 * np.pi, 11, endpoint=False)
    C, scale = nms.nms_correlation_2d(plan, img, rho, alpha)
    qy = np.linspace(-1.1, 1.3, 96)
    qz = np.linspace(-0.9, 1.2, 80)
    ref = S.correlation_2d_cartesian(img, qy, qz, rho, alpha)
    w = S.trapezoid_weights(qy)[:, None] * S.trapezoid_weights(qz)[None, :]
    sc_ref = np.sum(np.abs(w * img.reshape(96, 80)))
    np.testing.assert_allclose(scale, sc_ref, rtol=1e-12)
    assert np.max(np.abs(C - ref)) <= 1e-6 * sc_ref


def test_correlation_2d_polar_matches_oracle_and_device_output():
    import torch
    kw = dict(kind="polar", n0=40, n1=96, lo0=0.0, hi0=1.6)
    plan = plan_for(kw)
    img = nms.nms_response(plan, "SF")
    rho = np.array([0.0, 1.0, 4.0, 11.0, 25.0])
    alpha = np.array([0.0, 0.3, 1.9, 3.5, 5.0])
    ref = S.correlation_2d_polar(img, np.linspace(0, 1.6, 40), 96, rho, alpha)
    out = torch.empty((5, 5, 2), dtype=torch.float64, device="cuda")
    _, sc = nms.nms_correlation_2d(plan, torch.tensor(img, device="cuda"), rho, alpha, out=out)
    C = out[..., 0].cpu().numpy() + 1j * out[..., 1].cpu().numpy()
    assert np.max(np.abs(C - ref)) <= 1e-6 * float(sc.item())


def test_correlation_2d_gaussian_closed_form():
    # f = exp(-(a^2 q_y^2 + b^2 q_z^2)/2) on a wide grid: C = 2 pi/(a b) exp(-(rho_y^2/a^2 + rho_z^2/b^2)/2)
    a, b = 2.0, 3.5
    kw = dict(kind="cartesian", n0=321, n1=301, lo0=-14 / a, hi0=14 / a, lo1=-14 / b, hi1=14 / b)
    plan = plan_for(kw)
    g = og(kw)
    img = np.exp(-(a * a * g[0] ** 2 + b * b * g[1] ** 2) / 2)
    rho = np.array([0.0, 0.7, 2.0, 4.5])
    alpha = np.array([0.0, 0.4, np.pi / 2, 2.5, 4.0])
    C, sc = nms.nms_correlation_2d(plan, img, rho, alpha)
    ref = 2 * np.pi / (a * b) * np.exp(-(np.outer(rho, np.sin(alpha)) ** 2 / a ** 2
                                         + np.outer(rho, np.cos(alpha)) ** 2 / b ** 2) / 2)
    assert np.max(np.abs(C - ref)) <= 1e-6 * sc


def test_correlation_2d_full_detector_sampled():
    # 512 x 512 detector of the benchmark box grid and a 64 x 64 (rho, alpha)
    # output, checked against the oracle on a sample of outputs
    kw = dict(kind="cartesian", n0=512, n1=512, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
    plan = plan_for(kw, n=200)
    img = nms.nms_response(plan, "UNPOL")
    rho = np.linspace(0.0, 60.0, 64)
    alpha = np.linspace(0.0, np.pi, 64, endpoint=False)
    C, sc = nms.nms_correlation_2d(plan, img, rho, alpha)
    q = np.linspace(-2.0, 2.0, 512)
    rng = np.random.default_rng(2)
    for m, n in zip(rng.integers(0, 64, 6), rng.integers(0, 64, 6)):
        ref = S.correlation_2d_cartesian(img, q, q, [rho[m]], [alpha[n]])[0, 0]
        assert abs(C[m, n] - ref) <= 1e-6 * sc, (m, n)


def test_errors():
    plan = plan_for(dict(kind="list", n0=3, qlist=np.array([[0.1, 0.2], [0.3, -0.1], [0.0, 0.5]])))
    img = np.ones(3)
    with pytest.raises(nms.NmsError) as e:
        nms.nms_correlation_2d(plan, img, [1.0], [0.0])
    assert e.value.status == 4
    with pytest.raises(nms.NmsError) as e:
        nms.nms_angular_spectrum(plan, img, kmax=-1, bin_edges=[0.0, 1.0])
    assert e.value.status == 1
    pol = plan_for(dict(kind="polar", n0=4, n1=16, lo0=0.0, hi0=1.0))
    with pytest.raises(nms.NmsError):
        nms.nms_angular_spectrum(pol, np.ones(64), kmax=2, nbins=5)
