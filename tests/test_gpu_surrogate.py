"""GPU tests of the learned surrogate and of its data generator.

- nms_plan_object_iq: per-object orientation-averaged I(q) against the oracle;
- nms_surrogate_gradients: BF16 forward/backward against the FP64 MLP oracle
  evaluated at the same parameters;
- checkpoint/resume: save -> load gives the same network and the same
  continued training;
- the gain: trained on curves of the vortex family computed by the batched
  transform, the network answers held-out queries orders of magnitude faster
  than the transform, at a stated error, judged by the transform itself.
"""
import time

import numpy as np
import pytest

from oracle import mlp as OM
from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from paper_2601_18444_gb300 import surrogate as SG

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_object_iq_matches_oracle():
    params = I.vortex_family_params(5, seed=2)
    params[:, 0] = np.array([6.0, 9.0, 7.5, 11.0, 8.0])        # small radii keep the oracle quick
    params[:, 1] = 2.0
    edges = np.geomspace(0.08, 1.2, 33)
    Iq, qmean, _, _ = SG.generate_curves(params, edges, a=1.5, n_rot=3, grid=SG.default_grid(1.2, 48))
    f = SG.family_field(params, a=1.5)
    rot = I.random_rotations(3, seed=11)
    g = S.q_grid("cartesian", 48, 48, -1.2, 1.2, -1.2, 1.2)
    for k in range(5):
        a, b = f.offsets[k], f.offsets[k + 1]
        fk = I.Field(f.pos[a:b], f.vol[a:b], f.nuc[a:b], f.mag[a:b])
        acc = 0.0
        for R in rot:
            acc = acc + S.responses(S.amplitudes(fk, R, g[0], g[1]), g[2], g[3])["UNPOL"]
        Ir, cr, _ = S.azimuthal_average_cartesian(acc / 3, g[4], edges)
        ok = np.isfinite(Ir)
        np.testing.assert_allclose(Iq[k][ok], Ir[ok], rtol=1e-5, atol=1e-8 * np.nanmax(Ir))
        assert np.array_equal(np.isnan(Iq[k]), ~ok)


def test_chunked_generation_matches_one_plan():
    # the large-family generator (members built by spawned workers, several
    # plans) gives every member its curve from one plan over all members, to
    # the I(q) bar (each plan scales its operands by its own largest weight,
    # so the FP32 roundings differ)
    params = I.vortex_family_params(7, seed=31)
    params[:, 0] = np.linspace(6.0, 12.0, 7)
    edges = np.geomspace(0.08, 1.2, 21)
    grid = SG.default_grid(1.2, 40)
    I1, _, _, _ = SG.generate_curves(params, edges, a=2.0, n_rot=3, grid=grid)
    I2, _, _, terms, _ = SG.generate_curves_chunked(params, edges, a=2.0, n_rot=3, grid=grid, chunk=3, workers=2)
    ok = np.isfinite(I1)
    assert np.array_equal(ok, np.isfinite(I2)) and terms > 0
    np.testing.assert_allclose(I2[ok], I1[ok], rtol=1e-5, atol=0.0)


@pytest.mark.parametrize("H", [32, 256])
def test_gradients_match_fp64_oracle(H):
    nin, nout, B = 6, 24, 96
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(nin, H, nout, lo, hi, seed=5)
    rng = np.random.default_rng(1)
    X = I.vortex_family_params(B, seed=3).astype(np.float32)
    T = rng.normal(size=(B, nout)).astype(np.float32)
    ym, ys = rng.normal(size=nout).astype(np.float32), rng.uniform(0.5, 2, size=nout).astype(np.float32)
    nms.nms_surrogate_set_target_stats(s, ym, ys)
    g, loss = nms.nms_surrogate_gradients(s, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    theta = nms.nms_surrogate_get_params(s)
    # the oracle sees the GEMM weights rounded to BF16, as the kernels do
    th = theta.astype(np.float64)
    o2 = H * nin + H
    o3 = o2 + H * H + H
    bf = lambda v: torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    th[o2:o2 + H * H] = bf(theta[o2:o2 + H * H])
    th[o3:o3 + nout * H] = bf(theta[o3:o3 + nout * H])
    loss_ref, g_ref = OM.loss_and_grad(th, X.astype(np.float64), T.astype(np.float64), lo.astype(np.float64),
                                       hi.astype(np.float64), ym.astype(np.float64), ys.astype(np.float64),
                                       nin, H, nout)
    assert abs(loss - loss_ref) <= 2e-2 * abs(loss_ref)
    # element by element: each gradient is a sum over the batch of products
    # formed from BF16-rounded activations (relative 2^-8 each); its error is
    # bounded by a small multiple of the sum of the terms' magnitudes
    mag = OM.grad_magnitude(th, X.astype(np.float64), T.astype(np.float64), lo.astype(np.float64),
                            hi.astype(np.float64), ym.astype(np.float64), ys.astype(np.float64), nin, H, nout)
    assert np.all(mag >= np.abs(g_ref) * (1 - 1e-12))
    bound = 3e-2 * mag + 1e-6 * mag.max()
    bad = np.flatnonzero(np.abs(g - g_ref) > bound)
    assert bad.size == 0, (bad[:8], g[bad[:8]], g_ref[bad[:8]], mag[bad[:8]])
    # and block by block in norm, as a second view
    off = [0, H * nin, o2, o2 + H * H, o3, o3 + nout * H, len(theta)]
    for a, b in zip(off[:-1], off[1:]):
        rel = np.linalg.norm(g[a:b] - g_ref[a:b]) / max(np.linalg.norm(g_ref[a:b]), 1e-30)
        assert rel <= 2e-2, (a, b, rel)
    s.close()


@pytest.mark.parametrize("H,nout,n", [(256, 55, 1000), (256, 64, 128), (256, 7, 37), (256, 128, 333),
                                      (256, 200, 301), (64, 55, 300)])
def test_inference_matches_fp64_oracle(H, nout, n):
    # H = 256 runs the fused tensor-core kernel, once per 128 outputs (ragged
    # last tile, a single tile, fewer rows than a tile, a full pass of 128,
    # two passes whose outputs are a part of each row); H = 64 the
    # layer-by-layer path.  Against the FP64 forward at the same parameters, with the GEMM
    # weights rounded to BF16 as the kernels use them; the remaining gap is
    # the BF16 rounding of the hidden activations.
    nin = 6
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(nin, H, nout, lo, hi, seed=9)
    rng = np.random.default_rng(2)
    ym, ys = rng.normal(size=nout).astype(np.float32), rng.uniform(0.5, 2, size=nout).astype(np.float32)
    nms.nms_surrogate_set_target_stats(s, ym, ys)
    X = I.vortex_family_params(n, seed=4).astype(np.float32)
    out = torch.full((n, nout), float("nan"), device="cuda")
    nms.nms_surrogate_infer(s, torch.tensor(X, device="cuda"), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    theta = nms.nms_surrogate_get_params(s).astype(np.float64)
    o2 = H * nin + H
    o3 = o2 + H * H + H
    bf = lambda v: torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    theta[o2:o2 + H * H] = bf(theta[o2:o2 + H * H])
    theta[o3:o3 + nout * H] = bf(theta[o3:o3 + nout * H])
    yn = OM.forward(theta, X.astype(np.float64), lo.astype(np.float64), hi.astype(np.float64), nin, H, nout)["Y"]
    ref = yn * ys.astype(np.float64) + ym.astype(np.float64)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / ys.astype(np.float64)       # in units of the standardised output
    assert err.max() <= 2e-2, err.max()
    assert np.sqrt(np.mean(err ** 2)) <= 4e-3
    s.close()


@pytest.mark.parametrize("nout,n", [(55, 4096), (128, 2048), (200, 1000)])
def test_inference_matches_bf16_activation_forward(nout, n):
    # The fused kernel against the FP64 network with its GEMM weights and
    # hidden activations rounded to BF16 where the kernel rounds them (after
    # each SiLU): what remains is the order of the FP32 sums, layer 1 in FP32
    # and the fast exponential and division in SiLU, which now and then move
    # a BF16 rounding decision of an activation by one unit.
    nin, H = 6, 256
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(nin, H, nout, lo, hi, seed=5)
    rng = np.random.default_rng(6)
    ym, ys = rng.normal(size=nout).astype(np.float32), rng.uniform(0.5, 2, size=nout).astype(np.float32)
    nms.nms_surrogate_set_target_stats(s, ym, ys)
    X = I.vortex_family_params(n, seed=7).astype(np.float32)
    out = torch.full((n, nout), float("nan"), device="cuda")
    nms.nms_surrogate_infer(s, torch.tensor(X, device="cuda"), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    bf = lambda v: torch.tensor(v, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    W1, b1, W2, b2, W3, b3 = OM.split(nms.nms_surrogate_get_params(s).astype(np.float64), nin, H, nout)
    Xn = 2.0 * (X.astype(np.float64) - lo) / (hi.astype(np.float64) - lo) - 1.0
    H1 = bf(OM.silu(Xn @ W1.T + b1))
    H2 = bf(OM.silu(H1 @ bf(W2).T + b2))
    ref = (H2 @ bf(W3).T + b3) * ys.astype(np.float64) + ym.astype(np.float64)
    err = np.abs(got - ref) / ys.astype(np.float64)
    rms = np.sqrt(np.mean(err ** 2))
    # measured on GB300: max 3.7e-3 .. 4.1e-3 (rounding flips), RMS 4.1e-5 .. 5.7e-5
    assert err.max() <= 1e-2 and rms <= 2e-4, (err.max(), rms)
    s.close()


def test_training_learns_and_checkpoint_resumes(tmp_path):
    nin, H, nout, n = 6, 64, 16, 4096
    lo = np.zeros(nin, np.float32)
    hi = np.ones(nin, np.float32)
    rng = np.random.default_rng(2)
    Xh = rng.random((n, nin)).astype(np.float32)
    W = rng.normal(size=(nin, nout))
    Yh = np.sin(Xh @ W).astype(np.float32)
    X = torch.tensor(Xh, device="cuda")
    Y = torch.tensor(Yh, device="cuda")
    s = nms.nms_surrogate_create(nin, H, nout, lo, hi, seed=1)
    l0 = nms.nms_surrogate_train(s, X, Y, batch=256, epochs=1, lr=2e-3, seed=0)
    l1 = nms.nms_surrogate_train(s, X, Y, batch=256, epochs=60, lr=2e-3, seed=1)
    assert l1 < 0.1 * l0, (l0, l1)
    path = tmp_path / "sur.bin"
    nms.nms_surrogate_save(s, path)
    cont = nms.nms_surrogate_train(s, X, Y, batch=256, epochs=3, lr=2e-3, seed=7)
    w_cont = nms.nms_surrogate_get_params(s)
    s2 = nms.nms_surrogate_create(nin, H, nout, lo, hi, seed=99)
    nms.nms_surrogate_load(s2, path)
    res = nms.nms_surrogate_train(s2, X, Y, batch=256, epochs=3, lr=2e-3, seed=7)
    assert np.array_equal(nms.nms_surrogate_get_params(s2), w_cont) and abs(res - cont) <= 1e-6 * abs(cont)
    out1 = torch.empty((n, nout), device="cuda")
    out2 = torch.empty((n, nout), device="cuda")
    nms.nms_surrogate_infer(s, X, out1)
    nms.nms_surrogate_infer(s2, X, out2)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)


def test_surrogate_gain_over_exact_transform():
    # scaled-down vortex family: a = 2.5 nm lattice, 16 orientations,
    # 128^2 detector, 64 log bins 0.04-1.2 nm^-1
    edges = np.geomspace(0.04, 1.2, 65)
    p_train = I.vortex_family_params(2048, seed=21)
    p_test = I.vortex_family_params(256, seed=22)
    I_tr, _, t_tr, terms_tr = SG.generate_curves(p_train, edges, a=2.5, n_rot=16)
    I_te, _, t_te, _ = SG.generate_curves(p_test, edges, a=2.5, n_rot=16)
    ok = np.all(np.isfinite(I_tr), axis=0) & np.all(np.isfinite(I_te), axis=0)
    Y_tr, Y_te = SG.log_targets(I_tr[:, ok]), SG.log_targets(I_te[:, ok])
    nout = int(ok.sum())
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(6, 256, nout, lo, hi, seed=3)
    X = torch.tensor(p_train.astype(np.float32), device="cuda")
    Y = torch.tensor(Y_tr, device="cuda")
    nms.nms_surrogate_train(s, X, Y, batch=128, epochs=400, lr=1e-3, seed=4)
    Xt = torch.tensor(p_test.astype(np.float32), device="cuda")
    out = torch.empty((len(p_test), nout), device="cuda")
    nms.nms_surrogate_infer(s, Xt, out)
    pred = out.cpu().numpy()
    rms = float(np.sqrt(np.mean((pred - Y_te) ** 2)))
    rms_mean_curve = float(np.sqrt(np.mean((Y_tr.mean(0) - Y_te) ** 2)))
    # time per query: surrogate on 1M queries vs exact transform per curve
    q = torch.tensor(I.vortex_family_params(1 << 20, seed=23).astype(np.float32), device="cuda")
    big = torch.empty((1 << 20, nout), device="cuda")
    nms.nms_surrogate_infer(s, q, big)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nms.nms_surrogate_infer(s, q, big)
    torch.cuda.synchronize()
    t_sur = (time.perf_counter() - t0) / (1 << 20)
    t_exact = t_te / len(p_test)
    print(f"surrogate: held-out rms {rms:.3f} dex (mean-curve predictor {rms_mean_curve:.3f}), "
          f"{t_sur * 1e9:.1f} ns/query vs exact {t_exact * 1e3:.3f} ms/curve -> x{t_exact / t_sur:.0f}")
    assert rms < 0.35 * rms_mean_curve
    assert t_exact / t_sur > 1000
    s.close()
