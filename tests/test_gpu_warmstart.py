"""The learned warm start: the tensor-core network against the CPU
reference network, training, and what the trained network gains over the
method without it on a demagnetisation curve."""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _params_list(flat):
    sizes = omlp.SIZES
    out, o = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + n_in * n_out].reshape(n_out, n_in).astype(np.float64)
        o += n_in * n_out
        b = flat[o:o + n_out].astype(np.float64)
        o += n_out
        out.append((W, b))
    return out


def test_forward_matches_reference():
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=3)
    p = net.get_params()
    p[16 * 128:16 * 128 + 128] = np.random.default_rng(0).normal(size=128) * 0.1   # nonzero b1
    net.set_params(p)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(301, 16)).astype(np.float32)          # ragged tail
    Y = net.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    Yr, _ = omlp.forward(_params_list(p), X.astype(np.float64), round_bf16=True)
    scale = np.abs(Yr).max()
    np.testing.assert_allclose(Y, Yr, rtol=0, atol=1e-2 * scale)


def test_gradient_matches_reference():
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=5)
    p = net.get_params()
    rng = np.random.default_rng(2)
    X = rng.normal(size=(517, 16)).astype(np.float32)
    T = rng.normal(size=(517, 4)).astype(np.float32)
    g, loss = net.gradient(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    lr, gr = omlp.loss_and_grads(_params_list(p), X.astype(np.float64), T.astype(np.float64),
                                 round_bf16=True)
    assert loss == pytest.approx(lr, rel=1e-2)
    gflat = _params_list(g)
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(gflat, gr)):
        sw, sb = np.abs(rw).max(), np.abs(rb).max()
        np.testing.assert_allclose(gw, rw, rtol=0, atol=3e-2 * sw, err_msg=f"W{l + 1}")
        np.testing.assert_allclose(gb, rb, rtol=0, atol=3e-2 * sb, err_msg=f"b{l + 1}")


def test_training_fits_a_smooth_map():
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=7)
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.normal(size=(20000, 16)), dtype=torch.float32, device="cuda")
    R = torch.tensor(rng.normal(size=(16, 4)) / 4, dtype=torch.float32, device="cuda")
    T = torch.tanh(X @ R).contiguous()
    first = net.train_step(X[:4096].contiguous(), T[:4096].contiguous(), 1e-3, want_loss=True)
    for i in range(400):
        j = (i * 4096) % (20000 - 4096)
        net.train_step(X[j:j + 4096].contiguous(), T[j:j + 4096].contiguous(), 1e-3)
    _, last = net.gradient(X, T)
    assert last < 0.2 * first


def test_warm_start_gain_on_a_demag_curve():
    """Train on the method's own trajectory of one jittered hard-magnetic
    cube, then run the curve of another jitter of it with and without the
    warm start: the corrected starts must not change the curve (NCG runs to
    t1-t3 either way) and must save NCG iterations."""
    import torch
    from paper_1801_03690_gb300 import MLP, Magnet, Params, warmstart
    prm = Params(jmax=4, precision=1)
    train_wl = synth.hard_cube(n_mag=10, seed=2, n_fields=40)
    test_wl = synth.hard_cube(n_mag=10, seed=9, n_fields=40)
    fields = train_wl.fields[:16]                 # 0 .. -3.1 T: reversible part of the curve
    mag = Magnet()
    mag.upload_workload(train_wl)
    n_mag = mag.sizes()["n_mag"]
    net = MLP(seed=11)
    X, T, _ = warmstart.collect(mag, net, train_wl.m0, fields, n_mag, prm)
    s_m, s_p, _ = warmstart.train(net, X, T, steps=600, batch=8192, lr=2e-3)
    mag.close()
    mag = Magnet()
    mag.upload_workload(test_wl)
    base, nli_base = warmstart.curve(mag, test_wl.m0, fields, prm)
    warm, nli_warm = warmstart.curve(mag, test_wl.m0, fields, prm, mlp=net, scales=(s_m, s_p),
                                     max_change=0.0)          # reversible segment: no cap needed
    assert all(s["status"] == "ok" for s in base + warm)
    Mb = np.array([s["M"] for s in base])
    Mw = np.array([s["M"] for s in warm])
    np.testing.assert_allclose(Mw, Mb, atol=1e-4)
    print(f"NCG iterations without / with the warm start: {nli_base} / {nli_warm}")
    assert nli_warm < nli_base


def test_library_training_statistics_match_their_definitions():
    """The warm start's data arithmetic runs in the library: the input
    standardisation (mean and unbiased standard deviation per feature; a
    constant feature is only centred), the target scales (standard
    deviation of the m columns together and of the potential column) with
    the scaled targets, and a field step's targets ((after - before) / |dh|
    and the largest nodal change), against numpy in FP64."""
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=3)
    rng = np.random.default_rng(12)
    n = 50000
    Xh = rng.normal(size=(n, 16)) * rng.uniform(0.1, 5.0, 16) + rng.uniform(-3, 3, 16)
    Xh[:, 4] = 0.75                                   # constant feature
    Xh[:, 5] = 0.999 + 1e-3 * rng.normal(size=n)      # small spread on a large mean
    Xh = Xh.astype(np.float32)
    X = torch.tensor(Xh, device="cuda")
    net.fit_input_norm(X)
    mean, inv_sd = net.input_norm()
    x64 = Xh.astype(np.float64)
    mu, sd = x64.mean(0), x64.std(0, ddof=1)
    sd = np.where(sd > 1e-6 * (np.abs(mu) + 1.0), sd, 1.0)
    np.testing.assert_allclose(mean, mu, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(inv_sd, 1.0 / sd, rtol=1e-6)
    assert inv_sd[4] == 1.0

    Th = (rng.normal(size=(n, 4)) * np.array([0.01, 0.02, 0.03, 5.0])).astype(np.float32)
    T = torch.tensor(Th, device="cuda")
    Tn, s_m, s_p = net.fit_target_scales(T)
    t64 = Th.astype(np.float64)
    assert s_m == pytest.approx(t64[:, :3].reshape(-1).std(ddof=1), rel=1e-9)
    assert s_p == pytest.approx(t64[:, 3].std(ddof=1), rel=1e-9)
    ref = np.concatenate([Th[:, :3] / np.float32(s_m), Th[:, 3:] / np.float32(s_p)], axis=1)
    np.testing.assert_allclose(Tn.cpu().numpy(), ref, rtol=1e-6)

    X1h = Xh.copy()
    X1h[:, 0:3] += (1e-3 * rng.normal(size=(n, 3))).astype(np.float32)
    X1h[:, 15] += (0.1 * rng.normal(size=n)).astype(np.float32)
    X1h[777, 0:3] += np.float32(0.3)                 # one node turns further
    X0 = X.clone()
    X0[:, 12:15] = torch.tensor([0.02, -0.01, -0.05], device="cuda")   # field increment
    X1 = torch.tensor(X1h, device="cuda")
    T2, dh, change = net.step_targets(X0.contiguous(), X1.contiguous())
    dh_ref = np.linalg.norm(np.array([0.02, -0.01, -0.05], dtype=np.float32).astype(np.float64))
    assert dh == pytest.approx(dh_ref, rel=1e-6)
    d = X1h.astype(np.float64) - Xh.astype(np.float64)
    np.testing.assert_allclose(T2.cpu().numpy(), np.concatenate([d[:, :3], d[:, 15:16]], 1) / dh_ref,
                               rtol=1e-4, atol=1e-6)
    assert change == pytest.approx(np.linalg.norm(d[:, :3], axis=1).max(), rel=1e-5)
    X0[:, 12:15] = 0.0
    T3, dh0, _ = net.step_targets(X0.contiguous(), X1.contiguous())
    assert T3 is None and dh0 == 0.0


def _deviation_stats(Y, Yr):
    d = np.abs(Y - Yr) / np.abs(Yr).max()
    return float(d.max()), float(np.quantile(d, 0.5)), float(np.quantile(d, 0.9))


@pytest.mark.parametrize("n", [128, 301, 20000])
def test_tcgen05_forward_matches_reference_and_mma_sync(n):
    """The tcgen05 forward pass (default) against the oracle's network and
    against the warp-level mma.sync path, on full tiles, a ragged tail and
    many tiles.  All three round at the same points (BF16 inputs, weights,
    hidden activations); they differ in FP32 (GPU) vs FP64 (oracle)
    accumulation order, which moves an output by ~1e-6 of the largest and,
    where a hidden activation lies within that of a BF16 rounding boundary,
    flips it by one BF16 unit (2^-8 relative) -- measured: median 5e-9 and
    largest 9e-4 of the largest output over 20,000 rows; the bound on the
    largest is 2e-3.  The two GPU paths accumulate the same products in the
    same order (measured bitwise equal)."""
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=4)
    p = net.get_params()
    rng = np.random.default_rng(9)
    for off in (16 * 128, 16 * 128 + 128 + 128 * 128, 16 * 128 + 2 * (128 + 128 * 128)):
        p[off:off + 128] = rng.normal(size=128) * 0.1                  # nonzero biases
    net.set_params(p)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Y_tc = net.forward(Xd).cpu().numpy()
    net.set_tensor_path(1)
    Y_ms = net.forward(Xd).cpu().numpy()
    net.set_tensor_path(0)
    Yr, _ = omlp.forward(_params_list(p), X.astype(np.float64), round_bf16=True)
    for name, Y in (("tcgen05", Y_tc), ("mma.sync", Y_ms)):
        mx, med, q90 = _deviation_stats(Y, Yr)
        print(f"{name} vs oracle, n={n}: max {mx:.2e} median {med:.2e} q90 {q90:.2e} (of the largest output)")
        assert mx <= 2e-3 and med <= 1e-5, (name, mx, med)        # measured: max 9e-4, median 5e-9
    mx, med, q90 = _deviation_stats(Y_tc, Y_ms)
    print(f"tcgen05 vs mma.sync, n={n}: max {mx:.2e} median {med:.2e} q90 {q90:.2e}")
    assert mx <= 1e-6                                             # measured: bitwise equal
    assert np.isfinite(Y_tc).all()


@pytest.mark.parametrize("n", [517, 4096])
def test_tcgen05_weight_gradient_matches_mma_sync_and_reference(n):
    """The weight gradients on tcgen05 (one M = 128, K = 128-row MMA product
    per chunk of rows, default) against the mma.sync path on the same
    activations (the same FP32 sums of BF16 products) and against the
    oracle's network gradients."""
    import torch
    from paper_1801_03690_gb300 import MLP
    net = MLP(seed=6)
    p = net.get_params()
    rng = np.random.default_rng(8)
    X = torch.tensor(rng.normal(size=(n, 16)).astype(np.float32), device="cuda")
    T = torch.tensor(rng.normal(size=(n, 4)).astype(np.float32), device="cuda")
    g_tc, loss_tc = net.gradient(X, T)
    net.set_tensor_path(1)
    g_ms, loss_ms = net.gradient(X, T)
    net.set_tensor_path(0)
    assert loss_tc == loss_ms
    scale = np.abs(g_ms).max()
    err = np.abs(g_tc - g_ms).max() / scale
    print(f"tcgen05 vs mma.sync weight gradients, n={n}: max deviation {err:.2e} of the largest")
    assert err <= 1e-5
    lr, gr = omlp.loss_and_grads(_params_list(p), X.cpu().numpy().astype(np.float64),
                                 T.cpu().numpy().astype(np.float64), round_bf16=True)
    for (gw, gb), (rw, rb) in zip(_params_list(g_tc), gr):
        np.testing.assert_allclose(gw, rw, rtol=0, atol=3e-2 * np.abs(rw).max())
