"""The learned sensor predictor on real solver traces: training on the GPU lowers the loss, the
network beats the constant predictor on a held-out Reynolds number, the judge and fallback
bookkeeping are consistent, and -- with the sensor now as a fourth input, in the residual form --
the predicted flags beat reusing the current flags (persistence) on held-out 1024^2 cavities at a
2000-step horizon.  (Parity of the network's arithmetic with the oracle is in
test_gpu_predictor.py.)"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1507_06767_gb300 as pkg

    return pkg


def test_predictor_learns_from_solver_traces(L):
    import torch

    from paper_1507_06767_gb300 import learned as LN

    n, b, hz, u = 256, 16, 100, 0.1
    train = [LN.cavity_trace(n, re, u, b, 1000, 40, hz) for re in (300.0, 1500.0, 4000.0)]
    feats_e, kmax_e, tau_e = LN.cavity_trace(n, 900.0, u, b, 1000, 40, hz)
    assert torch.isfinite(kmax_e).all() and (kmax_e > 0).all()
    Xs, Ts = zip(*[LN.pairs(f, k) for f, k, _ in train])
    X, T = torch.cat(Xs), torch.cat(Ts)
    assert X.shape == (120, 3, 16, 16) and T.shape == (120, 1, 16, 16)
    net = L.Net(3, 16)
    shift, scale = LN.normalisation(u)
    net.set_normalisation(shift, scale)
    g = np.random.default_rng(5)
    theta = []
    for cin, cout in ((3, 16), (16, 16), (16, 1)):
        lim = np.sqrt(6.0 / (cin * 9))
        theta += [g.uniform(-lim, lim, cout * cin * 9), np.zeros(cout)]
    net.set_params(np.concatenate(theta))
    losses = LN.train(net, X, T, epochs=60, batch=8, lr=3e-3, seed=3)
    assert losses[-1] < 0.5 * losses[0]
    Xe, Te = LN.pairs(feats_e, kmax_e)
    y = net.forward(Xe).cpu().numpy()
    te = Te.cpu().numpy()
    mse = float(np.mean((y - te) ** 2))
    assert mse < np.var(te), (mse, np.var(te))
    j = LN.judge(net, feats_e, kmax_e, LN.threshold(tau_e, u, n), fallback_below=0.9)
    assert j["regrids"] == 40
    assert 0.0 <= j["fallback_fraction"] <= 1.0
    for k in ("agreement_predicted", "agreement_persistence", "agreement_used"):
        assert 0.0 <= j[k] <= 1.0
    print(j, losses[0], losses[-1], mse, np.var(te))
    net.close()


def test_judge_select_agreement_and_gather_kernels(L):
    """The regrid judge, the flag agreement and the minibatch gather on the device against their
    plain definitions: agreement = fraction of equal flags; the flags used are the new prediction
    when the previous prediction agreed with the exact flags on at least the set fraction (or
    there is no previous prediction), else the exact flags; gathered row k = source row idx[k],
    with an index outside the source flagged and not read."""
    import torch

    rng = np.random.default_rng(12)
    n = 4096
    a = torch.from_numpy(rng.integers(-1, 2, n).astype(np.int8)).cuda()
    b = a.clone()
    flip = rng.choice(n, 300, replace=False)
    b[torch.from_numpy(flip).cuda()] = torch.from_numpy(
        ((a.cpu().numpy()[flip] + 2) % 3 - 1).astype(np.int8)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lbm_flags_agreement(a, b, n, out)
    assert out.item() == pytest.approx((n - 300) / n, abs=0)
    L.lbm_flags_agreement(a, b, 0, out)
    assert out.item() == 1.0
    nxt = torch.from_numpy(rng.integers(-1, 2, n).astype(np.int8)).cuda()
    used = torch.empty(n, dtype=torch.int8, device="cuda")
    agree = torch.zeros(1, dtype=torch.float64, device="cuda")
    fell = torch.zeros(1, dtype=torch.int32, device="cuda")
    for thr, expect_exact in ((0.9, False), (0.95, True)):  # agreement 0.9268
        L.lbm_flags_judge_select(a, b, nxt, n, thr, used, agree, fell)
        assert agree.item() == pytest.approx((n - 300) / n, abs=0)
        assert fell.item() == int(expect_exact)
        assert torch.equal(used, b if expect_exact else nxt)
    L.lbm_flags_judge_select(None, b, nxt, n, 0.99, used, agree, fell)  # first regrid
    assert np.isnan(agree.item()) and fell.item() == 0 and torch.equal(used, nxt)
    with pytest.raises(L.LbmError):
        L.lbm_flags_judge_select(a, b, nxt, n, 1.5, used)
    src = torch.from_numpy(rng.normal(size=(37, 3, 5, 7)).astype(np.float32)).cuda()
    idx = torch.from_numpy(np.array([5, 0, 36, 5, 12], np.int32)).cuda()
    dst = torch.full((5, 3, 5, 7), -1.0, device="cuda")
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.lbm_gather_rows(src, 37, 3 * 5 * 7 * 4, idx, 5, dst, bad)
    assert torch.equal(dst, src[idx.long()]) and bad.item() == 0
    idx[2] = 37
    L.lbm_gather_rows(src, 37, 3 * 5 * 7 * 4, idx, 5, dst, bad)
    assert bad.item() == 1


def test_residual_log_and_maxima_match_their_definitions(L):
    import torch

    g = np.random.default_rng(21)
    n = 5000
    now = 10.0 ** g.uniform(-14, -1, n)
    nxt = now * 10.0 ** g.normal(0.0, 0.3, n)
    now[7], nxt[11] = np.nan, np.nan
    now[13] = 0.0  # below the floor
    floor = float(np.float32(1e-12))  # the calls take the floor as a float
    a = torch.from_numpy(nxt).cuda()
    b = torch.from_numpy(now).cuda()
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    L.lbm_net_log_residual(a, b, n, floor, t)
    want = (np.log10(np.maximum(nxt, floor)) - np.log10(np.maximum(now, floor))).astype(np.float32)
    got = t.cpu().numpy()
    ok = np.isfinite(want)
    assert np.isnan(got[~ok]).all() and (~ok).sum() == 2
    assert np.allclose(got[ok], want[ok], rtol=0, atol=1e-5)
    y = torch.from_numpy(g.normal(0.0, 0.3, n).astype(np.float32)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    L.lbm_net_to_maxima_residual(y, b, n, floor, out)
    want = np.maximum(now, floor) * 10.0 ** y.cpu().numpy().astype(np.float64)
    got = out.cpu().numpy()
    assert np.isnan(got[7]) and np.isnan(want[7])
    m = np.isfinite(want)
    assert np.allclose(got[m], want[m], rtol=1e-12, atol=0)
    with pytest.raises(L.LbmError):
        L.lbm_net_log_residual(a, b, n, 0.0, t)


def test_sensor_input_predictor_beats_persistence_at_2000_steps(L):
    """D2Q9 1024^2 cavities with Re from U[100, 5000] (seeded): 8 train, 4 held out; snapshots
    2000 steps apart after 2000 steps, 10 regrids each.  The residual predictor (block means and
    the log sensor maximum now in, the change of log10 K out) trained for 40 epochs agrees with the
    exact flags of the next regrid on more blocks than the current exact flags do: on average, in
    each held-out cavity and in the first two thirds of the runs (the flow still developing); in the
    last third the two are level (measured 0.9740 against 0.9745)."""
    import math

    import torch

    from paper_1507_06767_gb300 import learned as LN

    n, b, hz, S, u = 1024, 16, 2000, 10, 0.1
    g = np.random.default_rng(np.random.SeedSequence([1024, 5000, 7]))
    res = g.uniform(100.0, 5000.0, size=12)
    traces = [LN.cavity_trace(n, float(re), u, b, hz, S, hz, with_sensor=True) for re in res]
    Xs, Ts = zip(*[LN.pairs(f, k) for f, k, _ in traces[:8]])
    X, T = torch.cat(Xs), torch.cat(Ts)
    assert X.shape == (8 * S, 4, 64, 64)
    net = L.Net(4, 16)
    net.set_normalisation(*LN.normalisation(u, with_sensor=True))
    gg = np.random.default_rng(11)
    theta = []
    for cin, cout in ((4, 16), (16, 16), (16, 1)):
        lim = math.sqrt(6.0 / (cin * 9))
        theta += [gg.uniform(-lim, lim, cout * cin * 9), np.zeros(cout)]
    net.set_params(np.concatenate(theta))
    losses = LN.train(net, X, T, 40, 16, 2e-3, seed=7)
    assert losses[-1] < 0.5 * losses[0]
    per = []
    for (f, k, tau) in traces[8:]:
        j = LN.judge(net, f, k, LN.threshold(tau, u, n), 0.9)
        per.append(j["per_regrid"])
    r = np.array(per)  # [held-out cavity, (predicted, persistence, used), regrid]
    pred, pers = r[:, 0], r[:, 1]
    print("predicted", pred.mean(axis=1), "persistence", pers.mean(axis=1))
    assert pred.mean() > pers.mean() + 0.002, (pred.mean(), pers.mean())
    assert (pred.mean(axis=1) > pers.mean(axis=1)).all()
    early, mid, late = np.array_split(np.arange(S), 3)
    for part in (early, mid):
        assert pred[:, part].mean() > pers[:, part].mean() + 0.002, part
    assert pred[:, late].mean() > pers[:, late].mean() - 0.002
    net.close()
