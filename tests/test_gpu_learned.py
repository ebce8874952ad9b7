"""The learned sensor predictor on real solver traces (small cavities): training on the GPU lowers
the loss, the network beats the constant predictor on a held-out Reynolds number, and the judge
and fallback bookkeeping are consistent.  (Parity of the network's arithmetic with the oracle is
in test_gpu_predictor.py.)"""
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
