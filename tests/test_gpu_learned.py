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
