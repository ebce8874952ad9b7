"""GPU parity of the sensor predictor (lbm_block_features, lbm_net_*) with the numpy oracle
(oracle/predictor.py) and with the plain definition of the block means.

Tolerances: the network stores weights and activations in BF16 (8 significant bits, relative
rounding 2^-9) and accumulates in FP32, while the oracle is FP64 throughout.  Each layer adds a
few such roundings to every value, partly averaging out over its 9 * C terms, so the outputs are
compared norm-wise at 1e-2 relative and the gradients (three layers of products) at 3e-2; a wrong
index or a dropped term gives O(1) errors.  Adam is FP32 against FP64 on the same gradients: 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from oracle import predictor as P
from tests import seeded

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


def params(seed, cin, hidden, bias=0.1):
    shp = P.shapes(cin, hidden)
    lims = [np.sqrt(6.0 / (shp[k][1] * 9)) if k.startswith("W") else bias for k in P.PARAM_ORDER]
    arrs = seeded.uniform_arrays(seed, [shp[k] for k in P.PARAM_ORDER], lims)
    return dict(zip(P.PARAM_ORDER, arrs))


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def block_means(f, c, b):
    """Plain definition: per block of edge b, the mean over its cells of rho and u = j / rho."""
    q, nz, ny, nx = f.shape
    rho = f.sum(0)
    u = np.einsum("qa,qzyx->azyx", c.astype(np.float64), f) / rho
    chans = [rho, u[0], u[1]] + ([u[2]] if nz > 1 else [])
    bz = b if nz > 1 else 1
    nbz, nby, nbx = -(-nz // bz), -(-ny // b), -(-nx // b)
    out = np.empty((len(chans), nbz, nby, nbx))
    for k, ch in enumerate(chans):
        for z in range(nbz):
            for y in range(nby):
                for x in range(nbx):
                    out[k, z, y, x] = ch[z * bz:(z + 1) * bz, y * b:(y + 1) * b,
                                         x * b:(x + 1) * b].mean()
    return out.reshape(len(chans), -1)


@pytest.mark.parametrize("q,shape,dtype,tol", [(9, (1, 80, 96), "F64", 1e-6),
                                               (19, (33, 36, 40), "F32", 2e-6)])
def test_block_features_match_definition(L, q, shape, dtype, tol):
    import torch

    nz, ny, nx = shape
    lat = L.Lattice(q, nx, ny, nz, 0.7, dtype=getattr(L, "LBM_" + dtype))
    c, w, _ = O.lattice(q)
    f = w[:, None, None, None] * (1.0 + seeded.relative_perturbation(61 + q, (q,) + shape, 0.05))
    lat.set_populations(f)
    b = 16
    nb = L.lbm_nblocks(lat.h, b)
    out = torch.empty((3 if q == 9 else 4) * nb, dtype=torch.float32, device="cuda")
    L.lbm_block_features(lat.h, b, out)
    torch.cuda.synchronize()
    ref = block_means(lat.populations(), c, b)
    got = out.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())
    lat.close()


CASES = [(3, 16, 4, 64, 64), (3, 16, 3, 37, 29), (4, 8, 2, 20, 24)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_and_gradients_match_oracle(L, case):
    cin, hid, B, H, W = CASES[case]
    p = params(900 + case, cin, hid)
    g = seeded.rng(910 + case)
    shift = g.uniform(-0.5, 0.5, cin)
    scale = g.uniform(0.5, 2.0, cin)
    Xraw = g.normal(size=(B, cin, H, W)) / scale[None, :, None, None] + shift[None, :, None, None]
    T = g.normal(size=(B, 1, H, W))
    net = L.Net(cin, hid)
    net.set_normalisation(shift, scale)
    net.set_params(P.flatten(p))
    X = P.normalise(Xraw, shift, scale)
    Yref, _ = P.forward(p, X)
    y = net.forward(dev(Xraw)).cpu().numpy()
    assert nrel(y, Yref) <= 1e-2
    loss_ref, gref = P.gradients(p, X, T)
    loss = net.backward(dev(Xraw), dev(T))
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    got = P.unflatten(net.grads(), cin, hid)
    for k in P.PARAM_ORDER:
        assert nrel(got[k], gref[k]) <= 3e-2, k
    # deterministic: a second backward gives the same bits
    g1 = net.grads()
    net.backward(dev(Xraw), dev(T))
    assert np.array_equal(g1, net.grads())
    net.close()


def test_adam_matches_oracle(L):
    cin, hid = 3, 16
    net = L.Net(cin, hid)
    theta = P.flatten(params(920, cin, hid))
    net.set_params(theta)
    opt = P.Adam(theta.size, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    th = theta.astype(np.float32).astype(np.float64)
    for k in range(5):
        grad = seeded.rng(921 + k).normal(size=theta.size) * 10.0 ** seeded.rng(930 + k).uniform(
            -4, 0, size=theta.size)
        net.set_grads(grad)
        net.adam(1e-3)
        th = opt.step(th, grad.astype(np.float32).astype(np.float64))
    got = net.params()
    assert np.abs(got - th).max() <= 1e-5 * max(1.0, np.abs(th).max())
    net.close()


def test_training_fits_a_teacher_on_the_gpu(L):
    cin, hid = 3, 16
    teacher = params(940, cin, hid, bias=0.2)
    g = seeded.rng(941)
    X = g.normal(size=(16, cin, 32, 32))
    T, _ = P.forward(teacher, X)
    net = L.Net(cin, hid)
    net.set_params(P.flatten(params(942, cin, hid, bias=0.0)))
    x, t = dev(X), dev(T)
    first = net.backward(x, t)
    for _ in range(400):
        net.train_step(x, t, 1e-2, sync=False)
    last = net.backward(x, t)
    assert last < 0.2 * first and last < 0.3 * np.var(T)
    net.close()


def test_log_targets_and_maxima_round_trip(L):
    import torch

    K = 10.0 ** seeded.rng(950).uniform(-6, 0, size=1000)
    K[:3] = [0.0, 1e-20, np.nan]
    kd = torch.from_numpy(K).cuda()
    t = torch.empty(1000, dtype=torch.float32, device="cuda")
    L.lbm_net_log_targets(kd, 1000, -3.0, 1e-12, t)
    tt = t.cpu().numpy()
    ref = np.log10(np.maximum(np.nan_to_num(K, nan=np.nan), 1e-12)) + 3.0
    assert np.abs(tt[3:] - ref[3:]).max() <= 1e-5
    assert tt[0] == pytest.approx(-9.0) and tt[1] == pytest.approx(-9.0) and np.isnan(tt[2])
    back = torch.empty(1000, dtype=torch.float64, device="cuda")
    L.lbm_net_to_maxima(t, 1000, -3.0, back)
    bb = back.cpu().numpy()
    assert np.abs(bb[3:] / K[3:] - 1).max() <= 1e-5


def test_net_argument_errors(L):
    with pytest.raises(L.LbmError):
        L.lbm_net_create(5, 16)
    net = L.Net(3, 16)
    import torch

    x = torch.zeros((1, 3, 4, 4), device="cuda")
    with pytest.raises(L.LbmError) as ei:
        L.lbm_net_forward(net.n, x, 0, 4, 4, x)
    assert ei.value.status == L.LBM_EINVAL
    with pytest.raises(L.LbmError) as ei:
        net.adam(1e-3, beta1=1.0)
    assert ei.value.status == L.LBM_EINVAL
    net.close()
