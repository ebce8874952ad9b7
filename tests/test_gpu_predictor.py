"""GPU parity of the sensor predictor (lbm_block_features, lbm_net_*) with the numpy oracle
(oracle/predictor.py) and with the plain definition of the block means.

Tolerances: the network stores weights and activations in BF16 (8 significant bits, relative
rounding 2^-9) and accumulates in FP32.  The parity proper is element-wise and layer by layer
(test_each_layer_matches_oracle_elementwise): the oracle evaluates each layer in FP64 on the exact
BF16 operands the kernels read, which leaves only FP32 accumulation, bounded per element.  The
chained network is also compared with the oracle evaluated in FP64 throughout on the unrounded
parameters (test_forward_and_gradients_match_oracle): there the BF16 roundings of three layers
accumulate and some rounding decisions fall differently, so that end-to-end check is norm-wise,
at 1e-2 for the outputs and 3e-2 for the gradients.  Adam is FP32 against FP64 on the same
gradients: 1e-5.
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


U32 = 2.0 ** -24  # unit roundoff of FP32


def bf16_bits_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def check_rounded(gpu, z, tol, what):
    """gpu = BF16 rounding of ReLU of the FP32 value of z (a sum computed within tol of the exact
    pre-activation z): equal to bf16_round(max(z, 0)) wherever that cannot change inside
    [z - tol, z + tol]; elsewhere (ReLU and rounding are monotone) between the roundings of the two
    ends.  The ambiguous elements must be a small share (the bound is the worst case of a sum of
    up to 145 terms, some ten times the typical rounding error, so a few per cent are ambiguous)."""
    relu = lambda v: np.maximum(v, 0.0)  # noqa: E731
    ref = P.bf16_round(relu(z))
    lo, hi = P.bf16_round(relu(z - tol)), P.bf16_round(relu(z + tol))
    amb = lo != hi
    assert np.array_equal(gpu[~amb], ref[~amb]), (what, int((gpu[~amb] != ref[~amb]).sum()))
    assert np.all((gpu[amb] >= lo[amb]) & (gpu[amb] <= hi[amb])), what
    assert amb.mean() < 0.1, (what, amb.mean())


def check_sum(gpu, ref, mag, nterms, what):
    """gpu = an FP32 sum of nterms products whose exact value is ref and whose absolute terms add
    up to mag: |gpu - ref| <= (nterms + 1) u mag element by element."""
    err = np.abs(np.asarray(gpu, np.float64) - ref)
    bound = (nterms + 1) * U32 * mag + 1e-30
    assert np.all(err <= bound), (what, float((err / bound).max()))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_each_layer_matches_oracle_elementwise(L, case):
    """Element-wise parity of every layer of the forward and backward pass.  Each layer is
    evaluated by the oracle in FP64 on the exact BF16 operands the kernels read (the BF16 rounding
    of the parameters, and the kernels' own BF16 activations of the previous layer), so what is
    left is FP32 accumulation, bounded per element by (terms + 1) u sum|terms|; the BF16 rounding of
    an activation must equal the rounding of the oracle's value wherever the accumulation bound
    cannot move it across a rounding midpoint.  Weight gradients are reduced by 256 threads, each
    summing a strided share of the positions before a fixed tree over the threads, which bounds
    their terms per element by ceil(positions / 256) + 8."""
    cin, hid, B, H, W = CASES[case]
    p32 = P.flatten(params(960 + case, cin, hid)).astype(np.float32)
    g = seeded.rng(970 + case)
    shift = g.uniform(-0.5, 0.5, cin).astype(np.float32)
    scale = g.uniform(0.5, 2.0, cin).astype(np.float32)
    Xraw = (g.normal(size=(B, cin, H, W)) / scale[None, :, None, None]
            + shift[None, :, None, None]).astype(np.float32)
    T = g.normal(size=(B, 1, H, W)).astype(np.float32)
    net = L.Net(cin, hid)
    net.set_normalisation(shift, scale)
    net.set_params(p32)
    net.backward(dev(Xraw), dev(T))
    buf = lambda which, shape: net.buffer(which, shape)  # noqa: E731
    # parameters: BF16 rounding of the FP32 master copy, exactly
    pb = bf16_bits_to_f64(buf(L.LBM_NET_BUF_PARAMS_BF16, p32.size))
    assert np.array_equal(pb, P.bf16_round(p32.astype(np.float64)))
    p = P.unflatten(pb, cin, hid)
    pa = {k: np.abs(v) for k, v in p.items()}
    # normalised input: (x - shift) * scale in FP32 (the kernels' precision decides the rounding)
    x0 = bf16_bits_to_f64(buf(L.LBM_NET_BUF_X0, (B, cin, H, W)))
    xn = ((Xraw - shift[None, :, None, None]) * scale[None, :, None, None]).astype(np.float32)
    assert np.array_equal(x0, P.bf16_round(xn.astype(np.float64)))
    # layer 1 and 2: pre-activation in FP64 on the kernels' operands, ReLU, BF16 rounding
    a_in = x0
    acts = []
    for k, (Wk, bk, nt) in enumerate((("W1", "b1", 9 * cin), ("W2", "b2", 9 * hid))):
        z = P.conv3(a_in, p[Wk], p[bk])
        mag = P.conv3(np.abs(a_in), pa[Wk], pa[bk])
        a_gpu = bf16_bits_to_f64(buf((L.LBM_NET_BUF_A1, L.LBM_NET_BUF_A2)[k], (B, hid, H, W)))
        check_rounded(a_gpu, z, (nt + 1) * U32 * mag, f"A{k + 1}")
        acts.append(a_gpu)
        a_in = a_gpu
    A1, A2 = acts
    # output layer (FP32 output, no rounding to BF16)
    y = buf(L.LBM_NET_BUF_Y, (B, 1, H, W))
    check_sum(y, P.conv3(A2, p["W3"], p["b3"]), P.conv3(A2, pa["W3"], pa["b3"]), 9 * hid + 4, "Y")
    # a planted mistake in the oracle (the kernel taps mirrored) is caught by the same bound
    ybad = P.conv3(A2, p["W3"][:, :, ::-1, ::-1], p["b3"])
    err = np.abs(y - ybad) / ((9 * hid + 5) * U32 * P.conv3(A2, pa["W3"], pa["b3"]))
    assert (err > 1).mean() > 0.5
    # loss gradient dY = (2 / n)(Y - T): two FP32 roundings
    n = B * H * W
    dy = buf(L.LBM_NET_BUF_DY, (B, 1, H, W))
    dref = (2.0 / n) * (y.astype(np.float64) - T)
    assert np.all(np.abs(dy - dref) <= 3 * U32 * np.abs(dref) + 1e-45)
    dy = dy.astype(np.float64)
    grads = P.unflatten(net.grads().astype(np.float64), cin, hid)
    red = -(-n // 256) + 8  # terms of the weight-gradient reductions, per element
    # backward through layer 3, 2, 1 on the kernels' own upstream gradients
    dz2 = buf(L.LBM_NET_BUF_DZ2, (B, hid, H, W)).astype(np.float64)
    dz1 = buf(L.LBM_NET_BUF_DZ1, (B, hid, H, W)).astype(np.float64)
    for Wk, bk, d_out, a_low in (("W3", "b3", dy, A2), ("W2", "b2", dz2, A1), ("W1", "b1", dz1, x0)):
        check_sum(grads[Wk], P.conv3_weight_grad(d_out, a_low),
                  P.conv3_weight_grad(np.abs(d_out), np.abs(a_low)), red, "g" + Wk)
        check_sum(grads[bk], d_out.sum(axis=(0, 2, 3)), np.abs(d_out).sum(axis=(0, 2, 3)), red,
                  "g" + bk)
    for Wk, d_out, d_in, a_low in (("W3", dy, dz2, A2), ("W2", dz2, dz1, A1)):
        ref = P.conv3_input_grad(d_out, p[Wk]) * (a_low > 0)
        mag = P.conv3_input_grad(np.abs(d_out), pa[Wk])
        check_sum(d_in, ref, mag, 9 * p[Wk].shape[0], "d" + Wk)
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
