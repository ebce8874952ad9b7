"""Pins of the predictor oracle (oracle/predictor.py): the convolution against scipy's
correlation, every gradient against central finite differences, and Adam against its closed form
on constant gradients."""
import numpy as np
import pytest

from oracle import predictor as P
from tests import seeded

signal = pytest.importorskip("scipy.signal")


def params(seed, cin, hidden, bias=0.1):
    shp = P.shapes(cin, hidden)
    lims = [np.sqrt(6.0 / (shp[k][1] * 9)) if k.startswith("W") else bias for k in P.PARAM_ORDER]
    arrs = seeded.uniform_arrays(seed, [shp[k] for k in P.PARAM_ORDER], lims)
    return dict(zip(P.PARAM_ORDER, arrs))


def test_conv_is_zero_padded_correlation():
    g = seeded.rng(11)
    A = g.normal(size=(2, 3, 7, 9))
    W = g.normal(size=(4, 3, 3, 3))
    b = g.normal(size=4)
    out = P.conv3(A, W, b)
    for bi in range(2):
        for o in range(4):
            ref = sum(signal.correlate2d(A[bi, c], W[o, c], mode="same", boundary="fill")
                      for c in range(3)) + b[o]
            assert np.allclose(out[bi, o], ref, rtol=1e-13, atol=1e-13)


def test_conv_adjoints():
    # <conv(A, W), D> = <A, input_grad(D, W)> = <W, weight_grad(D, A)>
    g = seeded.rng(12)
    A = g.normal(size=(3, 2, 6, 5))
    W = g.normal(size=(4, 2, 3, 3))
    D = g.normal(size=(3, 4, 6, 5))
    lhs = np.sum(P.conv3(A, W) * D)
    assert np.isclose(lhs, np.sum(A * P.conv3_input_grad(D, W)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * P.conv3_weight_grad(D, A)), rtol=1e-12)


def test_gradients_match_finite_differences():
    cin, hidden = 3, 4
    p = params(13, cin, hidden, bias=0.3)
    g = seeded.rng(14)
    X = g.normal(size=(2, cin, 5, 6))
    T = g.normal(size=(2, 1, 5, 6))
    _, grads = P.gradients(p, X, T)
    theta = P.flatten(p)
    gflat = P.flatten(grads)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Yp, _ = P.forward(P.unflatten(tp, cin, hidden), X)
        Ym, _ = P.forward(P.unflatten(tm, cin, hidden), X)
        num[k] = (P.loss(Yp, T) - P.loss(Ym, T)) / (2 * h)
    # ReLU kinks are measure-zero for these draws; central differences are O(h^2)
    assert np.abs(num - gflat).max() <= 1e-7 * max(1.0, np.abs(gflat).max())
    assert np.abs(gflat).min() >= 0.0 and np.count_nonzero(gflat) > 0.9 * gflat.size


def test_adam_closed_form_on_constant_gradients():
    g = seeded.rng(15).normal(size=50)
    theta0 = seeded.rng(16).normal(size=50)
    opt = P.Adam(50, lr=0.01, eps=1e-8)
    th = theta0.copy()
    for t in range(1, 6):
        th = opt.step(th, g)
        # with a constant gradient both bias-corrected moments are exact: m^ = g, v^ = g^2
        assert np.allclose(th, theta0 - t * 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_training_fits_a_teacher_network():
    cin, hidden = 3, 8
    teacher = params(17, cin, hidden, bias=0.2)
    student = params(18, cin, hidden, bias=0.0)
    g = seeded.rng(19)
    X = g.normal(size=(8, cin, 12, 12))
    T, _ = P.forward(teacher, X)
    theta = P.flatten(student)
    opt = P.Adam(theta.size, lr=1e-2)
    first = None
    for _ in range(300):
        L, grads = P.gradients(P.unflatten(theta, cin, hidden), X, T)
        first = L if first is None else first
        theta = opt.step(theta, P.flatten(grads))
    L, _ = P.gradients(P.unflatten(theta, cin, hidden), X, T)
    assert L < 0.05 * first and L < 0.1 * np.var(T)


def test_bf16_round_hand_cases_and_library_conversion():
    # 8 significant bits: spacing 2^-7 on [1, 2); halves go to the even significand
    r = P.bf16_round
    assert r(1.0 + 2.0 ** -8) == 1.0                      # tie -> even (1.0000000)
    assert r(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even (1.0000010)
    assert r(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7  # above the tie
    assert r(-3.0 - 2.0 ** -7) == -3.0                    # tie at spacing 2^-6, negative
    assert r(0.0) == 0.0 and r(2.0 ** -126) == 2.0 ** -126
    assert r(255.5) == 256.0 and r(254.5) == 254.0        # spacing 1 on [128, 256)
    # against the library's round-to-nearest-even FP32 -> BF16 conversion on FP32 values
    torch = pytest.importorskip("torch")
    g = seeded.rng(77)
    x = (g.normal(size=20000) * 10.0 ** g.uniform(-6, 4, size=20000)).astype(np.float32)
    # add exact ties: FP32 values whose low 16 bits are 0x8000
    ties = (g.integers(0x3f000000, 0x41000000, size=2000, dtype=np.int64) & ~0xffff) | 0x8000
    x = np.concatenate([x, ties.astype(np.uint32).view(np.float32)])
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r(x.astype(np.float64)), lib)
