"""Learned predictor of the block sensor maxima: a 3-layer convolution network, its gradients and
its Adam update, in plain numpy float64.

TEST INFRASTRUCTURE ONLY: imported by the test suite alone; the product library never imports it
and shares no code with it.

The paper refines where the Knudsen sensor K (Sec. 3.2, Eq. sensor) is large and, in its dynamic
runs (Sec. 5.2), re-evaluates it every level-0 step.  The predictor reads block-averaged density and
velocity at time t and estimates log10 of each block's sensor maximum some steps later, so that a
regrid can refine ahead of the flow; the exact sensor stays the judge of its flags.  The network
is not in the paper; its definition here:

* input X[b, c, y, x], c = 0..Cin-1: features of block (y, x), normalised per channel as
  (x - shift[c]) * scale[c];
* Z1 = conv(X, W1) + b1, A1 = max(Z1, 0); Z2 = conv(A1, W2) + b2, A2 = max(Z2, 0);
  Y = conv(A2, W3) + b3 (one output channel), every conv 3 x 3 with zero padding ("same"):
  conv(A, W)[b, o, y, x] = sum_{c, i, j} W[o, c, i, j] A[b, c, y + i - 1, x + j - 1];
* loss L = mean over b, y, x of (Y - T)^2;
* Adam (Kingma and Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are passed around as a dict of arrays W1 [H, Cin, 3, 3], b1 [H], W2 [H, H, 3, 3],
b2 [H], W3 [1, H, 3, 3], b3 [1] (H hidden channels); ``PARAM_ORDER`` is the order of the flat
parameter vector.
"""
from __future__ import annotations

import numpy as np

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(cin: int, hidden: int):
    return {"W1": (hidden, cin, 3, 3), "b1": (hidden,), "W2": (hidden, hidden, 3, 3),
            "b2": (hidden,), "W3": (1, hidden, 3, 3), "b3": (1,)}


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(v, cin: int, hidden: int):
    out, o = {}, 0
    for k in PARAM_ORDER:
        shp = shapes(cin, hidden)[k]
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    assert o == len(v)
    return out


def conv3(A, W, b=None):
    """conv(A, W)[b, o, y, x] = sum_{c,i,j} W[o,c,i,j] A[b, c, y+i-1, x+j-1] (+ bias[o])."""
    B, C, H, Wd = A.shape
    Ap = np.pad(A, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((B, W.shape[0], H, Wd))
    for i in range(3):
        for j in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, i, j], Ap[:, :, i:i + H, j:j + Wd])
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv3_input_grad(dO, W):
    """d/dA of sum(dO * conv(A, W)): dA[b,c,y,x] = sum_{o,i,j} W[o,c,i,j] dO[b,o,y-i+1,x-j+1]."""
    B, O, H, Wd = dO.shape
    dOp = np.pad(dO, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((B, W.shape[1], H, Wd))
    for i in range(3):
        for j in range(3):
            # dO[y - i + 1] = dOp[y - i + 2]
            out += np.einsum("oc,bohw->bchw", W[:, :, i, j],
                             dOp[:, :, 2 - i:2 - i + H, 2 - j:2 - j + Wd])
    return out


def conv3_weight_grad(dO, A):
    """d/dW of sum(dO * conv(A, W)): dW[o,c,i,j] = sum_{b,y,x} dO[b,o,y,x] A[b,c,y+i-1,x+j-1]."""
    B, C, H, Wd = A.shape
    Ap = np.pad(A, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((dO.shape[1], C, 3, 3))
    for i in range(3):
        for j in range(3):
            out[:, :, i, j] = np.einsum("bohw,bchw->oc", dO, Ap[:, :, i:i + H, j:j + Wd])
    return out


def bf16_round(x):
    """Round to the nearest BF16 value (8 significant bits, the exponent range of FP32), ties to
    the even significand: the storage rounding of the network's weights and activations.  Written
    for finite values in the normal range, which is all the network produces (zeros stay zero)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                 # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)   # np.rint rounds halves to even


def normalise(X, shift, scale):
    X = np.asarray(X, dtype=np.float64)
    return (X - np.asarray(shift)[None, :, None, None]) * np.asarray(scale)[None, :, None, None]


def forward(p, X):
    """Returns (Y, cache) for normalised inputs X [B, Cin, H, W]."""
    Z1 = conv3(X, p["W1"], p["b1"])
    A1 = np.maximum(Z1, 0.0)
    Z2 = conv3(A1, p["W2"], p["b2"])
    A2 = np.maximum(Z2, 0.0)
    Y = conv3(A2, p["W3"], p["b3"])
    return Y, (X, Z1, A1, Z2, A2)


def loss(Y, T) -> float:
    return float(np.mean((Y - T) ** 2))


def gradients(p, X, T):
    """(loss, dict of dL/dparam) for the mean-square loss against targets T [B, 1, H, W]."""
    Y, (X, Z1, A1, Z2, A2) = forward(p, X)
    n = Y.size
    dY = 2.0 * (Y - T) / n
    g = {"W3": conv3_weight_grad(dY, A2), "b3": dY.sum(axis=(0, 2, 3))}
    dZ2 = conv3_input_grad(dY, p["W3"]) * (Z2 > 0)
    g["W2"] = conv3_weight_grad(dZ2, A1)
    g["b2"] = dZ2.sum(axis=(0, 2, 3))
    dZ1 = conv3_input_grad(dZ2, p["W2"]) * (Z1 > 0)
    g["W1"] = conv3_weight_grad(dZ1, X)
    g["b1"] = dZ1.sum(axis=(0, 2, 3))
    return loss(Y, T), g


class Adam:
    def __init__(self, nparams: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(nparams)
        self.v = np.zeros(nparams)
        self.t = 0
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * g
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * g * g
        mh = self.m / (1.0 - self.beta1 ** self.t)
        vh = self.v / (1.0 - self.beta2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
