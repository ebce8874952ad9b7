"""Learned sensor predictor around the C ABI: solver traces, training, and the dynamic-refinement
loop that regrids from predicted block maxima with the exact sensor as fallback and judge.

Every step runs in the library's kernels (lbm_step, lbm_sensor_dev, lbm_block_features,
lbm_net_*, lbm_flags_from_maxima); this module only sequences the calls and keeps the traces in
PyTorch CUDA tensors.

The paper regrids its dynamic cavity from the Knudsen sensor at every level-0 step (Sec. 5.2).
Here the network reads the block-averaged (rho, u_x, u_y) at time t and predicts log10 of each
block's sensor maximum at t + horizon; a regrid can then refine where the flow is going.  The
exact sensor at t + horizon judges the predicted flags, and a regrid falls back to the exact flags
whenever the agreement of the last judged prediction fell below a set fraction.

Two forms: `with_sensor=False` reads the three block means only; `with_sensor=True` also reads the
block's sensor maximum now, log10(K) - LOG_OFFSET as a fourth channel, and predicts the change of
log10 K over the horizon (the residual form), so that "no change" -- reusing the current sensor --
is the network's zero output.
"""
from __future__ import annotations

import numpy as np

from . import lbm as L

# input normalisation: rho - 1 ~ 1e-3..1e-2 and |u| <= u_lid in lattice units
LOG_OFFSET = -3.0   # targets are log10(K) - LOG_OFFSET
FLOOR_K = 1e-12


def normalisation(u_lid: float, with_sensor: bool = False):
    shift = [1.0, 0.0, 0.0] + ([0.0] if with_sensor else [])
    scale = [100.0, 1.0 / u_lid, 1.0 / u_lid] + ([1.0] if with_sensor else [])
    return np.array(shift, np.float32), np.array(scale, np.float32)


def threshold(tau: float, u_lid: float, n: int) -> float:
    """Refinement threshold: four times the Couette-level sensor of the mean lid shear."""
    return 4.0 * (4.0 / 3.0) * tau * u_lid / n


def cavity_trace(n: int, re: float, u_lid: float, block: int, warm: int, snapshots: int,
                 horizon: int, dtype=None, with_sensor: bool = False):
    """D2Q9 cavity of n^2 cells at Reynolds number re from rest: after `warm` steps, snapshots
    spaced `horizon` steps apart.  Returns (features [S+1, C, nb, nb] float32, block maxima
    [S+1, nb*nb] float64, tau), all on the GPU; features[k] and maxima[k] belong to the same step
    (the sensor of the last step).  C = 3 (rho, u_x, u_y), or 4 with the log sensor maximum as the
    last channel (with_sensor)."""
    import torch

    tau = 3.0 * u_lid * n / re + 0.5
    lat = L.Lattice(L.LBM_D2Q9, n, n, 1, tau, dtype=L.LBM_F32 if dtype is None else dtype,
                    lid=(u_lid, 0.0))
    L.lbm_set_sensor_every(lat.h, 0)  # the sensor on the last step of every lbm_step call
    nb = L.lbm_nblocks(lat.h, block)
    side = -(-n // block)
    feats = torch.empty((snapshots + 1, 4 if with_sensor else 3, side, side), dtype=torch.float32,
                        device="cuda")
    kmax = torch.empty((snapshots + 1, nb), dtype=torch.float64, device="cuda")
    lat.step(warm)
    for k in range(snapshots + 1):
        if k:
            lat.step(horizon)
        L.lbm_sensor_dev(lat.h, block, kmax[k])
        L.lbm_block_features(lat.h, block, feats[k])  # channels 0..2
        if with_sensor:
            L.lbm_net_log_targets(kmax[k], nb, LOG_OFFSET, FLOOR_K, feats[k, 3])
    torch.cuda.synchronize()
    lat.close()
    return feats, kmax, tau


def pairs(feats, kmax):
    """(inputs at t, targets at t + horizon in log units) from a trace; with the sensor channel
    (4 input channels) the targets are the change of log10 K (residual form)."""
    import torch

    t = torch.empty((kmax.shape[0] - 1, 1) + tuple(feats.shape[2:]), dtype=torch.float32,
                    device="cuda")
    if feats.shape[1] == 4:
        L.lbm_net_log_residual(kmax[1:].contiguous(), kmax[:-1].contiguous(), t.numel(), FLOOR_K, t)
    else:
        L.lbm_net_log_targets(kmax[1:], t.numel(), LOG_OFFSET, FLOOR_K, t)
    return feats[:-1].contiguous(), t


def train(net, X, T, epochs: int, batch: int, lr: float, seed: int):
    """Adam on shuffled minibatches; returns the per-epoch mean losses.  The order of the samples
    is drawn on the host from a seeded generator; each minibatch is gathered on the device by
    lbm_gather_rows (torch only holds the buffers)."""
    import torch

    g = np.random.default_rng(np.random.SeedSequence(seed))
    n = X.shape[0]
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=X.dtype, device="cuda")
    tb = torch.empty((batch,) + tuple(T.shape[1:]), dtype=T.dtype, device="cuda")
    xrow, trow = X[0].numel() * X.element_size(), T[0].numel() * T.element_size()
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    losses = []
    for _ in range(epochs):
        perm = torch.from_numpy(g.permutation(n).astype(np.int32)).cuda()
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            L.lbm_gather_rows(X, n, xrow, idx, batch, xb, bad, stream)
            L.lbm_gather_rows(T, n, trow, idx, batch, tb, bad, stream)
            tot += net.train_step(xb, tb, lr)
            cnt += 1
        losses.append(tot / max(cnt, 1))
    if int(bad.item()):
        raise RuntimeError("minibatch index outside the training set")
    return losses


def predicted_maxima(net, X, kmax_now=None):
    """Predicted block maxima at t + horizon; with the sensor channel (residual form) the maxima
    now, kmax_now, are the base the predicted change applies to."""
    import torch

    y = net.forward(X)
    out = torch.empty(y.numel(), dtype=torch.float64, device="cuda")
    if X.shape[1] == 4:
        L.lbm_net_to_maxima_residual(y, kmax_now.contiguous(), y.numel(), FLOOR_K, out)
    else:
        L.lbm_net_to_maxima(y, y.numel(), LOG_OFFSET, out)
    return out.view(X.shape[0], -1)


def flags(maxima_row, T):
    import torch

    out = torch.empty(maxima_row.numel(), dtype=torch.int8, device="cuda")
    L.lbm_flags_from_maxima(maxima_row, L.LBM_F64, maxima_row.numel(), L.LBM_FLAG_THRESHOLD, T,
                            out, None)
    return out


def judge(net, feats, kmax, T, fallback_below: float):
    """Run the regrid decisions over a trace of S + 1 snapshots.  At regrid k the exact flags E_k
    of the sensor now and the flags P_k predicted from the features now for snapshot k + 1 are
    formed; lbm_flags_judge_select compares the previous prediction P_{k-1} with E_k and uses P_k
    for the coming interval if they agreed on at least `fallback_below` of the blocks, else E_k.
    Each choice is judged against the exact flags E_{k+1}, as are P_k alone and the persistence
    baseline E_k.  Everything runs on the device; the S agreements of each kind come back once.
    Returns the means, the fraction of regrids that fell back, and the per-regrid agreements
    ("per_regrid": predicted, persistence, used)."""
    import torch

    S = kmax.shape[0] - 1
    nb = kmax.shape[1]
    pred = predicted_maxima(net, feats[:-1].contiguous(), kmax[:-1])
    E = [flags(kmax[k].contiguous(), T) for k in range(S + 1)]
    P = [flags(pred[k].contiguous(), T) for k in range(S)]
    used = torch.empty(nb, dtype=torch.int8, device="cuda")
    res = torch.empty((3, S), dtype=torch.float64, device="cuda")
    fell = torch.zeros(S, dtype=torch.int32, device="cuda")
    for k in range(S):
        L.lbm_flags_judge_select(P[k - 1] if k else None, E[k], P[k], nb, fallback_below, used,
                                 None, fell[k:k + 1])
        L.lbm_flags_agreement(P[k], E[k + 1], nb, res[0, k:k + 1])
        L.lbm_flags_agreement(E[k], E[k + 1], nb, res[1, k:k + 1])
        L.lbm_flags_agreement(used, E[k + 1], nb, res[2, k:k + 1])
    r = res.cpu().numpy()
    f = fell.cpu().numpy()
    return {"agreement_predicted": float(r[0].mean()),
            "agreement_persistence": float(r[1].mean()),
            "agreement_used": float(r[2].mean()),
            "fallback_fraction": float(f.mean()), "regrids": S,
            "per_regrid": r}
