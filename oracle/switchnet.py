"""SwitchNet, the paper's per-cell regime classifier (Table 1), in FP64 on the
CPU with the rounding points of the method's precision (BF16 weights and
activations, wider accumulation).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (Table 1: linear 10 -> 128 and 128 -> 256 with ReLU and residuals,
dropout 0.2, multi-head attention 256 -> 256, linear 256 -> 1 and sigmoid),
per cell, x the ten node channels E, B, J, rho:
  a_0 = bf16((x - mean_c) / std_c)
  a_1 = bf16(relu(W_0 a_0 + b_0) + pad(a_0))
  a_2 = bf16(relu(W_1 a_1 + b_1) keep / (1 - p) + pad(a_1))
  a_3 = bf16(W_v a_2 + b_v)            attention over a single token: the
  a_4 = bf16(W_o a_3 + b_o)            softmax weight is 1
  logit = bf16(w_4) . a_4 + b_4
Loss: the regime classifier's energy-weighted BCE
  L = (1/N) sum_c w_c BCE(sigmoid(logit_c), y_c),  w_c = 1 + lambda e_c / mean(e),
  e_c = (|E|^2 + |B|^2) / 2 of the raw features.
"""
import numpy as np
import torch

from . import dropout_mask
from .classifier import adam_update, bf16

LAYERS = [(10, 128), (128, 256), (256, 256), (256, 256), (256, 1)]
RELU = [True, True, False, False, False]
RESIDUAL = [True, True, False, False, False]
DROP_LAYER = 1


def _pad(a, c):
    if a.shape[1] == c:
        return a
    return torch.cat([a, torch.zeros((a.shape[0], c - a.shape[1]), dtype=a.dtype)], dim=1)


class OracleSwitchNet:
    def __init__(self, weights, dropout=0.2, seed=13, mean=None, std=None):
        """weights: five (W [co][ci], b [co]) FP32 arrays."""
        self.W = [torch.from_numpy(np.asarray(w, dtype=np.float32)).to(torch.float64) for w, _ in weights]
        self.b = [torch.from_numpy(np.asarray(b, dtype=np.float32)).to(torch.float64) for _, b in weights]
        self.p = round(float(dropout) * 65536.0) / 65536.0
        self.seed = int(seed)
        self.mean = torch.tensor(np.zeros(10) if mean is None else np.asarray(mean, np.float32), dtype=torch.float32)
        self.std = torch.tensor(np.ones(10) if std is None else np.asarray(std, np.float32), dtype=torch.float32)

    def forward(self, x, pass_index=-1, exact=False, record=False):
        """x: features [10, n] -> logits [n] (FP64)."""
        rnd = (lambda t: t) if exact else bf16
        xt = torch.as_tensor(np.asarray(x, dtype=np.float32))
        a = rnd(((xt - self.mean.view(10, 1)) / self.std.view(10, 1)).T.to(torch.float64))
        n = a.shape[0]
        acts, pres, keeps = [a], [], []
        for l in range(4):
            s = a @ (self.W[l] if exact else bf16(self.W[l])).T + self.b[l]
            pres.append(s)
            h = torch.relu(s) if RELU[l] else s
            keep = None
            if l == DROP_LAYER and pass_index >= 0 and self.p > 0:
                k = dropout_mask(1, LAYERS[l][1], n, self.seed, pass_index, l, self.p)[0]
                keep = torch.from_numpy(k.astype(np.float64)).T / (1.0 - self.p)
                h = h * keep
            keeps.append(keep)
            if RESIDUAL[l]:
                h = h + _pad(a, LAYERS[l][1])
            a = rnd(h)
            acts.append(a)
        logit = a @ (self.W[4] if exact else bf16(self.W[4]))[0] + self.b[4][0]
        return (logit, acts, pres, keeps) if record else logit

    def mc_statistics(self, x, passes):
        ps = torch.stack([torch.sigmoid(self.forward(x, pass_index=k)) for k in range(passes)])
        return ps.mean(0), ps.std(0, unbiased=False)


def loss_and_grads(net, x, y, pass_index, energy_weight=0.1, exact=False):
    """Loss and gradients of one training step (hyb_switchnet_train_step); the
    data gradient dz_l = bf16(dL/ds_l) is the rounded operand (and the output
    layer's weight gradient takes bf16(dL/dlogit)).  exact: no rounding."""
    rnd = (lambda t: t) if exact else bf16
    logit, acts, pres, keeps = net.forward(x, pass_index, exact=exact, record=True)
    xt = torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.float64)
    yt = torch.as_tensor(np.asarray(y, dtype=np.float64))
    e = 0.5 * (xt[:6] ** 2).sum(0)
    w = 1.0 + energy_weight * e / e.mean()
    bce = torch.clamp(logit, min=0) - logit * yt + torch.log1p(torch.exp(-logit.abs()))
    n = logit.numel()
    loss = (w * bce).sum() / n
    p = torch.sigmoid(logit)
    dlogit = w * (p - yt) / n
    grads = [None] * 5
    w4 = net.W[4] if exact else bf16(net.W[4])
    dl = rnd(dlogit)
    grads[4] = ((dl[:, None] * acts[4]).sum(0)[None, :], dl.sum().reshape(1))
    dz = rnd(dlogit[:, None] * w4[0][None, :])
    G = None
    for l in range(3, -1, -1):
        if l < 3:
            ds = G
            if RELU[l]:
                ds = ds * (pres[l] > 0)
            if keeps[l] is not None:
                ds = ds * keeps[l]
            dz = rnd(ds)
        ci = LAYERS[l][0]
        grads[l] = (dz.T @ acts[l][:, :ci], dz.sum(0))
        if l > 0:
            Wl = net.W[l] if exact else bf16(net.W[l])
            Gl = dz @ Wl
            if RESIDUAL[l]:
                Gl = Gl + G[:, :ci]
            G = Gl
    acc = ((p >= 0.5) == (yt >= 0.5)).double().mean()
    return dict(loss=float(loss), bce=float(bce.mean()), accuracy=float(acc), grads=grads, logit=logit)


def train_run(weights, x, y, steps, dropout, seed, energy_weight=0.1, lr=1e-3, mean=None, std=None):
    """`steps` Adam steps on one batch as hyb_switchnet_train_step takes them;
    returns the [(W, b)] after every step and the losses."""
    net = OracleSwitchNet(weights, dropout=dropout, seed=seed, mean=mean, std=std)
    mom = [[torch.zeros_like(t) for t in (w, w, b, b)] for w, b in zip(net.W, net.b)]
    history, losses = [], []
    for k in range(steps):
        out = loss_and_grads(net, x, y, k, energy_weight)
        losses.append(out["loss"])
        for l in range(5):
            gw, gb = out["grads"][l]
            net.W[l], mom[l][0], mom[l][1] = adam_update(net.W[l], gw, mom[l][0], mom[l][1], k + 1, lr)
            net.b[l], mom[l][2], mom[l][3] = adam_update(net.b[l], gb, mom[l][2], mom[l][3], k + 1, lr)
        history.append([(net.W[l].clone(), net.b[l].clone()) for l in range(5)])
    return history, losses


def auc(score, label):
    """Area under the ROC curve: the probability that a random positive scores
    above a random negative (ties count one half), by ranks (Mann-Whitney U)."""
    score = np.asarray(score, dtype=np.float64).ravel()
    label = np.asarray(label).ravel() > 0.5
    npos, nneg = int(label.sum()), int((~label).sum())
    if npos == 0 or nneg == 0:
        return float("nan")
    order = np.argsort(score, kind="mergesort")
    s = score[order]
    ranks = np.empty(len(s))
    i = 0
    while i < len(s):
        j = i
        while j + 1 < len(s) and s[j + 1] == s[i]:
            j += 1
        ranks[i:j + 1] = 0.5 * (i + j) + 1.0
        i = j + 1
    r = np.empty(len(s))
    r[order] = ranks
    return float((r[label].sum() - npos * (npos + 1) / 2.0) / (npos * nneg))
