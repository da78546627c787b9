"""The regime classifier in FP64 on the CPU (PyTorch CPU convolutions as the
library primitive), with the rounding points of the method's precision
(BF16 weights and activations between layers, wider accumulation).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (Methodology and Results: a convolutional network on per-channel
normalised fields with dropout kept active for Monte Carlo uncertainty):
  x_hat = bf16((x - mean_c) / std_c)
  a_l = bf16(dropout_l(relu(conv3(a_{l-1}; W_l, b_l))))     l = 0, 1, 2
  logit = conv3(a_2; W_3, b_3),   p = sigmoid(logit)
conv3 is the 3x3x3 cross-correlation with zero "same" padding; weights are
used rounded to BF16; dropout keeps a channel with the mask of
oracle.dropout_mask and scales kept values by 1 / (1 - p).
"""
import numpy as np
import torch
import torch.nn.functional as F

from . import dropout_mask

LAYERS = [(6, 32), (32, 32), (32, 16), (16, 1)]


def bf16(t):
    """Round to BF16 through FP32 (round to nearest even), back to FP64."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


class OracleCNN:
    def __init__(self, weights, dropout=0.2, seed=7, mean=None, std=None):
        """weights: list of (W [co][ci][3][3][3], b [co]) FP32 arrays."""
        self.W = [torch.from_numpy(np.asarray(w, dtype=np.float32)).to(torch.float64) for w, _ in weights]
        self.b = [torch.from_numpy(np.asarray(b, dtype=np.float32)).to(torch.float64) for _, b in weights]
        # p as the mask realises it: round(p 2^16) / 2^16
        self.p = round(float(dropout) * 65536.0) / 65536.0
        self.seed = int(seed)
        self.mean = torch.tensor(np.zeros(6) if mean is None else np.asarray(mean, np.float32), dtype=torch.float32)
        self.std = torch.tensor(np.ones(6) if std is None else np.asarray(std, np.float32), dtype=torch.float32)

    def normalise(self, x):
        x = torch.as_tensor(np.asarray(x, dtype=np.float32))
        xh = (x - self.mean.view(1, 6, 1, 1, 1)) / self.std.view(1, 6, 1, 1, 1)
        return bf16(xh)

    def forward(self, x, pass_index=-1, return_acts=False, cells=None):
        """x: [B, 6, D, H, W] -> logits [B, D, H, W] (FP64).  cells: optional
        index of every position of the box in a larger volume, for the dropout
        streams (a sub-box of a classified grid)."""
        a = self.normalise(x)
        acts = [a]
        B, _, D, H, W = a.shape
        V = D * H * W
        for l in range(3):
            z = F.conv3d(a, bf16(self.W[l]), self.b[l], padding=1)
            h = torch.relu(z)
            if pass_index >= 0 and self.p > 0:
                keep = dropout_mask(B, h.shape[1], V, self.seed, pass_index, l, self.p, cells=cells)
                h = h * torch.from_numpy(keep.reshape(h.shape).astype(np.float64)) / (1.0 - self.p)
            a = bf16(h)
            acts.append(a)
        logit = F.conv3d(a, bf16(self.W[3]), self.b[3], padding=1)[:, 0]
        return (logit, acts) if return_acts else logit

    def mc_statistics(self, x, passes, cells=None):
        """Mean and population standard deviation of sigmoid(logit) over the passes."""
        ps = torch.stack([torch.sigmoid(self.forward(x, pass_index=k, cells=cells)) for k in range(passes)])
        return ps.mean(0), ps.std(0, unbiased=False)


def _wgrad(a, dz):
    """dW[co][ci][kz][ky][kx] = sum_{b,z,y,x} dz[b,co,z,y,x] a_pad[b,ci,z+kz,y+ky,x+kx]."""
    B, ci, D, H, W = a.shape
    ap = F.pad(a, (1, 1, 1, 1, 1, 1))
    out = torch.zeros(dz.shape[1], ci, 3, 3, 3, dtype=torch.float64)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                sh = ap[:, :, kz:kz + D, ky:ky + H, kx:kx + W]
                out[:, :, kz, ky, kx] = torch.einsum("bozyx,bizyx->oi", dz, sh)
    return out


def train_grads(net, x, y, pass_index, energy_weight, exact=False):
    """Loss and gradients of one training step (see hyb_train_step):
    L = (1/N) sum_c w_c BCE(sigmoid(logit_c), y_c), w_c = 1 + lambda e_c / mean(e),
    e_c = (|E|^2 + |B|^2)/2 of the raw input.  exact=True drops every BF16
    rounding (for the finite-difference check)."""
    rnd = (lambda t: t) if exact else bf16
    W = [w if exact else bf16(w) for w in net.W]
    xr = torch.as_tensor(np.asarray(x, dtype=np.float32))
    a = ((xr - net.mean.view(1, 6, 1, 1, 1)) / net.std.view(1, 6, 1, 1, 1)).to(torch.float64)
    a = rnd(a)
    acts = [a]
    B, _, D, H, Wd = a.shape
    V = D * H * Wd
    keeps = []
    for l in range(3):
        h = torch.relu(F.conv3d(a, W[l], net.b[l], padding=1))
        keep = torch.ones_like(h)
        if pass_index >= 0 and net.p > 0:
            keep = torch.from_numpy(dropout_mask(B, h.shape[1], V, net.seed, pass_index, l, net.p)
                                    .reshape(h.shape).astype(np.float64)) / (1.0 - net.p)
        a = rnd(h * keep)
        keeps.append(keep)
        acts.append(a)
    logit = F.conv3d(a, W[3], net.b[3], padding=1)[:, 0]
    yt = torch.as_tensor(np.asarray(y, dtype=np.float64))
    e = 0.5 * (xr.to(torch.float64) ** 2).sum(1)
    w = 1.0 + energy_weight * e / e.mean()
    bce = torch.clamp(logit, min=0) - logit * yt + torch.log1p(torch.exp(-logit.abs()))
    N = logit.numel()
    loss = (w * bce).sum() / N
    p = torch.sigmoid(logit)
    dlogit = w * (p - yt) / N
    grads = [None] * 4
    # the last layer's weight gradient is a BF16 contraction like the others:
    # its operand dL/dlogit is rounded to BF16 (its bias gradient is not)
    grads[3] = (_wgrad(acts[3], rnd(dlogit)[:, None]), dlogit.sum().reshape(1))
    dA = F.conv_transpose3d(dlogit[:, None], W[3], padding=1)
    inv = 1.0 / (1.0 - net.p) if (pass_index >= 0 and net.p > 0) else 1.0
    for l in (2, 1, 0):
        dz = rnd(dA * (acts[l + 1] > 0) * inv)
        grads[l] = (_wgrad(acts[l][:, :W[l].shape[1]], dz), dz.sum(dim=(0, 2, 3, 4)))
        if l > 0:
            dA = rnd(F.conv_transpose3d(dz, W[l], padding=1))
    acc = ((p >= 0.5) == (yt >= 0.5)).double().mean()
    return dict(loss=float(loss), bce=float(bce.mean()), accuracy=float(acc), grads=grads, logit=logit)


def loss_only(net, x, y, pass_index, energy_weight):
    return train_grads(net, x, y, pass_index, energy_weight, exact=True)["loss"]


def adam_update(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on FP64 tensors; returns (w', m', v').
    t is the step count after this update (1 for the first step).  The paper
    leaves the optimizer unstated; Adam with these defaults is the reading the
    training step follows.
      m' = beta1 m + (1 - beta1) g,   v' = beta2 v + (1 - beta2) g^2
      w' = w - lr * (m' / (1 - beta1^t)) / (sqrt(v' / (1 - beta2^t)) + eps)"""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (torch.sqrt(vhat) + eps), m, v


def train_run(weights, x, y, steps, dropout, seed, energy_weight, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              mean=None, std=None):
    """`steps` training steps on one batch, as hyb_train_step takes them: the
    forward/backward of train_grads with the dropout masks of pass = step
    index (0, 1, ...), then Adam on FP64 master weights (the weights the
    network uses are those masters rounded to BF16 inside train_grads).
    Returns the final [(W, b)] as FP64 tensors, the per-step losses, the
    per-step gradients and the [(W, b)] after every step."""
    net = OracleCNN(weights, dropout=dropout, seed=seed, mean=mean, std=std)
    mw = [torch.zeros_like(w) for w in net.W]
    vw = [torch.zeros_like(w) for w in net.W]
    mb = [torch.zeros_like(b) for b in net.b]
    vb = [torch.zeros_like(b) for b in net.b]
    losses, grads, history = [], [], []
    for t in range(steps):
        out = train_grads(net, x, y, pass_index=t, energy_weight=energy_weight)
        losses.append(out["loss"])
        grads.append(out["grads"])
        for l in range(4):
            gw, gb = out["grads"][l]
            net.W[l], mw[l], vw[l] = adam_update(net.W[l], gw, mw[l], vw[l], t + 1, lr, beta1, beta2, eps)
            net.b[l], mb[l], vb[l] = adam_update(net.b[l], gb, mb[l], vb[l], t + 1, lr, beta1, beta2, eps)
        history.append([(net.W[l].clone(), net.b[l].clone()) for l in range(4)])
    return [(net.W[l], net.b[l]) for l in range(4)], losses, grads, history
