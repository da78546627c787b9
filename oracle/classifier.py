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
        self.p = float(dropout)
        self.seed = int(seed)
        self.mean = torch.tensor(np.zeros(6) if mean is None else np.asarray(mean, np.float32), dtype=torch.float32)
        self.std = torch.tensor(np.ones(6) if std is None else np.asarray(std, np.float32), dtype=torch.float32)

    def normalise(self, x):
        x = torch.as_tensor(np.asarray(x, dtype=np.float32))
        xh = (x - self.mean.view(1, 6, 1, 1, 1)) / self.std.view(1, 6, 1, 1, 1)
        return bf16(xh)

    def forward(self, x, pass_index=-1, return_acts=False):
        """x: [B, 6, D, H, W] -> logits [B, D, H, W] (FP64)."""
        a = self.normalise(x)
        acts = [a]
        B, _, D, H, W = a.shape
        V = D * H * W
        for l in range(3):
            z = F.conv3d(a, bf16(self.W[l]), self.b[l], padding=1)
            h = torch.relu(z)
            if pass_index >= 0 and self.p > 0:
                keep = dropout_mask(B, h.shape[1], V, self.seed, pass_index, l, self.p)
                h = h * torch.from_numpy(keep.reshape(h.shape).astype(np.float64)) / (1.0 - self.p)
            a = bf16(h)
            acts.append(a)
        logit = F.conv3d(a, bf16(self.W[3]), self.b[3], padding=1)[:, 0]
        return (logit, acts) if return_acts else logit

    def mc_statistics(self, x, passes):
        """Mean and population standard deviation of sigmoid(logit) over the passes."""
        ps = torch.stack([torch.sigmoid(self.forward(x, pass_index=k)) for k in range(passes)])
        return ps.mean(0), ps.std(0, unbiased=False)
