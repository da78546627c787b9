"""The field surrogate (the paper's StatePredictor, Results and Table 2) in
FP64 on the CPU, with PyTorch CPU convolutions as the library primitive and
the rounding points of the method's precision (BF16 weights and
activations, wider accumulation).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (Table 2: 3D convolutions 10 -> 13 -> 32 -> 64 -> 128 -> 32 -> 10 with
ReLU, residual connections on the first three layers and dropout 0.1 after
the second):
  a_0 = bf16((s - mean_c) / std_c)                      s: E, B, J, rho
  a_1 = bf16(relu(conv(a_0; W_0) + b_0) + pad(a_0))
  a_2 = bf16(relu(conv(a_1; W_1) + b_1) keep / (1 - p) + pad(a_1))
  a_3 = bf16(relu(conv(a_2; W_2) + b_2) + pad(a_2))
  a_4 = bf16(relu(conv(a_3; W_3) + b_3))
  a_5 = bf16(relu(conv(a_4; W_4) + b_4))
  y   = conv(a_5; W_5) + b_5,  prediction = s_c + dstd_c y_c
The output is the change of the state over the lead time in units dstd_c
(the spread of that change; std_c when not given), added to the input state
(a residual forecast: with every weight zero the prediction is the input,
persistence).
"pad" is the identity shortcut with the extra channels zero (the reading of
a residual between layers of different width); conv is the 3x3x3
cross-correlation with zero "same" padding and BF16-rounded weights; keep is
the dropout mask of oracle.dropout_mask (layer index 1).

Loss (Table 2: Huber with delta = 0.01 plus 0.1 times the energy violation):
  L = (1/N) sum huber(y - t_hat) + lambda v^2,  t_hat = (t - s) / dstd_c,
  v = (sum_b W(pred_b) - sum_b W(t_b)) / sum_b W(t_b),  W = (1/2) sum over a
  patch of the squares of channels 0..5 (E and B) in physical units: the
  relative violation of the batch's total field energy.  (Relative to each
  patch's own energy the violation diverges on patches of empty vacuum;
  per patch relative to the mean it outweighs the Huber term some 70-fold
  and the fit does not learn the fields.)
"""
import numpy as np
import torch
import torch.nn.functional as F

from . import charge_density, dropout_mask, node_fields, Particles
from .classifier import _wgrad, adam_update, bf16

LAYERS = [(10, 13), (13, 32), (32, 64), (64, 128), (128, 32), (32, 10)]
RESIDUAL = [True, True, True, False, False, False]
RELU = [True, True, True, True, True, False]
DROP_LAYER = 1


def _pad_channels(a, c):
    """a [B, ci, ...] zero-padded to c channels."""
    if a.shape[1] == c:
        return a
    z = torch.zeros((a.shape[0], c - a.shape[1]) + tuple(a.shape[2:]), dtype=a.dtype)
    return torch.cat([a, z], dim=1)


class OracleSurrogate:
    def __init__(self, weights, dropout=0.1, seed=11, mean=None, std=None, dstd=None):
        """weights: list of six (W [co][ci][3][3][3], b [co]) FP32 arrays."""
        self.W = [torch.from_numpy(np.asarray(w, dtype=np.float32)).to(torch.float64) for w, _ in weights]
        self.b = [torch.from_numpy(np.asarray(b, dtype=np.float32)).to(torch.float64) for _, b in weights]
        self.p = round(float(dropout) * 65536.0) / 65536.0
        self.seed = int(seed)
        self.mean = torch.tensor(np.zeros(10) if mean is None else np.asarray(mean, np.float32), dtype=torch.float32)
        self.std = torch.tensor(np.ones(10) if std is None else np.asarray(std, np.float32), dtype=torch.float32)
        ds = self.std.numpy() if dstd is None else np.where(np.asarray(dstd, np.float32) > 0,
                                                              np.asarray(dstd, np.float32), self.std.numpy())
        self.dstd = torch.tensor(ds, dtype=torch.float32)

    def normalise(self, x):
        x = torch.as_tensor(np.asarray(x, dtype=np.float32))
        return (x - self.mean.view(1, 10, 1, 1, 1)) / self.std.view(1, 10, 1, 1, 1)

    def _keep(self, B, C_, V, pass_index, cells=None):
        if pass_index < 0 or self.p <= 0:
            return None
        k = dropout_mask(B, C_, V, self.seed, pass_index, DROP_LAYER, self.p, cells=cells)
        return torch.from_numpy(k.astype(np.float64)) / (1.0 - self.p)

    def forward(self, x, pass_index=-1, exact=False, record=False):
        """x: states [B, 10, D, H, W] -> normalised output y (FP64); with
        record, also the activations a_l, the pre-activations s_l and the
        dropout factors.  exact drops every BF16 rounding."""
        rnd = (lambda t: t) if exact else bf16
        a = rnd(self.normalise(x).to(torch.float64))
        B, _, D, H, W = a.shape
        V = D * H * W
        acts, pres, keeps = [a], [], []
        for l, (ci, co) in enumerate(LAYERS):
            s = F.conv3d(a, self.W[l] if exact else bf16(self.W[l]), self.b[l], padding=1)
            pres.append(s)
            h = torch.relu(s) if RELU[l] else s
            keep = None
            if l == DROP_LAYER:
                # the mask covers the layer's channels padded to a multiple of 8
                kc = self._keep(B, (co + 7) // 8 * 8, V, pass_index)
                if kc is not None:
                    keep = kc[:, :co].reshape(B, co, D, H, W)
                    h = h * keep
            keeps.append(keep)
            if RESIDUAL[l]:
                h = h + _pad_channels(a, co)
            a = h if l == len(LAYERS) - 1 else rnd(h)
            acts.append(a)
        y = acts[-1]
        return (y, acts, pres, keeps) if record else y

    def predict(self, x, pass_index=-1, exact=False):
        y = self.forward(x, pass_index, exact)
        xs = torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.float64)
        return xs + y * self.dstd.view(1, 10, 1, 1, 1).to(torch.float64)

    def mc_statistics(self, x, passes):
        """Mean and population standard deviation of the prediction over the passes."""
        ps = torch.stack([self.predict(x, pass_index=k) for k in range(passes)])
        return ps.mean(0), ps.std(0, unbiased=False)


def loss_and_grads(net, x, t, pass_index, delta=0.01, energy_weight=0.1, exact=False):
    """Loss and gradients of one training step (hyb_surrogate_train_step): the
    forward above, the loss of the module docstring, and the backward with the
    data gradient dz_l = bf16(dL/ds_l) as the rounded operand (exact: no
    rounding).  Returns dict(loss, huber, energy, grads=[(gW, gb)] * 6, y)."""
    rnd = (lambda v: v) if exact else bf16
    y, acts, pres, keeps = net.forward(x, pass_index, exact=exact, record=True)
    sd = net.dstd.view(1, 10, 1, 1, 1).to(torch.float64)
    tt = torch.as_tensor(np.asarray(t, dtype=np.float32))
    xs = torch.as_tensor(np.asarray(x, dtype=np.float32))
    tn = ((tt - xs) / net.dstd.view(1, 10, 1, 1, 1)).to(torch.float64)
    B = y.shape[0]
    N = y.numel()
    r = y - tn
    ar = r.abs()
    hub = torch.where(ar <= delta, 0.5 * r * r, delta * (ar - 0.5 * delta))
    dhub = torch.where(ar <= delta, r, delta * torch.sign(r))
    pred = xs.to(torch.float64) + y * sd
    wp = 0.5 * (pred[:, :6] ** 2).sum(dim=(1, 2, 3, 4))
    wt = 0.5 * (tt[:, :6].to(torch.float64) ** 2).sum(dim=(1, 2, 3, 4))
    wtot = float(wt.sum())
    v = (float(wp.sum()) - wtot) / wtot if wtot > 0 else 0.0
    loss = hub.sum() / N + energy_weight * v * v
    G = dhub / N
    coef = 2.0 * v / wtot if wtot > 0 else 0.0
    G[:, :6] += energy_weight * coef * sd[:, :6] * pred[:, :6]
    grads = [None] * len(LAYERS)
    for l in range(len(LAYERS) - 1, -1, -1):
        ci, co = LAYERS[l]
        ds = G
        if RELU[l]:
            ds = ds * (pres[l] > 0)
        if keeps[l] is not None:
            ds = ds * keeps[l]
        dz = rnd(ds)
        grads[l] = (_wgrad(acts[l], dz), dz.sum(dim=(0, 2, 3, 4)))
        if l > 0:
            Wl = net.W[l] if exact else bf16(net.W[l])
            Gl = F.conv_transpose3d(dz, Wl, padding=1)
            if RESIDUAL[l]:
                Gl = Gl + G[:, :ci]
            G = Gl
    return dict(loss=float(loss), huber=float(hub.sum() / N), energy=v * v, grads=grads, y=y)


def train_run(weights, x, t, steps, dropout, seed, delta=0.01, energy_weight=0.1, lr=1e-3, mean=None, std=None,
              dstd=None):
    """`steps` steps on one batch as hyb_surrogate_train_step takes them
    (dropout masks of pass = step index, Adam on FP64 masters); returns the
    [(W, b)] after every step and the per-step losses."""
    net = OracleSurrogate(weights, dropout=dropout, seed=seed, mean=mean, std=std, dstd=dstd)
    mw = [torch.zeros_like(w) for w in net.W]
    vw = [torch.zeros_like(w) for w in net.W]
    mb = [torch.zeros_like(b) for b in net.b]
    vb = [torch.zeros_like(b) for b in net.b]
    history, losses = [], []
    for k in range(steps):
        out = loss_and_grads(net, x, t, k, delta, energy_weight)
        losses.append(out["loss"])
        for l in range(len(LAYERS)):
            gw, gb = out["grads"][l]
            net.W[l], mw[l], vw[l] = adam_update(net.W[l], gw, mw[l], vw[l], k + 1, lr)
            net.b[l], mb[l], vb[l] = adam_update(net.b[l], gb, mb[l], vb[l], k + 1, lr)
        history.append([(net.W[l].clone(), net.b[l].clone()) for l in range(len(LAYERS))])
    return history, losses


def node_state(g, E, B, J, species=(), fluids=(), rho_bg=None):
    """The ten node channels of hyb_node_state: E and B averaged to the nodes
    as the classifier takes them, J averaged over its two edges like E, and
    rho = the CIC charge of every particle species (q w / dV, times the charge
    state where given) + q n of every fluid + rho_bg.  species: (q, m, dict of
    x, y, z, ux, uy, uz, w[, zq]); fluids: (q, n)."""
    nz, ny, nx = g.shape
    out = np.zeros((10, nz, ny, nx))
    zero = np.zeros_like(np.asarray(E, dtype=np.float64))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e, b = node_fields(g, E, B, i, j, k)
                jn, _ = node_fields(g, J, zero, i, j, k)
                out[0:3, k, j, i] = e
                out[3:6, k, j, i] = b
                out[6:9, k, j, i] = jn
    rho = np.zeros(g.shape)
    for q, m, sp in species:
        zq = sp.get("zq")
        charge_density(g, Particles(q, m, sp["x"], sp["y"], sp["z"], sp["ux"], sp["uy"], sp["uz"],
                                    np.asarray(sp["w"], np.float64) * (1.0 if zq is None else np.asarray(zq, np.float64))),
                       rho)
    for q, n in fluids:
        rho += q * np.asarray(n, np.float64)
    if rho_bg is not None:
        rho += np.asarray(rho_bg, np.float64)
    out[9] = rho
    return out
