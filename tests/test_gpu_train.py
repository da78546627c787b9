"""GPU classifier training against the oracle: the gradients of one step of
the energy-weighted BCE through the BF16 tensor-core backward, on the same
weights, inputs and dropout masks; and a short training run that learns a
physics label."""
import math

import numpy as np
import pytest

from _util import require_gpu, rel_l2, seeded_classifier

pytestmark = pytest.mark.gpu


def _case(seed=1, B=2, D=4, H=16, W=16):
    """Normal inputs with a label a linear threshold of two channels decides."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 6, D, H, W)).astype(np.float32)
    y = (x[:, 0] + 0.5 * x[:, 1] > 0.2).astype(np.float32)
    return x, y


def test_one_step_gradients_match_oracle():
    P = require_gpu()
    import torch
    from oracle.classifier import OracleCNN, train_grads
    m, weights = seeded_classifier(P, 21, dropout=0.2, mc_passes=1, energy_weight=0.1)
    net = OracleCNN(weights, dropout=0.2, seed=21)
    x, y = _case()
    st = m.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    ref = train_grads(net, x, y, pass_index=0, energy_weight=0.1)
    assert st["loss"] == pytest.approx(ref["loss"], rel=1e-3)
    assert st["bce"] == pytest.approx(ref["bce"], rel=1e-3)
    for l in range(4):
        gw, gb = m.get_grad(l)
        rw, rb = ref["grads"][l]
        # 1e-3, except the first layer's weight gradient: BF16 rounding points
        # shared with the oracle still flip where FP32 and FP64 sums straddle a
        # rounding boundary, and the flips of every layer collect in layer 0
        # (measured up to 1.0e-3 there; an FP32-summing copy of the oracle
        # itself differs from the FP64 one by up to 1e-2 on such inputs)
        tol = 2e-3 if l == 0 else 1e-3
        assert rel_l2(gw, rw.numpy()) <= tol, (l, rel_l2(gw, rw.numpy()))
        assert rel_l2(gb, rb.numpy()) <= tol, (l, rel_l2(gb, rb.numpy()))


def test_training_lowers_the_loss():
    P = require_gpu()
    import torch
    from paper_2510_11174_gb300.model import Classifier
    m = Classifier(dropout=0.1, mc_passes=1, seed=3, lr=3e-3, energy_weight=0.1)
    x, y = _case(seed=5, B=4, D=8, H=16, W=16)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    first = m.train_step(xt, yt)
    for _ in range(80):
        last = m.train_step(xt, yt)
    assert last["loss"] < 0.5 * first["loss"]
    assert last["accuracy"] > 0.85
    assert last["step"] == 81


def test_three_adam_steps_match_oracle():
    """Three training steps (forward, backward, Adam) on the GPU against the
    oracle's own three steps from the same weights and data, update by update.
    Adam normalises by |g|: where a weight's gradient is well above the
    gradient parity at every step so far, each step's update must agree with
    the oracle's (first step: -lr sign(g) exactly); a weight whose gradient
    is near zero may take the opposite sign, which only the layer-wide bound
    covers."""
    P = require_gpu()
    import torch
    from oracle.classifier import train_run
    lr = 1e-3
    m, w0 = seeded_classifier(P, 21, dropout=0.2, mc_passes=1, energy_weight=0.1, lr=lr)
    x, y = _case(seed=2)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    gpu_hist = []
    for _ in range(3):
        m.train_step(xt, yt)
        gpu_hist.append([tuple(a.astype(np.float64) for a in m.get_layer(l)) for l in range(4)])
    ref, losses, grads, hist = train_run(w0, x, y, 3, dropout=0.2, seed=21, energy_weight=0.1, lr=lr)
    for l in range(4):
        for k in range(2):
            prev_g, prev_o = w0[l][k].astype(np.float64), w0[l][k].astype(np.float64)
            strong = np.ones(w0[l][k].shape, bool)
            for t in range(3):
                cur_g, cur_o = gpu_hist[t][l][k], hist[t][l][k].numpy()
                d_gpu, d_orc = cur_g - prev_g, cur_o - prev_o
                g = grads[t][l][k].numpy()
                strong &= np.abs(g) >= 0.3 * np.sqrt(np.mean(g ** 2))
                if strong.sum() >= 4:
                    # the update -lr m_hat / sqrt(v_hat) moves by about lr dg / sqrt(v_hat)
                    # for a gradient error dg; sqrt(v_hat) >= 0.3 rms(g) here, so a gradient
                    # parity of ~1e-3 rms(g) bounds the update error by about 3e-3 lr (m_hat
                    # itself may cancel between steps, so the error is taken relative to lr;
                    # measured: median 3.6e-3 lr, 99th percentile 6e-2 lr in layer 0)
                    err = np.abs(d_gpu - d_orc)[strong] / lr
                    assert np.median(err) <= 1e-2 and np.quantile(err, 0.99) <= 0.1, \
                        (l, k, t, np.median(err), np.quantile(err, 0.99))
                    if t == 0:   # the first step is -lr sign(g)
                        assert np.all(np.abs(np.abs(d_gpu[strong]) / lr - 1.0) <= 1e-3)
                # the first steps' bias-corrected moments keep |m_hat| / sqrt(v_hat) near 1
                assert np.all(np.abs(d_gpu) <= 1.2 * lr)
                assert rel_l2(d_gpu, d_orc) <= 0.1, (l, k, t, rel_l2(d_gpu, d_orc))
                prev_g, prev_o = cur_g, cur_o
