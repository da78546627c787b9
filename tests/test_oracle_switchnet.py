"""Pins of the SwitchNet oracle (oracle/switchnet.py): the attention layer on
a single token equals PyTorch's multi-head attention on a sequence of length
one (a library routine), the backward pass agrees with FP64 central
differences, and the AUC of known rankings."""
import math

import numpy as np
import pytest
import torch

from oracle import switchnet as S


def _weights(seed):
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in S.LAYERS:
        lim = math.sqrt(6.0 / ci)
        out.append((rng.uniform(-lim, lim, (co, ci)).astype(np.float32),
                    rng.uniform(-0.1, 0.1, co).astype(np.float32)))
    return out


def test_single_token_attention_is_the_value_and_output_projection():
    torch.manual_seed(0)
    mha = torch.nn.MultiheadAttention(256, 4, dtype=torch.float64)
    w = _weights(1)
    # layers 0 and 1 zero with zero biases: a_2 is the normalised input padded to 256
    w[0] = (np.zeros_like(w[0][0]), np.zeros_like(w[0][1]))
    w[1] = (np.zeros_like(w[1][0]), np.zeros_like(w[1][1]))
    net = S.OracleSwitchNet(w)
    x = np.random.default_rng(2).standard_normal((10, 50)).astype(np.float32)
    a2 = torch.zeros(50, 256, dtype=torch.float64)
    a2[:, :10] = torch.from_numpy(x.T.astype(np.float64))
    # the value and output projections of the attention layer (FP64)
    net.W[2] = mha.in_proj_weight[512:].detach().clone()
    net.b[2] = mha.in_proj_bias[512:].detach().clone()
    net.W[3] = mha.out_proj.weight.detach().clone()
    net.b[3] = mha.out_proj.bias.detach().clone()
    logit = net.forward(x, exact=True)
    with torch.no_grad():
        att, _ = mha(a2[None], a2[None], a2[None])           # (L = 1, N = 50, E = 256)
    ref = att[0] @ net.W[4][0] + net.b[4][0]
    np.testing.assert_allclose(logit.numpy(), ref.numpy(), rtol=1e-12, atol=1e-12)


def test_backward_matches_central_differences():
    w = _weights(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((10, 40)).astype(np.float32)
    y = (rng.random(40) < 0.4).astype(np.float64)
    net = S.OracleSwitchNet(w, dropout=0.2)
    out = S.loss_and_grads(net, x, y, 2, exact=True)
    h = 1e-6
    for l in range(5):
        gw, gb = out["grads"][l]
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in net.W[l].shape)
            w0 = net.W[l][idx].item()
            net.W[l][idx] = w0 + h
            lp = S.loss_and_grads(net, x, y, 2, exact=True)["loss"]
            net.W[l][idx] = w0 - h
            lm = S.loss_and_grads(net, x, y, 2, exact=True)["loss"]
            net.W[l][idx] = w0
            assert gw[idx].item() == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-10), (l, idx)
        c = int(rng.integers(0, net.b[l].shape[0]))
        b0 = net.b[l][c].item()
        net.b[l][c] = b0 + h
        lp = S.loss_and_grads(net, x, y, 2, exact=True)["loss"]
        net.b[l][c] = b0 - h
        lm = S.loss_and_grads(net, x, y, 2, exact=True)["loss"]
        net.b[l][c] = b0
        assert gb[c].item() == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-10), (l, c)


def test_auc_of_known_rankings():
    y = np.array([0, 0, 1, 1])
    assert S.auc([0.1, 0.2, 0.8, 0.9], y) == 1.0
    assert S.auc([0.9, 0.8, 0.2, 0.1], y) == 0.0
    assert S.auc([0.5, 0.5, 0.5, 0.5], y) == 0.5
    # one positive below one negative: 3 of 4 pairs ordered
    assert S.auc([0.1, 0.6, 0.5, 0.9], y) == 0.75
    rng = np.random.default_rng(5)
    s, lab = rng.random(2000), rng.random(2000) < 0.3
    pos, neg = s[lab], s[~lab]
    brute = np.mean((pos[:, None] > neg[None, :]) + 0.5 * (pos[:, None] == neg[None, :]))
    assert S.auc(s, lab) == pytest.approx(brute, abs=1e-12)
