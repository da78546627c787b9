"""Pins of the oracle's classifier: the orientation of the 3x3x3 taps (a
one-hot kernel is a shift), BF16 rounding points, the dropout mask law,
the MC statistics definitions, and the layers' composition against an
explicit-loop evaluation."""
import numpy as np
import pytest
import torch

import oracle
from oracle.classifier import LAYERS, OracleCNN, bf16


def _weights(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return [(scale * rng.standard_normal((co, ci, 3, 3, 3)).astype(np.float32) / np.sqrt(ci * 27),
             (0.1 * rng.standard_normal(co)).astype(np.float32)) for ci, co in LAYERS]


def test_one_hot_kernel_is_a_shift():
    x = torch.arange(2 * 1 * 4 * 5 * 6, dtype=torch.float64).reshape(2, 1, 4, 5, 6)
    w = torch.zeros(1, 1, 3, 3, 3, dtype=torch.float64)
    w[0, 0, 2, 1, 0] = 1.0  # (kz, ky, kx): output(z, y, x) = input(z + 1, y, x - 1)
    y = torch.nn.functional.conv3d(x, w, padding=1)
    assert torch.equal(y[:, 0, :3, :, 1:], x[:, 0, 1:, :, :5])
    assert torch.all(y[:, 0, 3] == 0) and torch.all(y[:, 0, :, :, 0] == 0)


def test_bf16_rounding_is_round_to_nearest_even():
    v = torch.tensor([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9], dtype=torch.float64)
    # BF16 keeps 8 significant bits: ties go to even, below-half rounds down
    assert bf16(v).tolist() == [1.0, 1.0 + 2 ** -6, 1.0]


def test_dropout_mask_law_and_pass_dependence():
    p = 0.2
    m0 = oracle.dropout_mask(2, 32, 4096, 7, 0, 1, p)
    m1 = oracle.dropout_mask(2, 32, 4096, 7, 1, 1, p)
    n = m0.size
    assert abs(m0.mean() - (1 - p)) < 3 * np.sqrt(p * (1 - p) / n)
    assert 0.25 < np.mean(m0 != m1) < 0.4          # independent passes: 2 p (1 - p) = 0.32
    # the documented Philox stream: channel 9 -> counter word (1 << 16) | 1,
    # field 9 % 8 = 1 = high half of word 0
    r = oracle.philox([17, 1, (1 << 16) | (9 // 8), 0], [7, 0xD0])
    assert m0[1, 9, 17] == (((int(r[0]) >> 16) & 0xFFFF) >= round(p * 65536))
    r = oracle.philox([17, 1, (1 << 16) | (30 // 8), 0], [7, 0xD0])
    assert m0[1, 30, 17] == ((int(r[3]) & 0xFFFF) >= round(p * 65536))


def test_mc_statistics_are_mean_and_population_std():
    net = OracleCNN(_weights(1), dropout=0.3, seed=11)
    x = np.random.default_rng(2).standard_normal((1, 6, 2, 16, 8)).astype(np.float32)
    m, s = net.mc_statistics(x, 5)
    ps = torch.stack([torch.sigmoid(net.forward(x, k)) for k in range(5)])
    assert torch.allclose(m, ps.mean(0)) and torch.allclose(s, torch.sqrt(((ps - ps.mean(0)) ** 2).mean(0)))
    # without dropout every pass is the same network
    net0 = OracleCNN(_weights(1), dropout=0.0, seed=11)
    m0, s0 = net0.mc_statistics(x, 3)
    assert torch.all(s0 == 0)


def test_oracle_backward_matches_central_differences():
    """Exact FP64 backward of the energy-weighted BCE against central differences."""
    from oracle.classifier import train_grads
    rng = np.random.default_rng(4)
    net = OracleCNN(_weights(3, scale=2.0), dropout=0.2, seed=5)
    x = rng.standard_normal((1, 6, 2, 16, 8)).astype(np.float32)
    y = (rng.random((1, 2, 16, 8)) < 0.4).astype(np.float32)
    out = train_grads(net, x, y, pass_index=2, energy_weight=0.1, exact=True)
    h = 1e-6
    for l in range(4):
        gw, gb = out["grads"][l]
        for idx in [(0, 0, 1, 1, 1), (gw.shape[0] - 1, gw.shape[1] - 1, 0, 2, 1), (0, gw.shape[1] // 2, 2, 0, 0)]:
            w0 = net.W[l][idx].item()
            net.W[l][idx] = w0 + h
            lp = train_grads(net, x, y, 2, 0.1, exact=True)["loss"]
            net.W[l][idx] = w0 - h
            lm = train_grads(net, x, y, 2, 0.1, exact=True)["loss"]
            net.W[l][idx] = w0
            fd = (lp - lm) / (2 * h)
            assert gw[idx].item() == pytest.approx(fd, rel=1e-6, abs=1e-11), (l, idx)
        b0 = net.b[l][0].item()
        net.b[l][0] = b0 + h
        lp = train_grads(net, x, y, 2, 0.1, exact=True)["loss"]
        net.b[l][0] = b0 - h
        lm = train_grads(net, x, y, 2, 0.1, exact=True)["loss"]
        net.b[l][0] = b0
        assert gb[0].item() == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-11), l


def test_adam_first_step_is_lr_times_sign():
    """First step: m_hat = g and v_hat = g^2 exactly, so w' = w - lr g / (|g| + eps)."""
    from oracle.classifier import adam_update
    rng = np.random.default_rng(8)
    w = torch.from_numpy(rng.standard_normal(200))
    g = torch.from_numpy(rng.standard_normal(200) * np.exp(rng.uniform(-20, 3, 200)))
    z = torch.zeros_like(w)
    w1, m1, v1 = adam_update(w, g, z, z, 1, lr=1e-3, eps=1e-8)
    assert torch.allclose(w1, w - 1e-3 * g / (g.abs() + 1e-8), rtol=0, atol=1e-15)
    assert torch.allclose(m1, 0.1 * g, rtol=1e-15, atol=0) and torch.allclose(v1, 1e-3 * g * g, rtol=1e-12, atol=0)


def test_adam_constant_gradient_keeps_the_first_step():
    """With a constant gradient the bias corrections are exact at every step:
    m_t = (1 - beta1^t) g and v_t = (1 - beta2^t) g^2, so every update is the first one."""
    from oracle.classifier import adam_update
    g = torch.tensor([3e-2, -2.5, 7e-9, -1e-3], dtype=torch.float64)
    w = torch.zeros(4, dtype=torch.float64)
    m = torch.zeros(4, dtype=torch.float64)
    v = torch.zeros(4, dtype=torch.float64)
    step = -2e-3 * g / (g.abs() + 1e-8)
    for t in range(1, 30):
        w_new, m, v = adam_update(w, g, m, v, t, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8)
        assert torch.allclose(w_new - w, step, rtol=1e-12, atol=0), t
        w = w_new


def test_adam_matches_torch_optimizer():
    """A sequence of random gradients against torch.optim.Adam in FP64 (an
    independent implementation of the same update)."""
    from oracle.classifier import adam_update
    rng = np.random.default_rng(9)
    w0 = rng.standard_normal(64)
    p = torch.nn.Parameter(torch.from_numpy(w0.copy()))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.85, 0.995), eps=1e-7)
    w = torch.from_numpy(w0.copy())
    m = torch.zeros(64, dtype=torch.float64)
    v = torch.zeros(64, dtype=torch.float64)
    for t in range(1, 12):
        g = torch.from_numpy(rng.standard_normal(64) * 10.0 ** rng.uniform(-4, 1))
        p.grad = g.clone()
        opt.step()
        w, m, v = adam_update(w, g, m, v, t, lr=3e-3, beta1=0.85, beta2=0.995, eps=1e-7)
        assert torch.allclose(w, p.detach(), rtol=0, atol=1e-13), t


def test_dropout_streams_of_a_sub_box_are_those_of_the_whole_grid():
    """A sub-box's masks taken by global cell index equal the whole grid's masks there."""
    D, H, W = 6, 8, 10
    full = oracle.dropout_mask(1, 16, D * H * W, 9, 2, 1, 0.2).reshape(16, D, H, W)
    z, y, x = np.meshgrid(np.arange(1, 4), np.arange(2, 7), np.arange(5, 9), indexing="ij")
    cells = ((z * H + y) * W + x).ravel()
    sub = oracle.dropout_mask(1, 16, cells.size, 9, 2, 1, 0.2, cells=cells).reshape(16, 3, 5, 4)
    assert np.array_equal(sub, full[:, 1:4, 2:7, 5:9])


def test_sub_box_forward_equals_whole_grid_away_from_the_cut():
    """Four 3x3x3 layers see 4 cells deep: a box with a 4-cell margin reproduces
    the whole grid's logits in its interior (same dropout streams)."""
    net = OracleCNN(_weights(6), dropout=0.2, seed=3)
    x = np.random.default_rng(7).standard_normal((1, 6, 12, 16, 14)).astype(np.float32)
    full = net.forward(x, pass_index=1)[0]
    z0, y0, x0 = 2, 3, 1
    box = x[:, :, z0:z0 + 10, y0:y0 + 12, x0:x0 + 11]
    z, y, xx = np.meshgrid(np.arange(z0, z0 + 10), np.arange(y0, y0 + 12), np.arange(x0, x0 + 11), indexing="ij")
    cells = ((z * 16 + y) * 14 + xx).ravel()
    sub = net.forward(box, pass_index=1, cells=cells)[0]
    assert torch.allclose(sub[4:6, 4:8, 4:7], full[z0 + 4:z0 + 6, y0 + 4:y0 + 8, x0 + 4:x0 + 7], rtol=0, atol=1e-12)


def _bf16(a):
    # round to nearest even BF16 through torch's own dtype conversion
    return torch.from_numpy(np.asarray(a, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def _brute_layer(a, W, b):
    """3x3x3 convolution with zero padding by explicit loops over the output
    cells and the taps: a [ci][D][H][W], W [co][ci][3][3][3] -> [co][D][H][W]."""
    ci, D, H, Wd = a.shape
    out = np.zeros((W.shape[0], D, H, Wd))
    for z in range(D):
        for y in range(H):
            for x in range(Wd):
                acc = b.astype(np.float64).copy()
                for kz in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            zz, yy, xx = z + kz - 1, y + ky - 1, x + kx - 1
                            if 0 <= zz < D and 0 <= yy < H and 0 <= xx < Wd:
                                acc += W[:, :, kz, ky, kx] @ a[:, zz, yy, xx]
                out[:, z, y, x] = acc
    return out


@pytest.mark.parametrize("pass_index", [-1, 0])
def test_layer_composition_matches_brute_force(pass_index):
    """The whole 6 -> 32 -> 32 -> 16 -> 1 network on a tiny box, computed here
    by explicit loops (BF16 inputs and weights, ReLU and dropout with inverted
    scaling after each hidden layer, BF16 activations, linear last layer),
    against the oracle's forward pass."""
    weights = _weights(3)
    net = OracleCNN(weights, dropout=0.25, seed=4)
    x = np.random.default_rng(9).standard_normal((1, 6, 3, 4, 5)).astype(np.float32)
    a = _bf16(x[0])
    D, H, Wd = a.shape[1:]
    for l, (W, b) in enumerate(weights):
        z = _brute_layer(a, _bf16(W), b)
        if l == 3:
            ref = z[0]
            break
        h = np.maximum(z, 0.0)
        if pass_index >= 0:
            keep = oracle.dropout_mask(1, h.shape[0], D * H * Wd, 4, pass_index, l, net.p).reshape(h.shape)
            h = h * keep / (1.0 - net.p)
        a = _bf16(h)
    got = net.forward(x, pass_index=pass_index)[0].numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
