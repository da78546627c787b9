"""Pins of the surrogate oracle (oracle/surrogate.py) that do not come from
the oracle itself: with every weight zero the residual forecast is the input
state (persistence); a choice of weights for which the network's output is
its normalised input (zero kernels on the shortcut layers, centre-tap +/-
identities on the others), so the prediction is x + std (x - mean) / std =
2 x - mean, with no spread over MC-dropout passes; a zero loss for a perfect
prediction and the Huber closed form for an offset; the backward pass
against FP64 central differences; and the node state's charge against the
particles' total charge."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import surrogate as S


def _identity_weights():
    """Layers 0..2 zero (their shortcuts carry the input), layer 3 splits
    every channel into its positive and negative part (centre tap +1 / -1),
    layer 4 passes both on, layer 5 subtracts them: y = x_hat."""
    w = [np.zeros((co, ci, 3, 3, 3), np.float32) for ci, co in S.LAYERS]
    b = [np.zeros(co, np.float32) for _, co in S.LAYERS]
    for c in range(10):
        w[3][c, c, 1, 1, 1] = 1.0
        w[3][10 + c, c, 1, 1, 1] = -1.0
        w[4][c, c, 1, 1, 1] = 1.0
        w[4][10 + c, 10 + c, 1, 1, 1] = 1.0
        w[5][c, c, 1, 1, 1] = 1.0
        w[5][c, 10 + c, 1, 1, 1] = -1.0
    return list(zip(w, b))


def _states(B=2, n=6, seed=1):
    rng = np.random.default_rng(seed)
    mean = rng.normal(0, 0.5, 10).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 10).astype(np.float32)
    x = (mean[None, :, None, None, None] + std[None, :, None, None, None] *
         rng.standard_normal((B, 10, n, n, n))).astype(np.float32)
    return x, mean, std


def test_zero_weights_forecast_persistence():
    x, mean, std = _states()
    zero = [(np.zeros((co, ci, 3, 3, 3), np.float32), np.zeros(co, np.float32)) for ci, co in S.LAYERS]
    net = S.OracleSurrogate(zero, mean=mean, std=std)
    np.testing.assert_array_equal(net.predict(x).numpy(), x.astype(np.float64))
    m, s = net.mc_statistics(x, 3)
    np.testing.assert_array_equal(m.numpy(), x.astype(np.float64))
    assert float(s.abs().max()) == 0.0


def test_identity_weights_give_twice_the_state_less_the_mean():
    x, mean, std = _states()
    net = S.OracleSurrogate(_identity_weights(), mean=mean, std=std)
    target = 2.0 * x.astype(np.float64) - mean[None, :, None, None, None]
    exact = net.predict(x, exact=True).numpy()
    np.testing.assert_allclose(exact, target, rtol=0, atol=1e-5)
    # BF16 rounding of the normalised input (8 significant bits): |error| <= 2^-8 |x_hat| std
    rounded = net.predict(x).numpy()
    xh = (x - mean[None, :, None, None, None]) / std[None, :, None, None, None]
    bound = 2.0 ** -8 * np.abs(xh) * std[None, :, None, None, None] + 1e-5
    assert np.all(np.abs(rounded - target) <= bound)


def test_identity_weights_have_no_mc_spread():
    x, mean, std = _states(seed=2)
    net = S.OracleSurrogate(_identity_weights(), dropout=0.1, mean=mean, std=std)
    m, s = net.mc_statistics(x, 4)
    np.testing.assert_array_equal(m.numpy(), net.predict(x).numpy())
    assert float(s.abs().max()) == 0.0


def test_change_unit_scales_the_forecast_change():
    x, mean, std = _states(seed=7)
    dstd = (0.25 + np.arange(10)).astype(np.float32)
    net = S.OracleSurrogate(_identity_weights(), mean=mean, std=std, dstd=dstd)
    xh = (x - mean[None, :, None, None, None]) / std[None, :, None, None, None]
    target = x.astype(np.float64) + dstd[None, :, None, None, None] * xh
    np.testing.assert_allclose(net.predict(x, exact=True).numpy(), target, rtol=0, atol=1e-4)


def test_loss_of_a_perfect_prediction_is_zero_and_huber_of_an_offset():
    x, mean, std = _states(seed=3)
    net = S.OracleSurrogate(_identity_weights(), mean=mean, std=std)
    # zero up to the FP32 rounding of the normalisation (the target change is
    # formed in FP32, the prediction in FP64)
    t = net.predict(x, exact=True).numpy().astype(np.float32)
    out = S.loss_and_grads(net, x, t, -1, exact=True)
    assert out["loss"] == pytest.approx(0.0, abs=1e-10)
    for gw, gb in out["grads"]:
        assert float(gw.abs().max()) < 1e-6 and float(gb.abs().max()) < 1e-6
    # channel 9 (rho, outside the energy) off by c in normalised units: every
    # value of that channel contributes delta (|c| - delta / 2) (|c| > delta)
    # or c^2 / 2 (|c| <= delta)
    for c, delta in ((0.3, 0.01), (0.004, 0.01)):
        tc = t.copy()
        tc[:, 9] -= c * std[9]
        out = S.loss_and_grads(net, x, tc, -1, delta=delta, exact=True)
        per = delta * (c - 0.5 * delta) if c > delta else 0.5 * c * c
        # (the offset is applied in FP32 to values of order 1: rel 1e-3)
        assert out["huber"] == pytest.approx(per / 10.0, rel=1e-3)
        assert out["energy"] == pytest.approx(0.0, abs=1e-10)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(4)
    weights = []
    for ci, co in S.LAYERS:
        lim = math.sqrt(6.0 / (27 * ci))
        weights.append((rng.uniform(-lim, lim, (co, ci, 3, 3, 3)).astype(np.float32),
                        rng.uniform(-0.1, 0.1, co).astype(np.float32)))
    x, mean, std = _states(B=2, n=4, seed=5)
    t = x + 0.3 * rng.standard_normal(x.shape).astype(np.float32) * std[None, :, None, None, None]
    net = S.OracleSurrogate(weights, dropout=0.1, mean=mean, std=std)
    out = S.loss_and_grads(net, x, t, 3, delta=0.01, energy_weight=0.1, exact=True)
    h = 1e-6
    for l in range(len(S.LAYERS)):
        gw, gb = out["grads"][l]
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in net.W[l].shape)
            w0 = net.W[l][idx].item()
            net.W[l][idx] = w0 + h
            lp = S.loss_and_grads(net, x, t, 3, exact=True)["loss"]
            net.W[l][idx] = w0 - h
            lm = S.loss_and_grads(net, x, t, 3, exact=True)["loss"]
            net.W[l][idx] = w0
            fd = (lp - lm) / (2 * h)
            assert gw[idx].item() == pytest.approx(fd, rel=1e-5, abs=1e-10), (l, idx)
        c = int(rng.integers(0, net.b[l].shape[0]))
        b0 = net.b[l][c].item()
        net.b[l][c] = b0 + h
        lp = S.loss_and_grads(net, x, t, 3, exact=True)["loss"]
        net.b[l][c] = b0 - h
        lm = S.loss_and_grads(net, x, t, 3, exact=True)["loss"]
        net.b[l][c] = b0
        assert gb[c].item() == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-10), (l, c)


def test_node_state_charge_sums_to_the_particle_charge():
    g = oracle.Grid.make(6, 5, 4, 0.5, 0.5, 0.5, 0.2, bc=(0, 0, 0))
    rng = np.random.default_rng(6)
    n = 50
    sp = dict(x=rng.uniform(0, 6, n), y=rng.uniform(0, 5, n), z=rng.uniform(0, 4, n), ux=np.zeros(n), uy=np.zeros(n),
              uz=np.zeros(n), w=rng.uniform(0.5, 1.5, n), zq=rng.integers(1, 4, n).astype(np.float64))
    fl_n = rng.uniform(0, 1, g.shape)
    zero = np.zeros((3,) + g.shape)
    st = S.node_state(g, zero, zero, zero, species=[(1.0, 1836.0, sp)], fluids=[(-1.0, fl_n)])
    total = st[9].sum() * 0.5 ** 3
    expect = float(np.sum(sp["w"] * sp["zq"])) - fl_n.sum() * 0.5 ** 3
    assert total == pytest.approx(expect, rel=1e-12)


def _bf16(a):
    # round to nearest even BF16 through torch's own dtype conversion
    return torch.from_numpy(np.asarray(a, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def _brute_conv(a, W, b):
    """3x3x3 cross-correlation with zero padding by explicit loops over the
    output cells and taps: a [ci][D][H][W] -> [co][D][H][W]."""
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


@pytest.mark.parametrize("pass_index", [-1, 1])
def test_layer_composition_matches_brute_force(pass_index):
    """The six layers on a tiny box by explicit loops (identity shortcuts on
    layers 0..2 with the extra channels zero, ReLU on 0..4, dropout with
    inverted scaling after layer 1, BF16 activations between layers, a linear
    last layer, the forecast added to the input) against the oracle."""
    rng = np.random.default_rng(12)
    weights = [((rng.standard_normal((co, ci, 3, 3, 3)) / np.sqrt(27 * ci)).astype(np.float32),
                (0.05 * rng.standard_normal(co)).astype(np.float32)) for ci, co in S.LAYERS]
    net = S.OracleSurrogate(weights, dropout=0.25, seed=13)
    x = rng.standard_normal((1, 10, 2, 3, 4)).astype(np.float32)
    a = _bf16(x[0])
    D, H, Wd = a.shape[1:]
    for l, (W, b) in enumerate(weights):
        co = W.shape[0]
        h = _brute_conv(a, _bf16(W), b)
        if l < 5:
            h = np.maximum(h, 0.0)
        if l == 1 and pass_index >= 0:
            keep = oracle.dropout_mask(1, (co + 7) // 8 * 8, D * H * Wd, 13, pass_index, 1, net.p)
            h = h * keep.reshape(-1, D, H, Wd)[:co] / (1.0 - net.p)
        if l < 3:
            pad = np.zeros_like(h)
            pad[:a.shape[0]] = a
            h = h + pad
        a = h if l == 5 else _bf16(h)
    pred = net.predict(x, pass_index=pass_index)[0].numpy()
    assert np.allclose(pred, x[0].astype(np.float64) + a, rtol=1e-12, atol=1e-12)
