"""SwitchNet on the GPU (hyb_switchnet_*: tcgen05 dense layers) against the
oracle: logits with and without dropout on a ragged number of cells, the
MC-dropout statistics, one step's gradients, three Adam steps, a falling
loss, and the rejection of an empty input."""
import numpy as np
import pytest
import torch

from _util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _features(n, seed):
    rng = np.random.default_rng(seed)
    mean = (0.3 * rng.standard_normal(10)).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 10).astype(np.float32)
    x = (mean[:, None] + std[:, None] * rng.standard_normal((10, n))).astype(np.float32)
    return x, mean, std


def _pair(seed=5, dropout=0.2, mc_passes=4, mean=None, std=None):
    P = require_gpu()
    from oracle import switchnet as S
    from paper_2510_11174_gb300 import inputs
    from paper_2510_11174_gb300.model import SwitchNet
    w = inputs.switchnet_weights(seed)
    m = SwitchNet(dropout=dropout, mc_passes=mc_passes, seed=seed, mean=mean, std=std)
    for l, (a, b) in enumerate(w):
        m.set_layer(l, a, b)
    return m, S.OracleSwitchNet(w, dropout=dropout, seed=seed, mean=mean, std=std), w


@pytest.mark.parametrize("pass_index", [-1, 3])
def test_forward_matches_oracle(pass_index):
    x, mean, std = _features(5000, 1)
    m, orc, _ = _pair(mean=mean, std=std)
    lg = m.forward(torch.from_numpy(x).cuda(), pass_index).cpu().numpy()
    ref = orc.forward(x, pass_index).numpy()
    assert rel_l2(lg, ref) <= 2e-3, rel_l2(lg, ref)
    m.close()


def test_mc_statistics_match_oracle():
    x, mean, std = _features(3000, 2)
    m, orc, _ = _pair(mean=mean, std=std, mc_passes=4)
    pm, ps = m.mc(torch.from_numpy(x).cuda())
    om, os_ = orc.mc_statistics(x, 4)
    assert rel_l2(pm.cpu().numpy(), om.numpy()) <= 2e-3
    assert rel_l2(ps.cpu().numpy(), os_.numpy()) <= 5e-2
    m.close()


def test_one_step_gradients_match_oracle():
    from oracle import switchnet as S
    x, mean, std = _features(6000, 3)
    y = (np.abs(x[1]) > 1.0).astype(np.float32)
    m, orc, _ = _pair(mean=mean, std=std)
    st = m.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    ref = S.loss_and_grads(orc, x, y, 0)
    assert st["loss"] == pytest.approx(ref["loss"], rel=2e-3)
    errs = []
    for l in range(5):
        gw, gb = m.get_grad(l)
        errs.append((rel_l2(gw, ref["grads"][l][0].numpy()), rel_l2(gb, ref["grads"][l][1].numpy())))
    assert all(ew <= 1e-2 and eb <= 1e-2 for ew, eb in errs), errs
    m.close()


def test_three_adam_steps_match_oracle():
    from oracle import switchnet as S
    x, mean, std = _features(4000, 4)
    y = (np.abs(x[1]) > 1.0).astype(np.float32)
    m, _, w = _pair(mean=mean, std=std)
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for _ in range(3):
        m.train_step(xs, ys)
    hist, _ = S.train_run(w, x, y, 3, dropout=0.2, seed=5, mean=mean, std=std)
    for l in range(5):
        gw, _ = m.get_layer(l)
        ow, _ = hist[-1][l]
        dw = np.abs((gw - w[l][0]) - (ow.numpy() - w[l][0])) / 1e-3
        assert np.median(dw) <= 2e-2 and np.quantile(dw, 0.99) <= 0.3, (l, np.median(dw), np.quantile(dw, 0.99))
    m.close()


def test_training_lowers_the_loss_and_empty_input_is_rejected():
    from paper_2510_11174_gb300._abi import HybError, HYB_EINVAL
    x, mean, std = _features(20000, 6)
    y = ((x[1] - mean[1]) ** 2 + (x[5] - mean[5]) ** 2 > 2.0 * std[1] * std[5]).astype(np.float32)
    m, _, _ = _pair(mean=mean, std=std)
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    st = [m.train_step(xs, ys) for _ in range(150)]
    assert st[-1]["loss"] < 0.7 * st[0]["loss"] and st[-1]["accuracy"] > 0.85, (st[0], st[-1])
    with pytest.raises(HybError) as ei:
        m.forward(torch.zeros((10, 0), device="cuda"))
    assert ei.value.code == HYB_EINVAL
    m.close()
