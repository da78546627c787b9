"""The field surrogate on the GPU (hyb_surrogate_*, tcgen05 convolutions in
channel chunks) against the oracle: the identity-map weights forecast
2 x - mean; forward passes with and without dropout, the MC-dropout statistics,
one step's gradients and three Adam steps on seeded weights and states; the
ten-channel node state of a hybrid run; and a falling loss."""
import numpy as np
import pytest
import torch

from _util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _pair(seed=3, dropout=0.1, mc_passes=4, mean=None, std=None, weights=None, dstd=None):
    P = require_gpu()
    from oracle import surrogate as S
    from paper_2510_11174_gb300 import inputs
    from paper_2510_11174_gb300.model import Surrogate
    weights = inputs.surrogate_weights(seed) if weights is None else weights
    m = Surrogate(dropout=dropout, mc_passes=mc_passes, seed=seed, mean=mean, std=std, dstd=dstd)
    for l, (w, b) in enumerate(weights):
        m.set_layer(l, w, b)
    return m, S.OracleSurrogate(weights, dropout=dropout, seed=seed, mean=mean, std=std, dstd=dstd), weights


def _identity_weights():
    from paper_2510_11174_gb300 import inputs
    w = [np.zeros((co, ci, 3, 3, 3), np.float32) for ci, co in inputs.SURROGATE_LAYERS]
    b = [np.zeros(co, np.float32) for _, co in inputs.SURROGATE_LAYERS]
    for c in range(10):
        w[3][c, c, 1, 1, 1] = 1.0
        w[3][10 + c, c, 1, 1, 1] = -1.0
        w[4][c, c, 1, 1, 1] = 1.0
        w[4][10 + c, 10 + c, 1, 1, 1] = 1.0
        w[5][c, c, 1, 1, 1] = 1.0
        w[5][c, 10 + c, 1, 1, 1] = -1.0
    return list(zip(w, b))


def test_identity_weights_give_twice_the_state_less_the_mean():
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(2, 16, seed=1)
    m, orc, _ = _pair(mean=mean, std=std, weights=_identity_weights())
    y = m.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = orc.predict(x).numpy()
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-5)
    xh = (x - mean[None, :, None, None, None]) / std[None, :, None, None, None]
    target = 2.0 * x - mean[None, :, None, None, None]
    assert np.all(np.abs(y - target) <= 2.0 ** -8 * np.abs(xh) * std[None, :, None, None, None] + 1e-5)
    m.close()


@pytest.mark.parametrize("pass_index", [-1, 5])
def test_forward_matches_oracle(pass_index):
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(2, 16, seed=2)
    m, orc, _ = _pair(mean=mean, std=std)
    y = m.forward(torch.from_numpy(x).cuda(), pass_index).cpu().numpy()
    ref = orc.predict(x, pass_index).numpy()
    err = rel_l2(y - x, ref - x)   # the predicted change
    assert err <= 1e-3, err        # measured 4e-4 .. 6e-4
    m.close()


def test_forward_with_a_change_unit_matches_oracle():
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(2, 16, seed=12)
    dstd = (0.05 * std).astype(np.float32)
    m, orc, _ = _pair(mean=mean, std=std, dstd=dstd)
    y = m.forward(torch.from_numpy(x).cuda(), 2).cpu().numpy()
    ref = orc.predict(x, 2).numpy()
    assert rel_l2(y - x, ref - x) <= 1e-3, rel_l2(y - x, ref - x)
    m.close()


def test_mc_statistics_match_oracle():
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(1, 16, seed=4)
    m, orc, _ = _pair(mean=mean, std=std, mc_passes=4)
    pm, ps = m.mc(torch.from_numpy(x).cuda())
    om, os_ = orc.mc_statistics(x, 4)
    assert rel_l2(pm.cpu().numpy() - x, om.numpy() - x) <= 2e-3
    assert float(ps.min()) >= 0.0
    assert rel_l2(ps.cpu().numpy(), os_.numpy()) <= 2e-2
    m.close()


def test_one_step_gradients_match_oracle():
    from oracle import surrogate as S
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(2, 16, seed=6)
    t = x + (0.2 * np.random.default_rng(7).standard_normal(x.shape) * std[None, :, None, None, None]).astype(np.float32)
    m, orc, _ = _pair(mean=mean, std=std)
    st = m.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    ref = S.loss_and_grads(orc, x, t, 0)
    assert st["loss"] == pytest.approx(ref["loss"], rel=2e-3)
    errs = []
    for l in range(6):
        gw, gb = m.get_grad(l)
        ow, ob = ref["grads"][l]
        errs.append((rel_l2(gw, ow.numpy()), rel_l2(gb, ob.numpy())))
    # BF16 flips between the FP32 and FP64 sums collect in the first layer's
    # weight gradient (measured 4.5e-3 .. 4.8e-3; the other layers 6e-5 .. 1.2e-3)
    assert errs[0][0] <= 1e-2 and all(ew <= 2.5e-3 for ew, _ in errs[1:]), errs
    assert all(eb <= 1e-3 for _, eb in errs), errs
    m.close()


def test_three_adam_steps_match_oracle():
    from oracle import surrogate as S
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(2, 16, seed=8)
    t = x + (0.2 * np.random.default_rng(9).standard_normal(x.shape) * std[None, :, None, None, None]).astype(np.float32)
    m, _, weights = _pair(mean=mean, std=std)
    xs, ts = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    for _ in range(3):
        m.train_step(xs, ts)
    hist, _ = S.train_run(weights, x, t, 3, dropout=0.1, seed=3, mean=mean, std=std)
    lr = 1e-3
    for l in range(6):
        w, b = m.get_layer(l)
        ow, ob = hist[-1][l]
        w0, b0 = weights[l]
        # Adam moves a weight by about lr per step: compare the moves, relative to lr
        dw = np.abs((w - w0) - (ow.numpy() - w0)) / lr
        assert np.median(dw) <= 2e-2 and np.quantile(dw, 0.99) <= 0.3, (l, np.median(dw), np.quantile(dw, 0.99))
    m.close()


def test_node_state_matches_oracle():
    P = require_gpu()
    from oracle import surrogate as S
    import oracle
    import oracle.sim as OS
    from paper_2510_11174_gb300 import inputs
    inp = inputs.ramp_slab(nx=64, ny=32, nz=32, a0=20.0, ppc=4, tile_capacity=4 * 512 * 4, vacuum_lambda=0.5,
                           slab_lambda=1.0, seed=5)
    inp["laser"]["t_peak"] = inp["laser"]["tau_fwhm"]
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"])
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=2, ppc=4, to_species=[0, 1])
    sim.step(30)
    sim.classify()
    sim.step(3)
    st = sim.node_state().cpu().numpy()
    E, B, J = sim.get_fields()
    d = sim.desc
    og = oracle.Grid.make(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, OS.courant_dt((d.dx, d.dy, d.dz), d.cfl_frac),
                          bc=tuple(d.bc))
    sps = [(-1.0, 1.0, sim.get_species(0)), (1.0, inputs.M_P, sim.get_species(1))]
    assert len(sps[0][2]["x"]) > 0
    fls = [(-1.0, sim.get_fluid(0)["n"]), (1.0, sim.get_fluid(1)["n"])]
    _, rho_bg = sim.get_regime()
    ref = S.node_state(og, E.astype(np.float64), B.astype(np.float64), J.astype(np.float64), sps, fls, rho_bg)
    for c in range(9):
        scale = max(float(np.abs(ref[c]).max()), 1e-30)
        assert np.max(np.abs(st[c] - ref[c])) <= 1e-6 * scale, c
    assert np.max(np.abs(st[9] - ref[9])) <= 1e-5 * float(np.abs(ref[9]).max())
    sim.close()


def test_training_lowers_the_loss():
    from paper_2510_11174_gb300 import inputs
    x, mean, std = inputs.random_states(4, 16, seed=10)
    # a smooth target: the state shifted by one cell along x
    t = np.roll(x, 1, axis=4)
    m, _, _ = _pair(mean=mean, std=std)
    xs, ts = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = [m.train_step(xs, ts)["loss"] for _ in range(60)]
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    m.close()
