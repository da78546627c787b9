"""GPU regime classifier (tensor-core convolutions) against the FP64 oracle on
the same BF16-rounded weights and inputs (rel-L2 <= 1e-3), the 1x1x1
special case against torch.matmul, and classification of a context's fields
with MC dropout."""
import math

import numpy as np
import pytest

from _util import require_gpu, rel_l2

pytestmark = pytest.mark.gpu


def _model(P, dropout=0.2, seed=7, mean=None, std=None):
    """A GPU classifier with seeded weights and the oracle network of the same weights."""
    from oracle.classifier import OracleCNN
    from _util import seeded_classifier
    m, weights = seeded_classifier(P, seed, dropout=dropout, mc_passes=4, mean=mean, std=std)
    return m, OracleCNN(weights, dropout=dropout, seed=seed, mean=mean, std=std)


@pytest.mark.parametrize("shape", [(2, 16, 16, 16), (1, 3, 32, 24), (1, 1, 16, 8)])
@pytest.mark.parametrize("pass_index", [-1, 3])
def test_forward_matches_oracle(shape, pass_index):
    P = require_gpu()
    import torch
    B, D, H, W = shape
    mean = [0.1, -0.2, 0.0, 0.05, 0.0, -0.1]
    std = [0.5, 1.0, 2.0, 0.7, 1.5, 0.9]
    m, net = _model(P, mean=mean, std=std)
    x = np.random.default_rng(3).standard_normal((B, 6, D, H, W)).astype(np.float32)
    y = m.forward(torch.from_numpy(x).cuda(), pass_index).cpu().numpy()
    ref = net.forward(x, pass_index).numpy()
    assert rel_l2(y, ref) <= 1e-3, rel_l2(y, ref)


def test_center_tap_network_is_a_gemm_chain():
    """With only the centre tap non-zero every layer is a per-cell GEMM:
    compare against torch.matmul in FP32 on the same BF16-rounded operands."""
    P = require_gpu()
    import torch
    m, _ = _model(P, dropout=0.0)
    rng = np.random.default_rng(5)
    mats = []
    for l, (ci, co) in enumerate([(6, 32), (32, 32), (32, 16), (16, 1)]):
        w = np.zeros((co, ci, 3, 3, 3), np.float32)
        w[:, :, 1, 1, 1] = rng.standard_normal((co, ci)) / math.sqrt(ci)
        b = (0.1 * rng.standard_normal(co)).astype(np.float32)
        m.set_layer(l, w, b)
        mats.append((w[:, :, 1, 1, 1], b))
    x = rng.standard_normal((1, 6, 2, 16, 8)).astype(np.float32)
    y = m.forward(torch.from_numpy(x).cuda(), -1).cpu().numpy()
    bf = lambda t: t.to(torch.bfloat16).to(torch.float32)
    a = bf(torch.from_numpy(x).cuda().permute(0, 2, 3, 4, 1).reshape(-1, 6))
    for l, (w, b) in enumerate(mats):
        z = torch.matmul(a, bf(torch.from_numpy(w).cuda()).t()) + torch.from_numpy(b).cuda()
        a = bf(torch.relu(z)) if l < 3 else z
    ref = a.reshape(1, 2, 16, 8).cpu().numpy()
    assert rel_l2(y, ref) <= 1e-5, rel_l2(y, ref)


def test_classify_context_fields_with_mc_dropout():
    P = require_gpu()
    import torch
    from _util import make_pair
    nx, ny, nz = 16, 16, 8
    rng = np.random.default_rng(9)
    E = (0.5 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    B = (0.5 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    sim, _ = make_pair(dict(grid=dict(nx=nx, ny=ny, nz=nz, dx=0.3), E=E, B=B), with_oracle=False)
    m, net = _model(P, dropout=0.2, seed=13)
    pm = torch.empty(nz * ny * nx, device="cuda")
    ps = torch.empty(nz * ny * nx, device="cuda")
    sim.classify(m, pm, ps)
    # the same node fields in numpy (E averaged from its two edges, B from its four faces, periodic)
    r = lambda a, s, ax: np.roll(a, s, axis=ax)
    f = np.stack([0.5 * (E[0] + r(E[0], 1, 2)), 0.5 * (E[1] + r(E[1], 1, 1)), 0.5 * (E[2] + r(E[2], 1, 0)),
                  0.25 * (B[0] + r(B[0], 1, 1) + r(B[0], 1, 0) + r(r(B[0], 1, 1), 1, 0)),
                  0.25 * (B[1] + r(B[1], 1, 2) + r(B[1], 1, 0) + r(r(B[1], 1, 2), 1, 0)),
                  0.25 * (B[2] + r(B[2], 1, 2) + r(B[2], 1, 1) + r(r(B[2], 1, 2), 1, 1))])[None].astype(np.float32)
    om, os_ = net.mc_statistics(f, 4)
    assert rel_l2(pm.cpu().numpy(), om.numpy().ravel()) <= 1e-3
    assert np.max(np.abs(ps.cpu().numpy() - os_.numpy().ravel())) <= 2e-3
