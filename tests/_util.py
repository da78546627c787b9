"""Helpers shared by the tests: build-on-demand of the CUDA library, running the
same seeded input through the CUDA path and the oracle, and comparisons."""
import numpy as np
import pytest


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_2510_11174_gb300 import build
    build.build()
    import paper_2510_11174_gb300 as P
    P.load()
    return P


def make_pair(inp, laser=None, tile=8, with_oracle=True):
    """Create a CUDA Simulation and an OracleSim from the same input dict."""
    P = require_gpu()
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g.get("cfl_frac", 0.95),
                       bc=g.get("bc", (0, 0, 0)), laser=laser, tile=tile)
    orc = None
    if with_oracle:
        import oracle.sim as S
        orc = S.OracleSim(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g.get("cfl_frac", 0.95),
                          bc=g.get("bc", (0, 0, 0)), laser=laser)
    for sp in inp.get("species", []):
        sim.load_species(**sp)
        if orc is not None:
            orc.load_species(**sp)
    if "E" in inp:
        sim.set_fields(inp["E"], inp["B"])
        if orc is not None:
            orc.set_fields(inp["E"], inp["B"])
    return sim, orc


def by_id(d):
    order = np.argsort(d["ids"], kind="stable")
    return {k: v[order] for k, v in d.items()}


def seeded_classifier(P, seed, out_bias=0.0, **kw):
    """A GPU Classifier holding seeded weights (inputs.classifier_weights) and
    those weights, so that the oracle takes the same inputs and none of its
    inputs comes from the CUDA path."""
    from paper_2510_11174_gb300 import inputs
    from paper_2510_11174_gb300.model import Classifier
    weights = inputs.classifier_weights(seed, out_bias=out_bias)
    m = Classifier(seed=seed, **kw)
    for l, (w, b) in enumerate(weights):
        m.set_layer(l, w, b)
    return m, weights
