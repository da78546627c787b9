"""Training data for the regime classifier from the method's own runs, and a
training loop on it (paper, Methodology: the networks learn from data the
simulation generates, the regime labels from the instability criterion the
method uses; Results: training over epochs with a decreasing loss).

``generate_patches`` runs ramp + slab hybrid simulations (the physics
criterion decides the regime, fluid and particles are converted as the
method does) with seeded pulse amplitudes (log-uniform) and densities
(log-uniform), and at every classification cuts random 32^3 patches of the
six node-field channels (``hyb_node_fields``).  A patch's label at a node is
the criterion's decision there now or at the next classification ("kinetic
now or soon"), so a network that learns it flags cells before the pulse
reaches them.  ``train`` runs ``hyb_train_step`` over shuffled batches.

``generate_state_pairs`` cuts the field surrogate's data from the same runs:
16^3 patches of the ten node channels (``hyb_node_state``: E, B, J, rho) at
one step and at the same place ``lead`` steps later (Results: the predictor
learns state transitions).  ``train_surrogate`` runs
``hyb_surrogate_train_step`` over shuffled batches and ``r2_mse`` scores a
prediction per channel (Results: R^2 and MSE per channel).

``generate_snapshots`` keeps whole grids instead (the six classifier
channels, the ten node channels and the lookahead label), so that the
convolutional classifier and the per-cell SwitchNet learn from the same runs
and are scored on the same held-out cells by ``auc`` (Results: SwitchNet's
AUC).

Orchestration only: the runs, the node fields and every training step run in
libhyb.so; torch indexing cuts the patches and stacks the batches.
"""
import math

import numpy as np

from . import inputs


def _run(P, nx, ny, nz, a0, dens, seed, stream, tau_fs=12.0):
    inp = inputs.ramp_slab(nx=nx, ny=ny, nz=nz, n_lo=0.01 * dens, n_hi=dens, n_slab=5.0 * dens, a0=a0,
                           tau_fs=tau_fs, vacuum_lambda=0.5, slab_lambda=1.0, ppc=4, tile_capacity=4 * 512 * 8,
                           seed=seed)
    inp["laser"]["t_peak"] = inp["laser"]["tau_fwhm"]
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"],
                       stream=stream, seed=seed)
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=2, ppc=4, to_species=[0, 1], quiet=True)
    return sim


def generate_patches(n_patches=4096, grid=(128, 128, 64), patch=32, runs=8, classifications=16, every=10,
                     a0_range=(10.0, 300.0), density_range=(0.2, 2.0), seed=11, stream=None):
    """(x [n, 6, p, p, p], y [n, p, p, p]) as torch CUDA tensors (FP32)."""
    import torch
    import paper_2510_11174_gb300 as P
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    per_snap = int(math.ceil(n_patches / (runs * (classifications - 1))))
    xs, ys = [], []
    st = stream if stream is not None else torch.cuda.Stream()
    for r in range(runs):
        a0 = float(np.exp(rng.uniform(math.log(a0_range[0]), math.log(a0_range[1]))))
        dens = float(np.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1]))))
        sim = _run(P, nx, ny, nz, a0, dens, seed + r, st.cuda_stream)
        snaps, masks = [], []
        for c in range(classifications):
            snaps.append(sim.node_fields())
            sim.classify()
            masks.append(torch.from_numpy(sim.get_regime()[0]).cuda())
            sim.step(every)
        sim.close()
        for c in range(classifications - 1):
            label = (masks[c] | masks[c + 1]).float()
            for _ in range(per_snap):
                z0, y0, x0 = (int(rng.integers(0, n - patch + 1)) for n in (nz, ny, nx))
                xs.append(snaps[c][:, z0:z0 + patch, y0:y0 + patch, x0:x0 + patch])
                ys.append(label[z0:z0 + patch, y0:y0 + patch, x0:x0 + patch])
    x = torch.stack(xs[:n_patches]).contiguous()
    y = torch.stack(ys[:n_patches]).contiguous()
    return x, y


def channel_stats(x):
    """Per-channel mean and standard deviation of the patches (the
    classifier's input normalisation)."""
    m = x.mean(dim=(0, 2, 3, 4))
    s = x.std(dim=(0, 2, 3, 4)).clamp_min(1e-6)
    return [float(v) for v in m], [float(v) for v in s]


def train(model, x, y, steps, batch=32, seed=5, log_every=0):
    """`steps` training steps on shuffled batches; returns the list of step statistics."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    perm = torch.randperm(n, generator=gen)
    pos = 0
    stats = []
    for k in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=gen)
            pos = 0
        idx = perm[pos:pos + batch].cuda()
        pos += batch
        st = model.train_step(x.index_select(0, idx), y.index_select(0, idx))
        stats.append(st)
        if log_every and (k + 1) % log_every == 0:
            print("step %d loss %.4f acc %.3f" % (k + 1, st["loss"], st["accuracy"]))
    return stats


def generate_state_pairs(n_pairs=2048, grid=(128, 128, 64), patch=16, runs=8, snapshots=12, every=5, lead=2,
                         a0_range=(10.0, 300.0), density_range=(0.2, 2.0), seed=13, stream=None, focus=0.5):
    """(x, t) torch CUDA tensors [n, 10, p, p, p]: states and the states `lead`
    steps later at the same patches, from ramp + slab hybrid runs.  A fraction
    `focus` of the patches is centred on cells where the field energy density
    is in the top 1 % of the snapshot (where the pulse acts on the plasma),
    the rest is placed uniformly."""
    import torch
    import paper_2510_11174_gb300 as P
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    per_snap = int(math.ceil(n_pairs / (runs * snapshots)))
    xs, ts = [], []
    st = stream if stream is not None else torch.cuda.Stream()
    for r in range(runs):
        a0 = float(np.exp(rng.uniform(math.log(a0_range[0]), math.log(a0_range[1]))))
        dens = float(np.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1]))))
        sim = _run(P, nx, ny, nz, a0, dens, seed + r, st.cuda_stream)
        sim.classify()
        for c in range(snapshots):
            sim.step(every)
            if c % 2 == 1:
                sim.classify()
            s0 = sim.node_state()
            sim.step(lead)
            s1 = sim.node_state()
            e = (s0[:6] ** 2).sum(0).reshape(-1)
            hot = torch.nonzero(e >= torch.quantile(e[::97], 0.99)).reshape(-1).cpu().numpy()
            for _ in range(per_snap):
                if len(hot) and rng.random() < focus:
                    c = int(hot[int(rng.integers(0, len(hot)))])
                    cz, cy, cx = c // (nx * ny), (c // nx) % ny, c % nx
                    z0, y0, x0 = (min(max(v - patch // 2, 0), n - patch) for v, n in ((cz, nz), (cy, ny), (cx, nx)))
                else:
                    z0, y0, x0 = (int(rng.integers(0, n - patch + 1)) for n in (nz, ny, nx))
                xs.append(s0[:, z0:z0 + patch, y0:y0 + patch, x0:x0 + patch])
                ts.append(s1[:, z0:z0 + patch, y0:y0 + patch, x0:x0 + patch])
        sim.close()
    return torch.stack(xs[:n_pairs]).contiguous(), torch.stack(ts[:n_pairs]).contiguous()


def train_surrogate(model, x, t, steps, batch=32, seed=5):
    """`steps` surrogate training steps on shuffled batches; returns the step statistics."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    perm = torch.randperm(n, generator=gen)
    pos = 0
    stats = []
    for _ in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=gen)
            pos = 0
        idx = perm[pos:pos + batch].cuda()
        pos += batch
        stats.append(model.train_step(x.index_select(0, idx), t.index_select(0, idx)))
    return stats


def r2_mse(pred, target, mean, std):
    """Per-channel R^2 and MSE of a prediction, both on the normalised values
    (x - mean_c) / std_c: R^2 = 1 - SS_res / SS_tot about the target's mean."""
    import torch
    mu = torch.tensor(mean, device=pred.device).view(1, -1, 1, 1, 1)
    sd = torch.tensor(std, device=pred.device).view(1, -1, 1, 1, 1)
    p = ((pred - mu) / sd).double()
    q = ((target - mu) / sd).double()
    res = ((p - q) ** 2).sum(dim=(0, 2, 3, 4))
    tot = ((q - q.mean(dim=(0, 2, 3, 4), keepdim=True)) ** 2).sum(dim=(0, 2, 3, 4))
    n = q.numel() / q.shape[1]
    r2 = 1.0 - res / tot.clamp_min(1e-300)
    return [float(v) for v in r2], [float(v) for v in res / n]


def generate_snapshots(grid=(128, 128, 64), runs=6, classifications=9, every=10, a0_range=(10.0, 300.0),
                       density_range=(0.2, 2.0), seed=21, stream=None):
    """List of (fields6 [6, nz, ny, nx], state10 [10, nz, ny, nx], label [nz, ny, nx])
    torch CUDA tensors per run and classification: the label is the physics
    criterion now or at the next classification."""
    import torch
    import paper_2510_11174_gb300 as P
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    out = []
    st = stream if stream is not None else torch.cuda.Stream()
    for r in range(runs):
        a0 = float(np.exp(rng.uniform(math.log(a0_range[0]), math.log(a0_range[1]))))
        dens = float(np.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1]))))
        sim = _run(P, nx, ny, nz, a0, dens, seed + r, st.cuda_stream)
        snaps, masks = [], []
        for c in range(classifications):
            snaps.append((sim.node_fields(), sim.node_state()))
            sim.classify()
            masks.append(torch.from_numpy(sim.get_regime()[0]).cuda())
            sim.step(every)
        sim.close()
        for c in range(classifications - 1):
            out.append((snaps[c][0], snaps[c][1], (masks[c] | masks[c + 1]).float()))
    return out


def auc(score, label):
    """Area under the ROC curve (the probability that a random kinetic cell
    scores above a random fluid cell, ties one half), from the ranks of the
    scores (Mann-Whitney U); torch tensors on any device."""
    import torch
    s = score.reshape(-1).double()
    y = label.reshape(-1) > 0.5
    npos, nneg = int(y.sum()), int((~y).sum())
    if npos == 0 or nneg == 0:
        return float("nan")
    order = torch.argsort(s, stable=True)
    ss = s[order]
    pos = torch.arange(1, len(ss) + 1, device=s.device, dtype=torch.float64)
    # tied scores share the mean of their positions
    new = torch.ones(len(ss), dtype=torch.bool, device=s.device)
    new[1:] = ss[1:] != ss[:-1]
    gid = torch.cumsum(new.long(), 0) - 1
    ng = int(gid[-1]) + 1
    sums = torch.zeros(ng, dtype=torch.float64, device=s.device).index_add_(0, gid, pos)
    cnt = torch.zeros(ng, dtype=torch.float64, device=s.device).index_add_(0, gid, torch.ones_like(pos))
    ranks = torch.empty_like(pos)
    ranks[order] = (sums / cnt)[gid]
    return float((ranks[y].sum() - npos * (npos + 1) / 2.0) / (npos * nneg))
