"""Laser-parameter search and tile-shape autotuning on top of batched runs.

* ``de_minimize`` -- differential evolution, DE/rand/1/bin (Storn & Price,
  J. Global Optim. 11, 1997) over a box: for every member x_i a mutant
  v = x_r1 + F (x_r2 - x_r3) from three other distinct members, binomial
  crossover with rate CR (one coordinate always from v), the trial clipped to
  the box, and greedy selection (the trial replaces x_i when it is no worse).
  The whole population is evaluated at once, so a generation is one batch.
* ``LaserScan`` -- the paper's optimisation of laser intensity, duration and
  spot size for a target plasma energy (Introduction; closing paragraph of the
  Results): every candidate (a0, tau_fwhm [fs], w0 [lambda]) is one hybrid
  ramp + slab run, a population is advanced as one ``Batch`` (one CUDA graph
  per step with a branch per run), reclassified by the physics criterion every
  ``classify_every`` steps, and scored by |W_plasma - W_target| / W_target,
  W_plasma the kinetic energy of fluids and particles after ``steps`` steps.
* ``autotune_tile`` -- picks a run's tile edge (4 or 8 cells) by timing a few
  steps of each candidate with CUDA events; a ``LaserScan`` tunes once for
  its grid and particle count and runs every candidate with that tile.

Host-side orchestration only: every step of every run executes in libhyb.so.
"""
import math

import numpy as np

from . import inputs


def de_minimize(f_batch, lo, hi, pop=16, generations=20, F=0.7, CR=0.9, seed=0, callback=None):
    """Minimise f over the box [lo, hi] by DE/rand/1/bin.  f_batch maps a
    population (pop x d array) to its objective values (pop array).  Returns
    dict(x, f, pop_x, pop_f, history) with history the best value after the
    initial population and after every generation."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = lo.size
    if pop < 4:
        raise ValueError("differential evolution needs at least 4 members")
    rng = np.random.default_rng(seed)
    X = lo + (hi - lo) * rng.random((pop, d))
    fx = np.asarray(f_batch(X), dtype=np.float64)
    history = [float(fx.min())]
    for gen in range(generations):
        V = np.empty_like(X)
        for i in range(pop):
            others = [j for j in range(pop) if j != i]
            r1, r2, r3 = rng.choice(others, 3, replace=False)
            v = X[r1] + F * (X[r2] - X[r3])
            take = rng.random(d) < CR
            take[rng.integers(d)] = True
            V[i] = np.clip(np.where(take, v, X[i]), lo, hi)
        fv = np.asarray(f_batch(V), dtype=np.float64)
        better = fv <= fx
        X[better] = V[better]
        fx[better] = fv[better]
        history.append(float(fx.min()))
        if callback is not None:
            callback(gen, X, fx)
    b = int(np.argmin(fx))
    return {"x": X[b].copy(), "f": float(fx[b]), "pop_x": X, "pop_f": fx, "history": history}


def _ramp_slab_run(P, nx, ny, nz, a0, tau_fs, w0_lambda, ppc, tile, stream, seed):
    inp = inputs.ramp_slab(nx=nx, ny=ny, nz=nz, vacuum_lambda=0.25, slab_lambda=0.5, a0=a0, tau_fs=tau_fs,
                           w0_lambda=w0_lambda, ppc=ppc, tile_capacity=8 * tile ** 3 * ppc, seed=seed)
    inp["laser"]["t_peak"] = inp["laser"]["tau_fwhm"]   # the pulse peaks one FWHM after the start
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"],
                       tile=tile, stream=stream, seed=seed)
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=ppc, to_species=[0, 1], quiet=True)
    sim.classify()
    return sim


def autotune_tile(make_sim, candidates=(8, 4), steps=4, warmup=2):
    """Time `steps` steps (after `warmup`) of make_sim(tile) for every tile edge
    in `candidates` with CUDA events on the simulation's stream; returns
    (best tile, {tile: ms per step})."""
    import torch
    times = {}
    for t in candidates:
        sim = make_sim(t)
        sim.step(warmup)
        st = sim.torch_stream if sim.torch_stream is not None else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        sim.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        times[t] = e0.elapsed_time(e1) / steps
        sim.close()
    return min(times, key=times.get), times


class LaserScan:
    """Hybrid ramp + slab runs of one grid for laser parameters
    (a0, tau_fwhm [fs], w0 [lambda]); see the module docstring."""

    def __init__(self, nx=64, ny=32, nz=32, ppc=4, steps=200, classify_every=10, target=None, autotune=True,
                 seed=7):
        import torch
        from . import Batch, Simulation  # noqa: F401  (the library must be built)
        import paper_2510_11174_gb300 as P
        self.P = P
        self.shape = (nx, ny, nz)
        self.ppc, self.steps, self.every, self.seed = ppc, steps, classify_every, seed
        self.target = target
        self.stream = torch.cuda.Stream()
        self.tile = 8
        self.tile_times = None
        self.evaluations = 0
        if autotune:
            mk = lambda t: _ramp_slab_run(P, nx, ny, nz, 10.0, 30.0, 2.0, ppc, t, self.stream.cuda_stream, seed)
            cands = tuple(t for t in (8, 4) if nx % t == 0 and ny % t == 0 and nz % t == 0)
            self.tile, self.tile_times = autotune_tile(mk, candidates=cands)

    def energies(self, params):
        """Plasma kinetic energy (fluids + particles) after `steps` steps for
        every row (a0, tau_fwhm_fs, w0_lambda) of params, all rows advanced as
        one batch."""
        P = self.P
        nx, ny, nz = self.shape
        sims = [_ramp_slab_run(P, nx, ny, nz, float(a0), float(tau), float(w0), self.ppc, self.tile,
                               self.stream.cuda_stream, self.seed) for a0, tau, w0 in np.asarray(params)]
        batch = P.Batch(sims, self.stream)
        done = 0
        while done < self.steps:
            k = min(self.every, self.steps - done)
            batch.step(k)
            done += k
            if done < self.steps:
                for s in sims:
                    s.classify()
        out = []
        for s in sims:
            d = s.diagnostics()
            out.append(sum(d["w_kin"]) + sum(d["w_fluid"]))
        batch.close()
        for s in sims:
            s.close()
        self.evaluations += len(sims)
        return np.asarray(out)

    def objective(self, params):
        w = self.energies(params)
        return np.abs(w - self.target) / abs(self.target)

    def optimize(self, lo=(1.0, 3.0, 0.5), hi=(30.0, 20.0, 3.0), pop=8, generations=4, seed=1):
        """Differential evolution over (a0, tau_fwhm [fs], w0 [lambda]) for the target energy."""
        if self.target is None:
            raise ValueError("LaserScan.optimize needs a target energy")
        return de_minimize(self.objective, lo, hi, pop=pop, generations=generations, seed=seed)


def intensity_w_cm2(a0, lambda_um=0.8):
    """Peak intensity of a linearly polarised pulse of normalised amplitude a0:
    I = a0^2 1.37e18 / lambda_um^2 W/cm^2 (the standard relativistic-intensity relation)."""
    return a0 * a0 * 1.37e18 / (lambda_um * lambda_um)


def a0_from_intensity(I_w_cm2, lambda_um=0.8):
    return math.sqrt(I_w_cm2 * lambda_um * lambda_um / 1.37e18)
