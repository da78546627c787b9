"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds none of the method's arithmetic: it only draws initial
particle sets and initial field configurations (FP32, so both sides start from
identical values).  The workloads follow the paper's setting (Methodology:
uniform Cartesian grid, macro-particles per cell weighted by density-volume
fraction, Gaussian laser) at the sizes of the benchmark configurations:

* ``ramp_slab`` -- the hybrid workload: pre-ionised hydrogen as cold electron
  and proton fluids on a linear underdense ramp (n_lo -> n_hi n_c over the
  first half of the box along x, after a vacuum gap) followed by an
  overdense slab, absorbing (Mur) faces, and a Gaussian pulse launched from
  the x_min side with a0 drawn log-uniformly from [10, 300]; the kinetic
  cells receive `ppc` macro-particles per species when they are classified.
* ``scan_runs`` -- a laser-parameter scan: independent ``ramp_slab`` runs of
  uneven grids with seeded pulse amplitudes, densities and particle counts.
* ``carbon_slab`` -- full PIC with ionization and QED: neutral carbon atoms
  (16 per cell) in a slab of atom density n_e,max / 6 (fully ionized it
  holds n_e,max electrons) with a flat top and Gaussian edges, a Gaussian
  pulse from the x_min side, and empty electron, photon and positron
  species that receive the ionization electrons, emitted photons and pairs.
* ``periodic_plasma`` -- pre-ionised hydrogen (e-, p+) at uniform density,
  `ppc` particles per cell per species at uniform random positions, Maxwellian
  momenta of temperature `T_keV` (non-relativistic Gaussian per component,
  sigma_u = sqrt(kT / m c^2)), plus a linearly polarised plane wave
  E_y = a0 cos(k x), B_z = a0 cos(k x) along x (k = 2 pi / box length for the
  fundamental mode that fits the box).
"""
import math

import numpy as np

M_P = 1836.15267343          # proton / electron mass ratio (CODATA 2018)
MC2_KEV = 510.99895000       # electron rest energy [keV]


def laser_units(lambda_um=0.8):
    """Length c/w0 in micrometres for the given wavelength."""
    return lambda_um / (2.0 * math.pi)


def uniform_particles(rng, n_cells, ppc, density, d, temperature_keV, mass, lo=(0, 0, 0), hi=None):
    """Uniformly placed particles (cell units) inside [lo, hi) with Maxwellian momenta."""
    nx, ny, nz = n_cells
    hi = hi if hi is not None else (nx, ny, nz)
    cells = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    n = int(cells * ppc)
    x = rng.uniform(lo[0], hi[0], n).astype(np.float32)
    y = rng.uniform(lo[1], hi[1], n).astype(np.float32)
    z = rng.uniform(lo[2], hi[2], n).astype(np.float32)
    for a, (v, h) in enumerate(((x, hi[0]), (y, hi[1]), (z, hi[2]))):
        np.minimum(v, np.nextafter(np.float32(h), np.float32(0)), out=v)
    sig = math.sqrt(temperature_keV / (MC2_KEV * mass))
    ux, uy, uz = (rng.standard_normal((3, n)) * sig).astype(np.float32)
    w = np.full(n, density * d[0] * d[1] * d[2] / ppc, np.float32)
    return dict(x=x, y=y, z=z, ux=ux, uy=uy, uz=uz, w=w)


def plane_wave_fields(nx, ny, nz, dx, a0, modes=1):
    """E_y = a0 cos(k x) at E_y nodes (i dx), B_z = a0 cos(k x) at B_z nodes
    ((i + 1/2) dx); k = 2 pi modes / (nx dx).  Shapes (3, nz, ny, nx) FP32."""
    k = 2.0 * math.pi * modes / (nx * dx)
    E = np.zeros((3, nz, ny, nx), np.float32)
    B = np.zeros((3, nz, ny, nx), np.float32)
    xe = np.arange(nx) * dx
    xb = (np.arange(nx) + 0.5) * dx
    E[1] = (a0 * np.cos(k * xe)).astype(np.float32)[None, None, :]
    B[2] = (a0 * np.cos(k * xb)).astype(np.float32)[None, None, :]
    return E, B


def periodic_plasma(n=32, ppc=8, density=0.1, temperature_keV=1.0, a0=1.0, cells_per_lambda=16,
                    seed=1, ny=None, nz=None):
    """The plain full-PIC workload: periodic box, e- and p+ at `density` n_c,
    `ppc` per cell per species, Maxwellian T, plane wave a0 (defaults: the
    32^3, lambda/16, 0.1 n_c, 8 ppc, 1 keV, a0 = 1 configuration)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    dx = 2.0 * math.pi / cells_per_lambda
    rng = np.random.default_rng(seed)
    d = (dx, dx, dx)
    ele = uniform_particles(rng, (n, ny, nz), ppc, density, d, temperature_keV, 1.0)
    ion = uniform_particles(rng, (n, ny, nz), ppc, density, d, temperature_keV, M_P)
    E, B = plane_wave_fields(n, ny, nz, dx, a0, modes=max(1, round(n / cells_per_lambda)))
    return dict(grid=dict(nx=n, ny=ny, nz=nz, dx=dx, cfl_frac=0.95, bc=(0, 0, 0)),
                species=[dict(q=-1.0, m=1.0, **ele), dict(q=1.0, m=M_P, **ion)], E=E, B=B)


OMEGA0_PER_FS = 2.0 * math.pi * 299792458.0 / 0.8e-6 * 1e-15   # w0 [1/fs] at 0.8 um


def ramp_slab(nx=256, ny=256, nz=128, cells_per_lambda=16, n_lo=0.01, n_hi=1.0, n_slab=5.0,
              slab_lambda=2.0, vacuum_lambda=1.0, a0=None, tau_fs=30.0, w0_lambda=2.0, seed=3, ppc=8,
              tile_capacity=8192, n_floor=1e-10):
    """The hybrid workload (defaults: 256 x 256 x 128, lambda/16).  Node
    densities n(x): 0 in the first `vacuum_lambda`, linear n_lo -> n_hi up to
    nx/2, n_slab over the next `slab_lambda`, 0 beyond; uniform in y and z.
    Fluids are at rest; densities below n_floor [n_c] count as vacuum (the
    donor-cell scheme spreads trace densities one node per step, which
    conversions must not turn into particles).  Returns grid, laser, fluids
    (electron, proton) and two empty particle species that receive the
    conversions."""
    dx = 2.0 * math.pi / cells_per_lambda
    rng = np.random.default_rng(seed)
    if a0 is None:
        a0 = float(np.exp(rng.uniform(math.log(10.0), math.log(300.0))))
    i = np.arange(nx, dtype=np.float64)
    x0 = int(round(vacuum_lambda * cells_per_lambda))
    x1 = nx // 2
    x2 = x1 + int(round(slab_lambda * cells_per_lambda))
    prof = np.zeros(nx)
    ramp = (i >= x0) & (i < x1)
    prof[ramp] = n_lo + (n_hi - n_lo) * (i[ramp] - x0) / max(1, x1 - 1 - x0)
    prof[(i >= x1) & (i < x2)] = n_slab
    n = np.broadcast_to(prof.astype(np.float32)[None, None, :], (nz, ny, nx)).copy()
    tau = tau_fs * OMEGA0_PER_FS
    laser = dict(a0=a0, tau_fwhm=tau, w0_spot=w0_lambda * 2.0 * math.pi, t_peak=1.5 * tau,
                 y_c=0.5 * (ny - 1), z_c=0.5 * (nz - 1), x_src=max(2, x0 // 2), pol=1)
    empty = np.zeros(0, np.float32)
    sp = lambda q, m: dict(q=q, m=m, x=empty, y=empty, z=empty, ux=empty, uy=empty, uz=empty, w=empty,
                           tile_capacity=tile_capacity)
    return dict(grid=dict(nx=nx, ny=ny, nz=nz, dx=dx, cfl_frac=0.95, bc=(1, 1, 1)), laser=laser,
                fluids=[dict(q=-1.0, m=1.0, n=n, n_floor=n_floor), dict(q=1.0, m=M_P, n=n, n_floor=n_floor)],
                species=[sp(-1.0, 1.0), sp(1.0, M_P)], ppc=ppc, a0=a0)


CARBON_IP_EV = [11.260, 24.383, 47.888, 64.494, 392.09, 489.99]   # NIST ASD
CARBON_L = [1, 1, 0, 0, 0, 0]                                      # 2p, 2p, 2s, 2s, 1s, 1s
M_C = 12.0 * M_P


def carbon_slab(n=128, cells_per_lambda=20, ppc=16, ne_max=10.0, plateau_lambda=2.0, edge_lambda=0.5,
                a0=100.0, tau_fs=30.0, w0_lambda=2.0, seed=2, caps=(163840, 12288, 32768, 8192), ny=None, nz=None):
    """Full PIC with ionization and QED (defaults: 128^3, lambda/20).  Atom
    density n_a(x) = (ne_max / 6) on a plateau of `plateau_lambda` centred in
    x, with Gaussian edges of width `edge_lambda` cut at 3 sigma; `ppc` atoms
    per cell at uniform random positions, weight n_a(x) dV / ppc, at rest.
    Species: 0 electrons (emit photons into 2), 1 carbon (Z = 0, ionizes into
    0), 2 photons (pairs into 0 and 3), 3 positrons (emit into 2).  `caps`
    are their initial slots per 8^3 tile: the electron tiles hold 6 electrons
    per atom slot with room for the pulse's snowplow (a front ionizes up to
    one level per ion and step, faster than the tiles can grow).  ny, nz
    (default n) give a transverse cross-section of the same slab and pulse
    axis (the pulse stays centred)."""
    dx = 2.0 * math.pi / cells_per_lambda
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    c0 = 0.5 * n
    half = 0.5 * plateau_lambda * cells_per_lambda
    sig = edge_lambda * cells_per_lambda
    lo, hi = int(math.floor(c0 - half - 3 * sig)), int(math.ceil(c0 + half + 3 * sig))
    lo, hi = max(lo, 1), min(hi, n - 2)

    def profile(x):
        d = np.maximum(np.abs(x - c0) - half, 0.0)
        return (ne_max / 6.0) * np.exp(-0.5 * (d / sig) ** 2)

    cells = (hi - lo) * ny * nz
    m = cells * ppc
    x = rng.uniform(lo, hi, m).astype(np.float32)
    y = rng.uniform(0, ny - 1, m).astype(np.float32)
    z = rng.uniform(0, nz - 1, m).astype(np.float32)
    w = (profile(x.astype(np.float64)) * dx ** 3 / ppc).astype(np.float32)
    zero = np.zeros(m, np.float32)
    ions = dict(q=1.0, m=M_C, x=x, y=y, z=z, ux=zero, uy=zero.copy(), uz=zero.copy(), w=w, zq=zero.copy(),
                ionize=dict(zmax=6, ip_eV=CARBON_IP_EV, l=CARBON_L, into=0), tile_capacity=caps[1])
    empty = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    electrons = dict(q=-1.0, m=1.0, qed=dict(photon_species=2, eps_min=2.0), tile_capacity=caps[0], **empty)
    photons = dict(q=0.0, m=0.0, kind=1, pairs=dict(electron=0, positron=3), tile_capacity=caps[2], **empty)
    positrons = dict(q=1.0, m=1.0, qed=dict(photon_species=2, eps_min=2.0), tile_capacity=caps[3], **empty)
    tau = tau_fs * OMEGA0_PER_FS
    laser = dict(a0=a0, tau_fwhm=tau, w0_spot=w0_lambda * 2.0 * math.pi, t_peak=1.5 * tau,
                 y_c=0.5 * (ny - 1), z_c=0.5 * (nz - 1), x_src=4, pol=1)
    return dict(grid=dict(nx=n, ny=ny, nz=nz, dx=dx, cfl_frac=0.95, bc=(1, 1, 1)), laser=laser,
                species=[electrons, ions, photons, positrons])


def scan_runs(n_runs=64, sizes=(64, 80, 96, 112), a0_range=(1.0, 300.0), density_range=(0.01, 2.0),
              ppc_choices=(8, 12, 16), seed=5):
    """Independent hybrid runs for a parameter scan: per run nx, ny, nz drawn
    from `sizes` (multiples of 16), a0 log-uniform in `a0_range`, the ramp +
    slab profile scaled by a density factor d log-uniform in `density_range`
    (ramp 0.01 d -> d n_c, slab 5 d n_c), `ppc` from `ppc_choices`; tiles hold
    three times the particles of a fully kinetic tile (the strongest pulses
    pile electrons up faster than the tiles grow)."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n_runs):
        nx, ny, nz = (int(v) for v in rng.choice(sizes, 3))
        a0 = float(np.exp(rng.uniform(math.log(a0_range[0]), math.log(a0_range[1]))))
        d = float(np.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1]))))
        ppc = int(rng.choice(ppc_choices))
        runs.append(ramp_slab(nx=nx, ny=ny, nz=nz, n_lo=0.01 * d, n_hi=d, n_slab=5.0 * d, a0=a0, seed=seed + r,
                              ppc=ppc, tile_capacity=3 * 512 * ppc, vacuum_lambda=1.0, slab_lambda=1.0))
    return runs


CLASSIFIER_LAYERS = [(6, 32), (32, 32), (32, 16), (16, 1)]


def classifier_weights(seed, out_bias=0.0, bias_scale=0.05):
    """Seeded FP32 weights of the regime classifier, [(W [co][ci][3][3][3], b [co])]:
    He-uniform W, U(-sqrt(6 / fan_in), sqrt(6 / fan_in)) with fan_in = 27 ci, small
    random hidden biases and a fixed output bias.  Both the GPU model (through
    hyb_model_set_layer) and the oracle take these."""
    rng = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(CLASSIFIER_LAYERS):
        lim = math.sqrt(6.0 / (27 * ci))
        w = rng.uniform(-lim, lim, (co, ci, 3, 3, 3)).astype(np.float32)
        b = (bias_scale * rng.standard_normal(co)).astype(np.float32) if l < 3 else np.full(co, out_bias, np.float32)
        out.append((w, b))
    return out


SURROGATE_LAYERS = [(10, 13), (13, 32), (32, 64), (64, 128), (128, 32), (32, 10)]


def surrogate_weights(seed, bias_scale=0.05):
    """Seeded FP32 weights of the field surrogate, [(W [co][ci][3][3][3], b [co])]:
    He-uniform W with fan_in = 27 ci and small random biases.  Both the GPU
    model (through hyb_surrogate_set_layer) and the oracle take these."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in SURROGATE_LAYERS:
        lim = math.sqrt(6.0 / (27 * ci))
        out.append((rng.uniform(-lim, lim, (co, ci, 3, 3, 3)).astype(np.float32),
                    (bias_scale * rng.standard_normal(co)).astype(np.float32)))
    return out


SWITCHNET_LAYERS = [(10, 128), (128, 256), (256, 256), (256, 256), (256, 1)]


def switchnet_weights(seed, bias_scale=0.05):
    """Seeded FP32 weights of SwitchNet, [(W [co][ci], b [co])]: He-uniform W
    with fan_in = ci and small random biases (GPU model and oracle take these)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in SWITCHNET_LAYERS:
        lim = math.sqrt(6.0 / ci)
        out.append((rng.uniform(-lim, lim, (co, ci)).astype(np.float32),
                    (bias_scale * rng.standard_normal(co)).astype(np.float32)))
    return out


def random_states(batch, n, seed, mean_scale=0.5, std_range=(0.5, 2.0)):
    """Seeded states [batch, 10, n, n, n] (FP32) with per-channel mean and
    spread, and those per-channel means and spreads (the normalisation)."""
    rng = np.random.default_rng(seed)
    mean = (mean_scale * rng.standard_normal(10)).astype(np.float32)
    std = rng.uniform(*std_range, 10).astype(np.float32)
    x = (mean[None, :, None, None, None] + std[None, :, None, None, None] *
         rng.standard_normal((batch, 10, n, n, n))).astype(np.float32)
    return x, mean, std


def field_packet(nx, ny, nz, dx, a0=10.0, x_c=None, w0=None, length=None, noise=0.05, seed=0):
    """Seeded synthetic E, B (3 x nz x ny x nx FP32 each): a linearly polarised
    wave packet along x (E_y, B_z) with a Gaussian envelope in x and in the
    transverse radius, on top of Gaussian noise of amplitude `noise` * a0 in
    every component."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) * dx)[None, None, :]
    y = ((np.arange(ny) - ny / 2) * dx)[None, :, None]
    z = ((np.arange(nz) - nz / 2) * dx)[:, None, None]
    x_c = nx * dx / 2 if x_c is None else x_c
    w0 = ny * dx / 5 if w0 is None else w0
    length = nx * dx / 8 if length is None else length
    env = a0 * np.exp(-((x - x_c) / length) ** 2 - (y ** 2 + z ** 2) / w0 ** 2)
    E = (noise * a0 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    B = (noise * a0 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    E[1] += (env * np.cos(x)).astype(np.float32)
    B[2] += (env * np.cos(x)).astype(np.float32)
    return E, B
