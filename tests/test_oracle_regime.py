"""Pins of the oracle's regime switching: the criterion marks what its
thresholds say and dilates by the stated distance; conversions keep the
discrete Gauss law (with the residual background charge), the number of
real particles, the momentum and, for fluid -> particles, the kinetic energy
exactly."""
import math

import numpy as np
import pytest

import oracle


def _grid(bc=(0, 0, 0)):
    return oracle.Grid.make(16, 12, 8, 0.3, 0.3, 0.3, 0.15, bc=bc)


def test_criterion_marks_strong_field_region_dilated():
    g = _grid()
    E = oracle.zeros_field(g)
    B = oracle.zeros_field(g)
    E[1][4, 6, 8] = 3.0          # E_y at (8, 6.5, 4): node fields |E| >= 1 at (8,6,4) and (8,7,4)
    ne = np.zeros(g.shape)
    m = oracle.regime_criterion(g, E, B, ne, dilate=2, chi_thr=1e9)
    z, y, x = np.nonzero(m)
    assert (x.min(), x.max()) == (6, 10) and (y.min(), y.max()) == (4, 9) and (z.min(), z.max()) == (2, 6)
    m0 = oracle.regime_criterion(g, E, B, ne, dilate=0, chi_thr=1e9)
    assert np.count_nonzero(m0) == 2


def test_criterion_density_and_compression():
    g = _grid()
    E = oracle.zeros_field(g)
    B = oracle.zeros_field(g)
    ne = np.full(g.shape, 0.1)
    ne[3, 3, 3] = 1.5
    m = oracle.regime_criterion(g, E, B, ne, dilate=0)
    assert np.count_nonzero(m) == 1 and m[3, 3, 3] == 1
    # converging flow along x: v = -0.5 tanh(x - x0) -> dt div v strongly negative at x0
    u = np.zeros((3,) + g.shape)
    x = np.arange(16) * g.dx
    u[0] = (-3.0 * np.tanh((x - x[8]) / g.dx))[None, None, :]
    m = oracle.regime_criterion(g, E, B, np.full(g.shape, 0.1), fluid_u=u, dilate=0)
    assert np.all(m[:, :, 8] == 1) and np.count_nonzero(m[:, :, 2]) == 0


def _rho_total(g, species, fluids, rho_bg):
    rho = np.zeros(g.shape)
    for sp in species:
        oracle.charge_density(g, sp, rho)
    for fl in fluids:
        rho += fl.q * fl.n
    return rho + rho_bg


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_fluid_to_particles_keeps_gauss_law_number_momentum_energy(bc):
    g = _grid(bc)
    rng = np.random.default_rng(2)
    fl = oracle.Fluid(-1.0, 1.0, 0.2 + rng.random(g.shape), 0.3 * rng.standard_normal((3,) + g.shape))
    mask = (rng.random(g.shape) < 0.3).astype(np.uint8)
    rho_bg = np.zeros(g.shape)
    before = _rho_total(g, [], [fl], rho_bg)
    dV = g.dx * g.dy * g.dz
    num0 = fl.n[mask == 1].sum() * dV
    mom0 = (fl.n * fl.u)[:, mask == 1].sum(axis=1) * dV
    en0 = oracle.fluid_energy(g, oracle.Fluid(-1.0, 1.0, fl.n * mask, fl.u))
    sp = oracle.fluid_to_particles(g, mask, fl, 8, 5, 0, 1, rho_bg)
    assert sp.n == 8 * np.count_nonzero(mask)
    after = _rho_total(g, [oracle.Particles(-1.0, 1.0, sp.x, sp.y, sp.z, sp.ux, sp.uy, sp.uz, sp.w)], [fl], rho_bg)
    assert np.max(np.abs(after - before)) < 1e-12 * np.max(np.abs(before))
    assert sp.w.sum() == pytest.approx(num0, rel=1e-13)
    assert np.allclose(np.stack([(sp.w * sp.ux).sum(), (sp.w * sp.uy).sum(), (sp.w * sp.uz).sum()]), mom0,
                       rtol=1e-12, atol=1e-14)
    assert oracle.energy_particles(sp) == pytest.approx(en0, rel=1e-12)
    assert np.all(fl.n[mask == 1] == 0)
    # positions lie in the nodes' dual cells and inside the domain
    hi = [16, 12, 8] if bc[0] == 0 else [15, 11, 7]
    for v, h in zip((sp.x, sp.y, sp.z), hi):
        assert v.min() >= 0 and v.max() <= h


def test_particles_to_fluid_keeps_node_charge_number_momentum():
    g = _grid()
    rng = np.random.default_rng(3)
    n = 3000
    sp = oracle.Particles(-1.0, 1.0, rng.uniform(0, 16, n), rng.uniform(0, 12, n), rng.uniform(0, 8, n),
                          *(0.2 * rng.standard_normal((3, n))), rng.uniform(0.5, 1.5, n) * 1e-3)
    fl = oracle.Fluid(-1.0, 1.0, np.full(g.shape, 0.05), 0.1 * rng.standard_normal((3,) + g.shape))
    mask = (rng.random(g.shape) < 0.5).astype(np.uint8)
    rho_bg = np.zeros(g.shape)
    before = _rho_total(g, [sp], [fl], rho_bg)
    dV = g.dx * g.dy * g.dz
    num0 = sp.w.sum() + fl.n.sum() * dV
    mom0 = np.array([(sp.w * sp.ux).sum(), (sp.w * sp.uy).sum(), (sp.w * sp.uz).sum()]) + \
        (fl.n * fl.u).sum(axis=(1, 2, 3)) * dV
    k = oracle.particles_to_fluid(g, mask, sp, fl)
    assert 0 < k < n
    after = _rho_total(g, [sp], [fl], rho_bg)
    assert np.max(np.abs(after - before)) < 1e-12 * np.max(np.abs(before))
    assert sp.w.sum() + fl.n.sum() * dV == pytest.approx(num0, rel=1e-13)
    mom1 = np.array([(sp.w * sp.ux).sum(), (sp.w * sp.uy).sum(), (sp.w * sp.uz).sum()]) + \
        (fl.n * fl.u).sum(axis=(1, 2, 3)) * dV
    assert np.allclose(mom1, mom0, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1)])
def test_dilate_matches_brute_force(bc):
    from oracle.sim import dilate
    g = oracle.Grid.make(9, 7, 5, 0.3, 0.3, 0.3, 0.15, bc=bc)
    raw = (np.random.default_rng(1).random(g.shape) > 0.93).astype(np.uint8)
    r = 2
    ref = np.zeros_like(raw)
    nz, ny, nx = g.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                hit = 0
                for dk in range(-r, r + 1):
                    for dj in range(-r, r + 1):
                        for di in range(-r, r + 1):
                            q = [i + di, j + dj, k + dk]
                            n = [nx, ny, nz]
                            ok = True
                            for a in range(3):
                                if bc[a] == 0:
                                    q[a] %= n[a]
                                elif not 0 <= q[a] < n[a]:
                                    ok = False
                            if ok and raw[q[2], q[1], q[0]]:
                                hit = 1
                ref[k, j, i] = hit
    assert np.array_equal(dilate(g, raw, r), ref)


def test_node_fields_of_linear_fields_are_exact():
    # E_a sampled at its edge positions (i + 1/2 along a) and B_a at its face
    # centres (half-integer along the two other axes): averaging a linear
    # function over symmetric neighbours returns its value at the node
    from oracle.sim import node_fields
    g = oracle.Grid.make(8, 6, 5, 0.3, 0.3, 0.3, 0.15, bc=(1, 1, 1))
    nz, ny, nx = g.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = lambda x, y, z, c: c + 0.3 * x - 0.2 * y + 0.7 * z
    E = np.stack([lin(i + 0.5, j, k, 1.0), lin(i, j + 0.5, k, 2.0), lin(i, j, k + 0.5, 3.0)])
    B = np.stack([lin(i, j + 0.5, k + 0.5, 4.0), lin(i + 0.5, j, k + 0.5, 5.0), lin(i + 0.5, j + 0.5, k, 6.0)])
    f = node_fields(g, E, B)
    inner = (slice(1, None), slice(1, None), slice(1, None))
    for c in range(6):
        assert np.allclose(f[c][inner], lin(i, j, k, c + 1.0)[inner], atol=1e-12), c
    # at the lower faces of non-periodic axes the missing neighbour counts as zero
    assert np.allclose(f[0][:, :, 0], 0.5 * E[0][:, :, 0])


def test_oracle_all_kinetic_classification():
    from oracle.sim import OracleSim
    o = OracleSim(8, 8, 8, 0.3, bc=(1, 1, 1))
    o.load_species(-1.0, 1.0, *[np.zeros(0, np.float32)] * 7)
    n = np.full((8, 8, 8), 0.2)
    n[:, :, :2] = 0.0
    o.load_fluid(-1.0, 1.0, n, n_floor=0.0)
    o.set_regime(ppc=3, to_species=[0], policy="all_kinetic", dilate=0)
    rho0 = -n.copy()
    o.classify()
    assert o.mask.all()
    assert o.species[0].n == 3 * np.count_nonzero(n > 0)
    assert np.all(o.fluids[0].n == 0.0)
    rho = oracle.charge_density(o.g, o.species[0]) + o.rho_bg
    assert np.max(np.abs(rho - rho0)) <= 1e-12
    assert math.isclose(float(np.sum(o.species[0].w)), float(np.sum(n)) * 0.3 ** 3, rel_tol=1e-12)


def test_oracle_converts_only_nodes_that_switch_to_kinetic():
    """Fluid that flows into a node already kinetic stays fluid: a second
    classification with the same mask creates no particles, one that adds
    nodes creates ppc particles at each new node only."""
    from oracle.sim import OracleSim
    o = OracleSim(8, 8, 8, 0.3, bc=(1, 1, 1))
    o.load_species(-1.0, 1.0, *[np.zeros(0, np.float32)] * 7)
    o.load_fluid(-1.0, 1.0, np.full((8, 8, 8), 0.2), n_floor=0.0)
    o.set_regime(ppc=2, to_species=[0], dilate=0)
    m1 = np.zeros((8, 8, 8), np.uint8)
    m1[2:4, 2:4, 2:4] = 1
    o.classify(mask=m1)
    assert o.species[0].n == 2 * 8
    o.fluids[0].n[m1 == 1] = 0.05             # fluid flowed back into the kinetic nodes
    o.classify(mask=m1)
    assert o.species[0].n == 2 * 8 and np.all(o.fluids[0].n[m1 == 1] == 0.05)
    m2 = m1.copy()
    m2[5, 5, 5] = 1
    o.classify(mask=m2)
    assert o.species[0].n == 2 * 9


@pytest.mark.parametrize("ppc,lattice", [(8, (2, 2, 2)), (4, (2, 2, 1)), (27, (3, 3, 3)), (2, (2, 1, 1)),
                                         (12, (3, 2, 2)), (1, (1, 1, 1))])
def test_quiet_start_places_the_sub_lattice_centres(ppc, lattice):
    """Quiet start: node c's particles sit at c - 1/2 + (m + 1/2) / l_a along each
    axis, an l_x x l_y x l_z lattice as close to cubic as ppc allows."""
    g = _grid()
    fl = oracle.Fluid(-1.0, 1.0, np.zeros(g.shape), np.zeros((3,) + g.shape))
    fl.n[3, 5, 7] = 0.4
    mask = np.zeros(g.shape, np.uint8)
    mask[3, 5, 7] = 1
    sp = oracle.fluid_to_particles(g, mask, fl, ppc, 5, 0, 1, np.zeros(g.shape), quiet=True)
    grid = np.stack(np.meshgrid(*[(np.arange(l) + 0.5) / l - 0.5 for l in lattice], indexing="ij"), -1)
    want = grid.reshape(-1, 3) + [7, 5, 3]
    got = np.stack([sp.x, sp.y, sp.z], -1)
    lex = lambda a: a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
    assert sp.n == ppc and np.allclose(lex(got), lex(want), rtol=0, atol=1e-14)


@pytest.mark.parametrize("ppc", [8, 27])
def test_quiet_start_of_a_uniform_fluid_leaves_no_residual_charge(ppc):
    """A uniform periodic fluid converted everywhere with quiet start gives
    particles whose CIC charge is the fluid's charge at every node, so the
    residual background charge vanishes (random positions leave shot noise)."""
    g = _grid()
    fl = oracle.Fluid(-1.0, 1.0, np.full(g.shape, 0.3), np.zeros((3,) + g.shape))
    mask = np.ones(g.shape, np.uint8)
    rho_bg = np.zeros(g.shape)
    oracle.fluid_to_particles(g, mask, fl, ppc, 5, 0, 1, rho_bg, quiet=True)
    assert np.max(np.abs(rho_bg)) < 1e-13
    fl2 = oracle.Fluid(-1.0, 1.0, np.full(g.shape, 0.3), np.zeros((3,) + g.shape))
    rho_bg2 = np.zeros(g.shape)
    oracle.fluid_to_particles(g, mask, fl2, ppc, 5, 0, 1, rho_bg2, quiet=False)
    assert np.max(np.abs(rho_bg2)) > 1e-3


def test_reach_zeroes_the_statistics_away_from_matter_and_keeps_them_near_it():
    """With a reach the classifier's statistics stay those of the whole grid on
    the x-planes within reach + dilate of matter (fluid above its floor in
    planes 10..12, one particle in plane 30) and are zero elsewhere; the
    planes are found by brute force over the nodes and particles."""
    from oracle.classifier import OracleCNN
    from oracle.sim import OracleSim
    from paper_2510_11174_gb300 import inputs
    nx, ny, nz = 48, 8, 4
    rng = np.random.default_rng(3)
    E = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    B = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    n = np.zeros((nz, ny, nx))
    n[:, :, 10:13] = 0.5
    n[1, 2, 9] = 1e-12                        # below the floor: not matter
    net = OracleCNN(inputs.classifier_weights(4), dropout=0.2, seed=4)
    out = {}
    for reach in (0, 3):
        o = OracleSim(nx, ny, nz, 0.3, bc=(1, 1, 1))
        one = lambda v: np.array([v], np.float32)
        o.load_species(-1.0, 1.0, one(30.5), one(4.0), one(2.0), one(0.0), one(0.0), one(0.0), one(1e-3))
        o.load_fluid(-1.0, 1.0, n, n_floor=1e-10)
        o.set_fields(E, B)
        o.set_regime(ppc=1, to_species=[-1], dilate=1, reach=reach)
        assert list(o.matter_planes()) == [10, 11, 12, 30]
        out[reach] = o.classify(net, passes=2)
    (pm0, ps0), (pm3, ps3) = out[0], out[3]
    keep = np.zeros(nx, dtype=bool)
    keep[10 - 4:30 + 1 + 4] = True            # reach 3 + dilate 1 around planes 10 .. 30
    assert np.array_equal(pm3[:, :, keep], pm0[:, :, keep]) and np.array_equal(ps3[:, :, keep], ps0[:, :, keep])
    assert not pm3[:, :, ~keep].any() and not ps3[:, :, ~keep].any()
    assert pm0[:, :, ~keep].all()


def test_reach_on_a_periodic_axis_keeps_every_plane_when_the_range_wraps():
    """Matter near x = 0 of a periodic box: its neighbourhood wraps round to the
    last planes, so the restricted statistics equal the whole grid's
    everywhere; away from the ends only the range is kept."""
    from oracle.classifier import OracleCNN
    from oracle.sim import OracleSim
    from paper_2510_11174_gb300 import inputs
    nx, ny, nz = 32, 8, 4
    rng = np.random.default_rng(5)
    E = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    B = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    net = OracleCNN(inputs.classifier_weights(6), dropout=0.2, seed=6)
    out = {}
    for lo_plane in (1, 14):
        n = np.zeros((nz, ny, nx))
        n[:, :, lo_plane:lo_plane + 2] = 0.5
        for reach in (0, 2):
            o = OracleSim(nx, ny, nz, 0.3, bc=(0, 0, 0))
            o.load_species(-1.0, 1.0, *[np.zeros(0, np.float32)] * 7)
            o.load_fluid(-1.0, 1.0, n, n_floor=1e-10)
            o.set_fields(E, B)
            o.set_regime(ppc=1, to_species=[-1], dilate=1, reach=reach)
            out[lo_plane, reach] = o.classify(net, passes=2)[0]
    assert np.array_equal(out[1, 2], out[1, 0])           # wraps: every plane kept
    keep = np.zeros(nx, dtype=bool)
    keep[14 - 3:16 + 3] = True
    assert np.array_equal(out[14, 2][:, :, keep], out[14, 0][:, :, keep])
    assert not out[14, 2][:, :, ~keep].any()
