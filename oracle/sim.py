"""The oracle's time step, in the paper's stage order (Methodology: laser
excitation, ionization, particle movement, fluid changes, field update), as a
plain sequence of calls into the FP64 C routines.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per step n -> n+1:
  J = 0
  for each species: gather E^n, B^n at x^n, Boris u^{n-1/2} -> u^{n+1/2},
                    move x^n -> x^{n+1}, reflect, Esirkepov deposit J^{n+1/2}
  add the laser source current at t^{n+1/2}
  B^{n+1/2} = B^n - dt/2 curl E^n;  E^{n+1} = E^n + dt (curl B^{n+1/2} - J);
  Mur faces;  B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}
"""
import math

import numpy as np

from . import (Fluid, Grid, Particles, charge_density, energy_fields, energy_particles, fdtd_b_half, fdtd_e,
               fluid_energy, fluid_step, fluid_to_particles, gather_species, ionize, laser_source, particles_to_fluid,
               photon_move, push_deposit, qed_emit, qed_kappa, qed_pairs, qed_tau0, regime_criterion, zeros_field)


def node_fields(g, E, B):
    """The six field components at the nodes (the classifier's input): each E
    component averaged over the two edges that meet at the node along its
    axis, each B component over the four faces around it; a neighbour outside
    a non-periodic axis counts as zero.  Returns [6, nz, ny, nx]."""
    def at(F, shifts):
        out = np.asarray(F, dtype=np.float64)
        for axis, sh in shifts:
            nd = 2 - axis                     # array axis of grid axis `axis` (x fastest)
            out = np.roll(out, 1, axis=nd) if sh else out
            if sh and g.bc[axis]:
                sl = [slice(None)] * 3
                sl[nd] = 0
                out = out.copy()
                out[tuple(sl)] = 0.0
        return out
    f = np.zeros((6,) + tuple(g.shape))
    for a in range(3):
        f[a] = 0.5 * (at(E[a], [(a, 1)]) + at(E[a], []))
    for a in range(3):
        p, q = [b for b in range(3) if b != a]
        f[3 + a] = 0.25 * (at(B[a], [(p, 1), (q, 1)]) + at(B[a], [(q, 1)]) + at(B[a], [(p, 1)]) + at(B[a], []))
    return f


def dilate(g, raw, r):
    """Chebyshev dilation by r nodes: a node is set when any node within r
    along every axis is (periodic axes wrap, others stop at the edge)."""
    m = np.asarray(raw, dtype=bool)
    for a in range(3):
        nd = 2 - a
        out = m.copy()
        for d in range(1, r + 1):
            for sgn in (1, -1):
                sh = np.roll(m, sgn * d, axis=nd)
                if g.bc[a]:
                    sl = [slice(None)] * 3
                    sl[nd] = slice(0, d) if sgn > 0 else slice(-d, None)
                    sh[tuple(sl)] = False
                out |= sh
        m = out
    return m.astype(np.uint8)


def courant_dt(d, cfl_frac):
    """cfl_frac times the 3D Yee Courant limit 1 / sqrt(sum 1/d_i^2) (c = 1)."""
    return cfl_frac / math.sqrt(sum(1.0 / v ** 2 for v in d))


class OracleSim:
    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, dt=0.0, cfl_frac=0.95, bc=(0, 0, 0), laser=None,
                 lambda_um=0.8, seed=1, shape_order=1):
        dy = dx if dy is None else dy
        dz = dx if dz is None else dz
        if not dt > 0:
            dt = courant_dt((dx, dy, dz), cfl_frac)
        self.g = Grid.make(nx, ny, nz, dx, dy, dz, dt, bc, order=shape_order)
        self.E = zeros_field(self.g)
        self.B = zeros_field(self.g)
        self.J = zeros_field(self.g)
        self.laser = laser
        self.lambda_m = lambda_um * 1e-6
        self.seed = seed
        self.species = []
        self.ionize_cfg = []
        self.kind = []
        self.qed_cfg = []
        self.pair_cfg = []
        self.w_ionize = 0.0
        self.n_ionize = 0
        self.w_photon_untracked = 0.0
        self.w_pair_deficit = 0.0
        self.n_emit = 0
        self.n_pair = 0
        self.fluids = []
        self.n_clamped = 0
        self.nstep = 0
        self.regime = dict(a_thr=1.0, n_thr=1.0, c_thr=0.1, chi_thr=1e-3, dilate=2, k_sigma=1.0, ppc=8,
                           to_species=[], policy="default", quiet=False)
        self.epoch = 0
        self.mask = np.zeros(self.g.shape, dtype=np.uint8)   # every node fluid before a classification
        self.rho_bg = np.zeros(self.g.shape)

    def load_species(self, q, m, x, y, z, ux, uy, uz, w, zq=None, ids=None, ionize=None, kind=0, qed=None,
                     pairs=None, pusher="boris", **_):
        sid = len(self.species)
        sp = Particles(q, m, x, y, z, ux, uy, uz, w, zq=zq, ids=ids, pusher=pusher)
        if qed or pairs:
            sp.tau = qed_tau0(sp.ids, self.seed, sid)
        self.species.append(sp)
        self.ionize_cfg.append(ionize)
        self.kind.append(int(kind))
        self.qed_cfg.append(qed)
        self.pair_cfg.append(pairs)
        return sid

    def load_fluid(self, q, m, n, ux=None, uy=None, uz=None, n_floor=1e-10, temperature_keV=0.0, gamma_ad=5.0 / 3.0,
                   n_ref=1.0, **_):
        """A fluid species on the nodes (arrays shaped (nz, ny, nx)); warm with
        p = n_ref T (n / n_ref)^gamma_ad when temperature_keV > 0."""
        n = np.asarray(n, dtype=np.float64)
        u = np.zeros((3,) + n.shape)
        for a, v in enumerate((ux, uy, uz)):
            if v is not None:
                u[a] = np.asarray(v, dtype=np.float64)
        K = (temperature_keV / 510.99895) / n_ref ** (gamma_ad - 1.0) if temperature_keV > 0 else 0.0
        self.fluids.append(Fluid(q, m, n, u, n_floor=n_floor, K=K, gamma_ad=gamma_ad))
        return len(self.fluids) - 1

    def set_regime(self, a_thr=1.0, n_thr=1.0, c_thr=0.1, chi_thr=1e-3, dilate=2, k_sigma=1.0, ppc=8,
                   to_species=None, policy="default", quiet=False, reach=0):
        self.regime = dict(a_thr=a_thr, n_thr=n_thr, c_thr=c_thr, chi_thr=chi_thr, dilate=dilate,
                           k_sigma=k_sigma, ppc=ppc, to_species=list(to_species or []), policy=policy,
                           quiet=bool(quiet), reach=int(reach))

    def matter_planes(self):
        """x-indices of the planes that hold matter: a fluid above its floor at
        a node of the plane, or a particle in a cell of the plane (floor(x),
        at most nx - 1)."""
        nx = self.g.shape[2]
        hold = np.zeros(nx, dtype=bool)
        for fl in self.fluids:
            hold |= (fl.n > fl.n_floor).any(axis=(0, 1))
        for sp in self.species:
            if sp.n:
                hold[np.clip(np.floor(sp.x).astype(np.int64), 0, nx - 1)] = True
        return np.nonzero(hold)[0]

    def classify(self, net=None, passes=16, mask=None):
        """Regime decision and conversions (Methodology: fluid where the flow
        is stable, PIC where the classifier or the physics flags it):
        physics criterion on the electron density (fluid + CIC of the
        electron macro-particles) and the first electron fluid's velocity,
        and/or the classifier's MC-dropout decision p_mean + k_sigma p_std >=
        0.5 on the node fields, each dilated; then per fluid f the fluid at
        nodes that switch to kinetic (kinetic now, fluid at the previous
        classification) becomes macro-particles of species to_species[f] and
        that species' particles whose nearest node is fluid go back into f.
        Returns (p_mean, p_std) of the classifier, or (None, None).  A given
        `mask` (1 = kinetic) replaces the decision: the conversions alone."""
        r, g = self.regime, self.g
        if mask is not None:
            return self._convert(np.ascontiguousarray(mask, dtype=np.uint8)) or (None, None)
        all_k = r["policy"] == "all_kinetic"
        physics = not all_k and (net is None or r["policy"] == "union")
        mask = np.full(g.shape, 1 if all_k else 0, dtype=np.uint8)
        pm = ps = None
        if physics:
            ne = np.zeros(g.shape)
            for sp, k in zip(self.species, self.kind):
                if k == 0 and sp.q < 0 and sp.zq is None:
                    ne -= charge_density(g, sp) / (-sp.q)
            fe = next((fl for fl in self.fluids if fl.q < 0), None)
            if fe is not None:
                ne += fe.n
            mask |= regime_criterion(g, self.E, self.B, ne, fluid_u=None if fe is None else fe.u,
                                     lambda_m=self.lambda_m, a_thr=r["a_thr"], n_thr=r["n_thr"], c_thr=r["c_thr"],
                                     chi_thr=r["chi_thr"], dilate=r["dilate"])
        if net is not None and not all_k:
            x = node_fields(g, self.E, self.B)[None]
            if passes > 1:
                pm, ps = net.mc_statistics(x, passes)
                pm, ps = pm[0].numpy(), ps[0].numpy()
            else:
                import torch
                pm, ps = torch.sigmoid(net.forward(x, pass_index=-1))[0].numpy(), np.zeros(g.shape)
            if r.get("reach", 0) > 0:
                # the classifier's statistics only near matter: within reach + dilate
                # planes (in x) of a plane holding matter; zero elsewhere
                planes, nx = self.matter_planes(), g.shape[2]
                keep = np.zeros(nx, dtype=bool)
                if planes.size:
                    R = r["reach"] + r["dilate"]
                    lo, hi = planes.min() - R, planes.max() + 1 + R
                    if self.g.bc[0] == 0 and (lo < 0 or hi > nx):
                        lo, hi = 0, nx   # a periodic x-axis: a range that reaches an end wraps round
                    keep[max(0, lo):min(nx, hi)] = True
                pm = np.where(keep[None, None, :], pm, 0.0)
                ps = np.where(keep[None, None, :], ps, 0.0)
            mask |= dilate(g, pm + r["k_sigma"] * ps >= 0.5, r["dilate"])
        self._convert(mask)
        return pm, ps

    def _convert(self, mask):
        r, g = self.regime, self.g
        for f, fl in enumerate(self.fluids):
            ts = r["to_species"]
            sid = ts[f] if f < len(ts) else -1
            if sid is None or sid < 0:
                continue
            switched = (mask != 0) & (self.mask == 0)
            new = fluid_to_particles(g, switched.astype(np.uint8), fl, r["ppc"], self.seed, sid, self.epoch,
                                     self.rho_bg, quiet=r.get("quiet", False))
            dst = self.species[sid]
            if dst.tau is not None:
                new.tau = qed_tau0(new.ids, self.seed, sid)
            if dst.zq is not None:
                new.zq = np.zeros(new.n)
            dst.append(new)
            particles_to_fluid(g, mask, dst, fl)
        self.epoch += 1
        self.mask = mask

    def set_fields(self, E, B):
        self.E[:] = np.asarray(E, dtype=np.float64)
        self.B[:] = np.asarray(B, dtype=np.float64)

    def step(self, n=1):
        g = self.g
        for _ in range(n):
            self.J[:] = 0.0
            for si, sp in enumerate(self.species):
                if self.kind[si] == 1:
                    # photons: fields at x^n for pair creation, then a straight move at c
                    if self.pair_cfg[si]:
                        gather_species(g, self.E, self.B, sp)
                    photon_move(g, sp)
                    continue
                sp.eb = np.zeros((sp.n, 6)) if (self.ionize_cfg[si] or self.qed_cfg[si]) else None
                push_deposit(g, self.E, self.B, self.J, sp)
            # stochastic events on the pushed particles (E^n, B^n at x^n, u^{n+1/2});
            # every new particle starts at x^{n+1} and joins its species after all
            # events of the step, so none of them is pushed or converted this step
            spawned = [[] for _ in self.species]
            kappa = qed_kappa(self.lambda_m)
            for si, sp in enumerate(self.species):
                ion = self.ionize_cfg[si]
                if ion:
                    new, en = ionize(sp, ion["zmax"], ion["ip_eV"], ion["l"], self.lambda_m, g.dt, self.seed, si,
                                     self.nstep)
                    if self.qed_cfg[ion["into"]] or self.pair_cfg[ion["into"]]:
                        new.tau = qed_tau0(new.ids, self.seed, ion["into"])
                    spawned[ion["into"]].append(new)
                    self.w_ionize += en
                    self.n_ionize += new.n
                qc = self.qed_cfg[si]
                if qc:
                    eps_min = qc.get("eps_min", 0.0) or 2.0
                    ph, lost, ev = qed_emit(sp, kappa, g.dt, eps_min, self.seed, si, self.nstep)
                    self.n_emit += ev
                    target = qc.get("photon_species", -1)
                    if target is not None and target >= 0:
                        spawned[target].append(ph)
                        self.w_photon_untracked += lost
                    else:
                        self.w_photon_untracked += lost + float(np.sum(ph.w * np.sqrt(ph.ux ** 2 + ph.uy ** 2 +
                                                                                       ph.uz ** 2)))
                pc = self.pair_cfg[si]
                if pc:
                    el, po, deficit, ev = qed_pairs(sp, kappa, g.dt, self.seed, si, self.nstep)
                    spawned[pc["electron"]].append(el)
                    spawned[pc["positron"]].append(po)
                    self.w_pair_deficit += deficit
                    self.n_pair += ev
                sp.eb = None
            for si, lst in enumerate(spawned):
                for new in lst:
                    if self.species[si].tau is not None and new.tau is None:
                        new.tau = qed_tau0(new.ids, self.seed, si)
                    if self.species[si].tau is None:
                        new.tau = None
                    self.species[si].append(new)
            # cold fluids: Lorentz force, donor-cell transport, face currents into J
            for fl in self.fluids:
                self.n_clamped += fluid_step(g, self.E, self.B, self.J, fl)
            if self.laser:
                L = self.laser
                laser_source(g, self.J, self.nstep, L["x_src"], L.get("pol", 1), L["a0"], L["tau_fwhm"],
                             L["t_peak"], L["w0_spot"], L["y_c"], L["z_c"])
            fdtd_b_half(g, self.E, self.B)
            fdtd_e(g, self.E, self.B, self.J)
            fdtd_b_half(g, self.E, self.B)
            self.nstep += 1

    def diagnostics(self):
        we, wb = energy_fields(self.g, self.E, self.B)
        w_kin = [float(np.sum(sp.w * np.sqrt(sp.ux ** 2 + sp.uy ** 2 + sp.uz ** 2))) if k == 1
                 else energy_particles(sp) for sp, k in zip(self.species, self.kind)]
        return {"step": self.nstep, "w_e": we, "w_b": wb, "w_kin": w_kin,
                "count": [sp.n for sp in self.species], "w_ionize": self.w_ionize, "n_ionize": self.n_ionize,
                "w_photon_untracked": self.w_photon_untracked, "w_pair_deficit": self.w_pair_deficit,
                "n_emit": self.n_emit, "n_pair": self.n_pair,
                "w_fluid": [fluid_energy(self.g, fl) for fl in self.fluids], "n_clamped": self.n_clamped}
