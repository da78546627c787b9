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

from . import (Grid, Particles, energy_fields, energy_particles, fdtd_b_half, fdtd_e, ionize, laser_source,
               push_deposit, zeros_field)


def courant_dt(d, cfl_frac):
    """cfl_frac times the 3D Yee Courant limit 1 / sqrt(sum 1/d_i^2) (c = 1)."""
    return cfl_frac / math.sqrt(sum(1.0 / v ** 2 for v in d))


class OracleSim:
    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, dt=0.0, cfl_frac=0.95, bc=(0, 0, 0), laser=None,
                 lambda_um=0.8, seed=1):
        dy = dx if dy is None else dy
        dz = dx if dz is None else dz
        if not dt > 0:
            dt = courant_dt((dx, dy, dz), cfl_frac)
        self.g = Grid.make(nx, ny, nz, dx, dy, dz, dt, bc)
        self.E = zeros_field(self.g)
        self.B = zeros_field(self.g)
        self.J = zeros_field(self.g)
        self.laser = laser
        self.lambda_m = lambda_um * 1e-6
        self.seed = seed
        self.species = []
        self.ionize_cfg = []
        self.w_ionize = 0.0
        self.n_ionize = 0
        self.nstep = 0

    def load_species(self, q, m, x, y, z, ux, uy, uz, w, zq=None, ids=None, ionize=None, **_):
        self.species.append(Particles(q, m, x, y, z, ux, uy, uz, w, zq=zq, ids=ids))
        self.ionize_cfg.append(ionize)
        return len(self.species) - 1

    def set_fields(self, E, B):
        self.E[:] = np.asarray(E, dtype=np.float64)
        self.B[:] = np.asarray(B, dtype=np.float64)

    def step(self, n=1):
        g = self.g
        for _ in range(n):
            self.J[:] = 0.0
            for sp, ion in zip(self.species, self.ionize_cfg):
                sp.eb = np.zeros((sp.n, 6)) if ion else None
                push_deposit(g, self.E, self.B, self.J, sp)
            # field ionization with E^n at x^n (recorded by the push); new electrons
            # start at x^{n+1} and are not pushed before the next step
            for si, (sp, ion) in enumerate(zip(self.species, self.ionize_cfg)):
                if not ion:
                    continue
                new, en = ionize(sp, ion["zmax"], ion["ip_eV"], ion["l"], self.lambda_m, g.dt, self.seed, si,
                                 self.nstep)
                self.species[ion["into"]].append(new)
                self.w_ionize += en
                self.n_ionize += new.n
                sp.eb = None
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
        return {"step": self.nstep, "w_e": we, "w_b": wb,
                "w_kin": [energy_particles(sp) for sp in self.species],
                "count": [sp.n for sp in self.species], "w_ionize": self.w_ionize, "n_ionize": self.n_ionize}
