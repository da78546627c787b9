"""FP64 CPU oracle for the hybrid fluid-kinetic step of arXiv 2510.11174.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2510_11174_gb300``) never imports, links
or runs it, and the two share no code: the oracle is a separate, plain,
double-precision implementation written from the paper's Methodology section
and the textbook methods it names, so that the CUDA path can be checked
against it.

The arithmetic lives in the C files next to this module (compiled with gcc
into ``liboracle.so``); this module only marshals numpy arrays.
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("bc", C.c_int * 3), ("order", C.c_int)]

    @classmethod
    def make(cls, nx, ny, nz, dx, dy, dz, dt, bc=(0, 0, 0), order=1):
        g = cls()
        g.order = int(order)
        g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
        g.dx, g.dy, g.dz, g.dt = float(dx), float(dy), float(dz), float(dt)
        for a in range(3):
            g.bc[a] = int(bc[a])
        return g

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


class Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_long),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p),
                ("w", C.c_void_p), ("zq", C.c_void_p), ("id", C.c_void_p), ("eb", C.c_void_p),
                ("pusher", C.c_int)]


_P = C.c_void_p
_D3 = C.c_void_p * 3


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_P, _P, _P]
    L.orc_u01.argtypes = [C.c_uint32]
    L.orc_u01.restype = C.c_double
    L.orc_fdtd_b_half.argtypes = [C.POINTER(Grid), _D3, _D3]
    L.orc_fdtd_e.argtypes = [C.POINTER(Grid), _D3, _D3, _D3]
    L.orc_gather.argtypes = [C.POINTER(Grid), _D3, _D3, C.c_double, C.c_double, C.c_double, _P, _P]
    L.orc_boris.argtypes = [C.c_double, _P, _P, _P]
    L.orc_tsc.argtypes = [C.c_double]
    L.orc_tsc.restype = C.c_double
    L.orc_vay.argtypes = [C.c_double, _P, _P, _P]
    L.orc_higuera_cary.argtypes = [C.c_double, _P, _P, _P]
    L.orc_esirkepov.argtypes = [C.POINTER(Grid), C.c_double] + [C.c_double] * 6 + [_D3]
    L.orc_push_deposit.argtypes = [C.POINTER(Grid), _D3, _D3, _D3, C.POINTER(Species)]
    L.orc_energy_fields.argtypes = [C.POINTER(Grid), _D3, _D3, _P]
    L.orc_energy_particles.argtypes = [C.POINTER(Species)]
    L.orc_energy_particles.restype = C.c_double
    L.orc_charge_density.argtypes = [C.POINTER(Grid), C.POINTER(Species), _P]
    L.orc_div_e.argtypes = [C.POINTER(Grid), _D3, _P]
    L.orc_laser_source.argtypes = [C.POINTER(Grid), C.c_int, C.c_int] + [C.c_double] * 6 + [C.c_long, _D3]
    L.orc_plasma_scales.argtypes = [C.c_double, _P]
    L.orc_laser_scales.argtypes = [C.c_double, _P]
    L.orc_adk_rate.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
    L.orc_adk_rate.restype = C.c_double
    L.orc_keldysh.argtypes = [C.c_double] * 3
    L.orc_keldysh.restype = C.c_double
    L.orc_mpi_rate.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double]
    L.orc_mpi_rate.restype = C.c_double
    L.orc_blend_weight.argtypes = [C.c_double]
    L.orc_blend_weight.restype = C.c_double
    L.orc_ionization_rate.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double]
    L.orc_ionization_rate.restype = C.c_double
    L.orc_ionize.argtypes = [C.POINTER(Species), _P, C.c_int, _P, _P, C.c_double, C.c_double, C.c_double,
                             C.c_uint32, C.c_uint32, C.c_long, C.POINTER(Species), C.c_long, _P]
    L.orc_ionize.restype = C.c_long
    for nm in ("orc_bessel_k", "orc_bessel_k_int"):
        getattr(L, nm).argtypes = [C.c_double, C.c_double]
        getattr(L, nm).restype = C.c_double
    for nm in ("orc_airy_ai", "orc_airy_aip", "orc_airy_int"):
        getattr(L, nm).argtypes = [C.c_double]
        getattr(L, nm).restype = C.c_double
    for nm in ("orc_qed_h", "orc_qed_power", "orc_qed_T"):
        getattr(L, nm).argtypes = [C.c_double]
        getattr(L, nm).restype = C.c_double
    for nm in ("orc_qed_em_density", "orc_qed_pair_density", "orc_qed_em_sample", "orc_qed_pair_sample"):
        getattr(L, nm).argtypes = [C.c_double, C.c_double]
        getattr(L, nm).restype = C.c_double
    L.orc_chi.argtypes = [C.c_double, _P, _P, _P, C.c_int]
    L.orc_chi.restype = C.c_double
    L.orc_splitmix64.argtypes = [C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_derived_id.argtypes = [C.c_uint64, C.c_long, C.c_uint]
    L.orc_derived_id.restype = C.c_uint64
    L.orc_qed_tau0.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
    L.orc_qed_tau0.restype = C.c_double
    L.orc_qed_emit.argtypes = [C.POINTER(Species), _P, C.c_double, C.c_double, C.c_double, C.c_uint32, C.c_uint32,
                               C.c_long, C.POINTER(Species), _P, C.c_long, _P]
    L.orc_qed_emit.restype = C.c_long
    L.orc_photon_move.argtypes = [C.POINTER(Grid), C.POINTER(Species)]
    L.orc_gather_species.argtypes = [C.POINTER(Grid), _D3, _D3, C.POINTER(Species)]
    L.orc_qed_pairs.argtypes = [C.POINTER(Species), _P, _P, C.c_double, C.c_double, C.c_uint32, C.c_uint32, C.c_long,
                                C.POINTER(Species), _P, C.POINTER(Species), _P, C.c_long, _P]
    L.orc_qed_pairs.restype = C.c_long
    L.orc_node_fields.argtypes = [C.POINTER(Grid), _D3, _D3, C.c_int, C.c_int, C.c_int, _P, _P]
    L.orc_fluid_step.argtypes = [C.POINTER(Grid), _D3, _D3, _D3, C.c_double, C.c_double, _P, _D3, C.c_double,
                                 C.c_double, C.c_double]
    L.orc_fluid_step.restype = C.c_long
    L.orc_fluid_energy.argtypes = [C.POINTER(Grid), C.c_double, _P, _D3]
    L.orc_fluid_energy.restype = C.c_double
    L.orc_regime_criterion.argtypes = [C.POINTER(Grid), _D3, _D3, _P, C.c_void_p] + [C.c_double] * 5 + [C.c_int, _P]
    L.orc_fluid_to_particles.argtypes = [C.POINTER(Grid), _P, C.c_double, _P, _D3, C.c_double, C.c_int, C.c_uint32,
                                         C.c_uint32, C.c_uint32, C.POINTER(Species), C.c_long, _P, C.c_int]
    L.orc_fluid_to_particles.restype = C.c_long
    L.orc_particles_to_fluid.argtypes = [C.POINTER(Grid), _P, C.POINTER(Species), _P, _D3, C.c_double, _P]
    L.orc_particles_to_fluid.restype = C.c_long
    L.orc_dropout_mask.argtypes = [_P, C.c_int, C.c_int, C.c_long, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double]
    L.orc_dropout_mask_cells.argtypes = [_P, C.c_int, C.c_int, C.c_long, _P, C.c_uint32, C.c_uint32, C.c_uint32,
                                         C.c_double]
    for name, fn in _EXTRA_DECLS:
        fn(L)


_EXTRA_DECLS = []


def _ptr(a):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _f3(F):
    """(3, nz, ny, nx) float64 array -> array of 3 pointers."""
    assert F.dtype == np.float64 and F.shape[0] == 3 and F.flags["C_CONTIGUOUS"]
    return _D3(*[F[c].ctypes.data_as(C.c_void_p) for c in range(3)])


# --------------------------------------------------------------------------- Philox
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(x):
    return lib().orc_u01(int(x))


# --------------------------------------------------------------------------- fields
def zeros_field(g):
    return np.zeros((3,) + g.shape, dtype=np.float64)


def fdtd_b_half(g, E, B):
    lib().orc_fdtd_b_half(C.byref(g), _f3(E), _f3(B))


def fdtd_e(g, E, B, J):
    lib().orc_fdtd_e(C.byref(g), _f3(E), _f3(B), _f3(J))


def energy_fields(g, E, B):
    out = np.zeros(2)
    lib().orc_energy_fields(C.byref(g), _f3(E), _f3(B), _ptr(out))
    return out


def div_e(g, E):
    out = np.zeros(g.shape)
    lib().orc_div_e(C.byref(g), _f3(E), _ptr(out))
    return out


# --------------------------------------------------------------------------- particles
class Particles:
    """Host particle set in FP64: positions in cell units, u = gamma*beta."""

    FIELDS = ("x", "y", "z", "ux", "uy", "uz", "w")

    PUSHERS = {"boris": 0, "vay": 1, "higuera_cary": 2}

    def __init__(self, q, m, x, y, z, ux, uy, uz, w, zq=None, ids=None, tau=None, pusher="boris"):
        self.q, self.m = float(q), float(m)
        self.pusher = self.PUSHERS[pusher]
        for name, v in zip(self.FIELDS, (x, y, z, ux, uy, uz, w)):
            setattr(self, name, np.ascontiguousarray(v, dtype=np.float64).copy())
        self.zq = None if zq is None else np.ascontiguousarray(zq, dtype=np.float64).copy()
        self.tau = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64).copy()
        self.ids = (np.arange(len(self.x), dtype=np.uint64) if ids is None
                    else np.ascontiguousarray(ids, dtype=np.uint64).copy())
        self.eb = None  # set to a (n, 6) array to record E^n, B^n at x^n during the push

    @property
    def n(self):
        return len(self.x)

    def cstruct(self):
        s = Species()
        s.q, s.m, s.n = self.q, self.m, self.n
        for name in self.FIELDS:
            setattr(s, name, _ptr(getattr(self, name)).value)
        s.zq = None if self.zq is None else _ptr(self.zq).value
        s.id = _ptr(self.ids).value
        s.eb = None if self.eb is None else _ptr(self.eb).value
        s.pusher = self.pusher
        return s

    def append(self, other):
        for name in self.FIELDS:
            setattr(self, name, np.concatenate([getattr(self, name), getattr(other, name)]))
        if self.zq is not None:
            self.zq = np.concatenate([self.zq, other.zq])
        if self.tau is not None:
            self.tau = np.concatenate([self.tau, other.tau])
        self.ids = np.concatenate([self.ids, other.ids])

    def select(self, mask):
        for name in self.FIELDS:
            setattr(self, name, np.ascontiguousarray(getattr(self, name)[mask]))
        if self.zq is not None:
            self.zq = np.ascontiguousarray(self.zq[mask])
        if self.tau is not None:
            self.tau = np.ascontiguousarray(self.tau[mask])
        self.ids = np.ascontiguousarray(self.ids[mask])


def gather(g, E, B, pos):
    e = np.zeros(3)
    b = np.zeros(3)
    lib().orc_gather(C.byref(g), _f3(E), _f3(B), float(pos[0]), float(pos[1]), float(pos[2]),
                     _ptr(e), _ptr(b))
    return e, b


def boris(qm_dt_half, e, b, u, pusher="boris"):
    """One momentum update u^{n-1/2} -> u^{n+1/2} in the fields e, b by the
    Boris, Vay or Higuera-Cary pusher."""
    e = np.ascontiguousarray(e, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    fn = {"boris": lib().orc_boris, "vay": lib().orc_vay, "higuera_cary": lib().orc_higuera_cary}[pusher]
    fn(float(qm_dt_half), _ptr(e), _ptr(b), _ptr(uu))
    return uu


def esirkepov(g, qw, p0, p1, J):
    lib().orc_esirkepov(C.byref(g), float(qw), *[float(v) for v in p0], *[float(v) for v in p1], _f3(J))


def push_deposit(g, E, B, J, sp):
    s = sp.cstruct()
    lib().orc_push_deposit(C.byref(g), _f3(E), _f3(B), _f3(J), C.byref(s))


def energy_particles(sp):
    s = sp.cstruct()
    return lib().orc_energy_particles(C.byref(s))


def charge_density(g, sp, rho=None):
    if rho is None:
        rho = np.zeros(g.shape)
    s = sp.cstruct()
    lib().orc_charge_density(C.byref(g), C.byref(s), _ptr(rho))
    return rho


def plasma_scales(n_m3):
    """(w_p, E_0, B_0, J_0, rho_0) in SI for electron density n [m^-3]."""
    out = np.zeros(5)
    lib().orc_plasma_scales(float(n_m3), _ptr(out))
    return out


def laser_scales(lambda_m):
    """(w0, n_c, E_ref, c/w0) in SI for wavelength lambda [m]."""
    out = np.zeros(4)
    lib().orc_laser_scales(float(lambda_m), _ptr(out))
    return out


def laser_source(g, J, step, x_src, pol, a0, tau_fwhm, t_peak, w0_spot, y_c, z_c):
    lib().orc_laser_source(C.byref(g), int(x_src), int(pol), float(a0), float(tau_fwhm), float(t_peak),
                           float(w0_spot), float(y_c), float(z_c), int(step), _f3(J))


# --------------------------------------------------------------------------- ionization
HARTREE_EV = 27.211386245988      # CODATA 2018
T_ATOMIC = 2.4188843265857e-17    # atomic unit of time [s]
E_ATOMIC = 5.14220674763e11       # atomic unit of field [V/m]


def adk_rate(F, Ip, Z, l=0, m=0):
    return lib().orc_adk_rate(float(F), float(Ip), float(Z), int(l), int(m))


def keldysh(F, Ip, w0):
    return lib().orc_keldysh(float(F), float(Ip), float(w0))


def mpi_rate(F, Ip, Z, l, w0):
    return lib().orc_mpi_rate(float(F), float(Ip), float(Z), int(l), float(w0))


def blend_weight(gamma):
    return lib().orc_blend_weight(float(gamma))


def ionization_rate(F, Ip, Z, l, w0):
    """Blended ADK/MPI rate [1/atomic time] at field F [atomic units]."""
    return lib().orc_ionization_rate(float(F), float(Ip), float(Z), int(l), float(w0))


def atomic_units(lambda_m, dt_norm):
    """(w0 in a.u., E_ref/E_atomic, dt in a.u.) for wavelength lambda and dt in 1/w0."""
    w0, nc, Eref, L = laser_scales(lambda_m)
    return w0 * T_ATOMIC, Eref / E_ATOMIC, dt_norm / w0 / T_ATOMIC


def ionize(ions, zmax, Ip_eV, lq, lambda_m, dt_norm, seed, sp_index, step):
    """One Monte Carlo ionization pass over `ions` (uses ions.eb from the push).
    Returns (new electron Particles, ionization energy in units m_e c^2 * n_c (c/w0)^3)."""
    w0_au, eratio, dt_au = atomic_units(lambda_m, dt_norm)
    Ip = np.ascontiguousarray(np.asarray(Ip_eV, dtype=np.float64) / HARTREE_EV)
    lqa = np.ascontiguousarray(np.asarray(lq, dtype=np.int32))
    cap = ions.n
    out = Particles(-1.0, 1.0, *([np.zeros(cap)] * 7))
    out.ids = np.zeros(cap, dtype=np.uint64)
    si, so = ions.cstruct(), out.cstruct()
    en = np.zeros(1)
    n = lib().orc_ionize(C.byref(si), _ptr(ions.eb), int(zmax), _ptr(Ip), _ptr(lqa), w0_au, eratio, dt_au,
                         int(seed) & 0xFFFFFFFF, int(sp_index), int(step), C.byref(so), cap, _ptr(en))
    out.select(np.arange(n))
    # Hartree -> m_e c^2
    return out, en[0] * HARTREE_EV / 510998.95


# --------------------------------------------------------------------------- Airy
def bessel_k(nu, x):
    return lib().orc_bessel_k(float(nu), float(x))


def bessel_k_int(nu, x):
    return lib().orc_bessel_k_int(float(nu), float(x))


def airy_ai(z):
    return lib().orc_airy_ai(float(z))


def airy_aip(z):
    return lib().orc_airy_aip(float(z))


def airy_int(z):
    """int_z^inf Ai(t) dt, z >= 0."""
    return lib().orc_airy_int(float(z))


# --------------------------------------------------------------------------- QED (LCFA)
ALPHA = 7.2973525693e-3


def qed_kappa(lambda_m):
    """hbar w0 / (m c^2) = E_ref / E_s for the laser wavelength."""
    hbar, me, c = 1.054571817e-34, 9.1093837015e-31, 299792458.0
    return hbar * 2 * math.pi * c / lambda_m / (me * c * c)


def qed_h(chi):
    return lib().orc_qed_h(float(chi))


def qed_power(chi):
    return lib().orc_qed_power(float(chi))


def qed_T(chi):
    return lib().orc_qed_T(float(chi))


def qed_em_density(chi, xi):
    return lib().orc_qed_em_density(float(chi), float(xi))


def qed_pair_density(chi, xi):
    return lib().orc_qed_pair_density(float(chi), float(xi))


def qed_em_sample(chi, r):
    return lib().orc_qed_em_sample(float(chi), float(r))


def qed_pair_sample(chi, r):
    return lib().orc_qed_pair_sample(float(chi), float(r))


def chi_param(kappa, e, b, u, photon=False):
    e = np.ascontiguousarray(e, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_chi(float(kappa), _ptr(e), _ptr(b), _ptr(u), int(photon))


def derived_id(pid, step, tag):
    return lib().orc_derived_id(int(pid), int(step), int(tag))


def qed_tau0(ids, seed, sp_index):
    return np.array([lib().orc_qed_tau0(int(i), int(seed) & 0xFFFFFFFF, int(sp_index)) for i in ids])


def _empty(n, q, m):
    out = Particles(q, m, *([np.zeros(n)] * 7))
    out.ids = np.zeros(n, dtype=np.uint64)
    return out


def qed_emit(sp, kappa, dt, eps_min, seed, sp_index, step):
    """Emission pass over `sp` (uses sp.eb and sp.tau).  Returns
    (photon Particles with .tau, energy of photons not kept, number of events)."""
    cap = sp.n
    ph = _empty(cap, 0.0, 0.0)
    ph_tau = np.zeros(cap)
    tal = np.zeros(2)
    s, so = sp.cstruct(), ph.cstruct()
    n = lib().orc_qed_emit(C.byref(s), _ptr(sp.tau), float(kappa), float(dt), float(eps_min),
                           int(seed) & 0xFFFFFFFF, int(sp_index), int(step), C.byref(so), _ptr(ph_tau), cap, _ptr(tal))
    ph.select(np.arange(n))
    ph.tau = np.ascontiguousarray(ph_tau[:n])
    return ph, tal[0], int(tal[1])


def gather_species(g, E, B, sp):
    """Fill sp.eb with E, B at the particle positions."""
    sp.eb = np.zeros((sp.n, 6))
    s = sp.cstruct()
    lib().orc_gather_species(C.byref(g), _f3(E), _f3(B), C.byref(s))


def photon_move(g, sp):
    s = sp.cstruct()
    lib().orc_photon_move(C.byref(g), C.byref(s))


def qed_pairs(ph, kappa, dt, seed, sp_index, step):
    """Pair pass over photons (uses ph.eb, ph.tau); removes converted photons.
    Returns (electrons, positrons, energy deficit, events)."""
    cap = ph.n
    el, po = _empty(cap, -1.0, 1.0), _empty(cap, 1.0, 1.0)
    el_tau, po_tau = np.zeros(cap), np.zeros(cap)
    alive = np.ones(cap, dtype=np.uint8)
    tal = np.zeros(2)
    s, se, sq = ph.cstruct(), el.cstruct(), po.cstruct()
    n = lib().orc_qed_pairs(C.byref(s), _ptr(ph.tau), _ptr(alive), float(kappa), float(dt), int(seed) & 0xFFFFFFFF,
                            int(sp_index), int(step), C.byref(se), _ptr(el_tau), C.byref(sq), _ptr(po_tau), cap,
                            _ptr(tal))
    for o, t in ((el, el_tau), (po, po_tau)):
        o.select(np.arange(n))
        o.tau = np.ascontiguousarray(t[:n])
    ph.select(alive.astype(bool))
    return el, po, tal[0], int(tal[1])


# --------------------------------------------------------------------------- cold fluid
class Fluid:
    """A fluid species on the nodes: density n [n_c] and u = gamma beta; cold,
    or with the adiabatic pressure p = K n^gamma_ad (K [m_e c^2 n_c^(1 - gamma_ad)])."""

    def __init__(self, q, m, n, u=None, n_floor=1e-10, K=0.0, gamma_ad=5.0 / 3.0):
        self.q, self.m, self.n_floor = float(q), float(m), float(n_floor)
        self.K, self.gamma_ad = float(K), float(gamma_ad)
        self.n = np.ascontiguousarray(n, dtype=np.float64).copy()
        self.u = (np.zeros((3,) + self.n.shape) if u is None
                  else np.ascontiguousarray(u, dtype=np.float64).copy())


def node_fields(g, E, B, i, j, k):
    e = np.zeros(3)
    b = np.zeros(3)
    lib().orc_node_fields(C.byref(g), _f3(E), _f3(B), int(i), int(j), int(k), _ptr(e), _ptr(b))
    return e, b


def fluid_step(g, E, B, J, fl):
    """One fluid step; adds the face currents to J.  Returns the number of clamped nodes."""
    return lib().orc_fluid_step(C.byref(g), _f3(E), _f3(B), _f3(J), fl.q, fl.m, _ptr(fl.n), _f3(fl.u),
                                fl.n_floor, fl.K, fl.gamma_ad)


def fluid_energy(g, fl):
    return lib().orc_fluid_energy(C.byref(g), fl.m, _ptr(fl.n), _f3(fl.u))


# --------------------------------------------------------------------------- regime switching
REGIME_DEFAULTS = dict(a_thr=1.0, n_thr=1.0, c_thr=0.1, chi_thr=1e-3, dilate=2)


def regime_criterion(g, E, B, ne, fluid_u=None, kappa=None, lambda_m=0.8e-6, **thr):
    """Physics criterion mask (1 = kinetic) at the nodes, dilated."""
    t = dict(REGIME_DEFAULTS)
    t.update(thr)
    kappa = qed_kappa(lambda_m) if kappa is None else kappa
    ne = np.ascontiguousarray(ne, dtype=np.float64)
    mask = np.zeros(g.shape, dtype=np.uint8)
    fu = None if fluid_u is None else _f3(np.ascontiguousarray(fluid_u, dtype=np.float64))
    lib().orc_regime_criterion(C.byref(g), _f3(E), _f3(B), _ptr(ne), fu, float(kappa), float(t["a_thr"]),
                               float(t["n_thr"]), float(t["c_thr"]), float(t["chi_thr"]), int(t["dilate"]),
                               _ptr(mask))
    return mask


def fluid_to_particles(g, mask, fl, ppc, seed, sp_index, epoch, rho_bg, quiet=False):
    """Convert the fluid at kinetic nodes into particles (returns Particles):
    Philox-uniform positions in the node's dual cell, or with quiet=True the
    centres of an lx x ly x lz sub-lattice of it."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    cap = int(np.count_nonzero(mask)) * ppc
    out = _empty(max(cap, 1), fl.q, fl.m)
    n = lib().orc_fluid_to_particles(C.byref(g), _ptr(mask), fl.q, _ptr(fl.n), _f3(fl.u), fl.n_floor, int(ppc),
                                     int(seed) & 0xFFFFFFFF, int(sp_index), int(epoch), C.byref(out.cstruct()),
                                     max(cap, 1), _ptr(rho_bg), int(bool(quiet)))
    out.select(np.arange(n))
    return out


def particles_to_fluid(g, mask, sp, fl):
    """Move the particles whose nearest node is fluid into the fluid; returns the count."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    alive = np.ones(max(sp.n, 1), dtype=np.uint8)
    n = lib().orc_particles_to_fluid(C.byref(g), _ptr(mask), C.byref(sp.cstruct()), _ptr(fl.n), _f3(fl.u),
                                     fl.n_floor, _ptr(alive))
    sp.select(alive[:sp.n].astype(bool))
    return n


def dropout_mask(B, C_, V, seed, pass_index, layer, p, cells=None):
    """uint8 keep mask [B][C][V] of the classifier's dropout; `cells` (int64,
    V values) names the cell whose stream each position takes (default:
    position v is cell v)."""
    keep = np.zeros((B, C_, V), dtype=np.uint8)
    if cells is None:
        lib().orc_dropout_mask(_ptr(keep), int(B), int(C_), int(V), int(seed) & 0xFFFFFFFF, int(pass_index),
                               int(layer), float(p))
    else:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        assert cells.size == V
        lib().orc_dropout_mask_cells(_ptr(keep), int(B), int(C_), int(V), _ptr(cells), int(seed) & 0xFFFFFFFF,
                                     int(pass_index), int(layer), float(p))
    return keep
