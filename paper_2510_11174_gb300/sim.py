"""Thin Python front end over the C ABI (include/hyb.h).

Argument marshalling only: arrays are handed to libhyb.so as host pointers
(numpy) or device pointers (torch CUDA tensors); PyTorch provides the CUDA
stream the context runs on.  Every step of the method runs in the library.
"""
import ctypes as C

import numpy as np

from . import _abi
from ._abi import check


def _torch():
    import torch
    return torch


def _ptr_and_dev(a, dtype):
    """Return (pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, False, None
    if isinstance(a, np.ndarray):
        arr = np.ascontiguousarray(a, dtype=dtype)
        return arr.ctypes.data, False, arr
    torch = _torch()
    if isinstance(a, torch.Tensor):
        tdt = {np.float32: torch.float32, np.uint64: torch.int64}[dtype]
        t = a.contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        if t.is_cuda:
            # the context runs on its own stream: make the producer's work visible
            torch.cuda.current_stream(t.device).synchronize()
        return t.data_ptr(), t.is_cuda, t
    arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return arr.ctypes.data, False, arr


class Simulation:
    """One hybrid fluid-kinetic context on the current CUDA device.

    Geometry: nx*ny*nz cells of size (dx, dy, dz) [c/w0]; bc per axis
    0 = periodic, 1 = Mur + reflecting walls.  dt <= 0 picks cfl_frac times the
    Courant limit.  ``laser`` is None or a dict with keys a0, tau_fwhm, w0_spot,
    t_peak, y_c, z_c, x_src, pol (Gaussian soft source).
    """

    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, dt=0.0, cfl_frac=0.95, bc=(0, 0, 0),
                 lambda_um=0.8, laser=None, seed=1, tile=8, stream=None, arena=None, shape_order=1):
        self._lib = _abi.load()
        d = _abi.hyb_grid_desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.dx = dx
        d.dy = dx if dy is None else dy
        d.dz = dx if dz is None else dz
        d.dt, d.cfl_frac = dt, cfl_frac
        for a in range(3):
            d.bc[a] = bc[a]
        d.lambda_um = lambda_um
        if laser:
            d.laser_kind = _abi.HYB_LASER_GAUSS
            for k in ("a0", "tau_fwhm", "w0_spot", "t_peak", "y_c", "z_c"):
                setattr(d, k, float(laser[k]))
            d.x_src, d.pol = int(laser["x_src"]), int(laser.get("pol", 1))
        d.seed = seed
        d.tile = tile
        d.shape_order = shape_order
        self.torch_stream = None
        if stream is None:
            # the legacy default stream cannot be captured into a CUDA graph:
            # run on torch's current stream unless that is the default one
            torch = _torch()
            cur = torch.cuda.current_stream()
            if cur.cuda_stream == 0:
                cur = torch.cuda.Stream()
            self.torch_stream = cur
            stream = cur.cuda_stream
        d.stream = stream
        self._arena = arena
        if arena is not None:
            d.arena_dev = arena.data_ptr()
            d.arena_bytes = arena.numel() * arena.element_size()
        self.desc = d
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        h = C.c_void_p()
        check(self._lib.hyb_init_grid(C.byref(d), C.byref(h)))
        self._ctx = h
        self.n_species = 0

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.hyb_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ set-up
    PUSHERS = {"boris": 0, "vay": 1, "higuera_cary": 2}

    def load_species(self, q, m, x, y, z, ux, uy, uz, w, zq=None, ids=None, tile_capacity=0, ionize=None,
                     kind=0, qed=None, pairs=None, pusher="boris"):
        """Add a species; returns its id.  ``ionize`` = dict(zmax, ip_eV, l, into)
        makes it field-ionizable (zq = charge states required); kind = 1 makes
        a photon species; ``qed`` = dict(photon_species, eps_min) turns on
        photon emission by a lepton species; ``pairs`` = dict(electron,
        positron) turns on pair creation by a photon species; ``pusher`` is
        "boris", "vay" or "higuera_cary"."""
        d = _abi.hyb_species_desc()
        d.q, d.m = q, m
        d.kind = int(kind)
        d.pusher = self.PUSHERS[pusher]
        d.photon_species = d.pair_electron = d.pair_positron = -1
        if qed:
            d.qed = 1
            d.photon_species = int(qed.get("photon_species", -1))
            d.photon_eps_min = float(qed.get("eps_min", 0.0))
        if pairs:
            d.pair_electron = int(pairs["electron"])
            d.pair_positron = int(pairs["positron"])
        if ionize:
            d.zmax = int(ionize["zmax"])
            for lev in range(d.zmax):
                d.ip_eV[lev] = float(ionize["ip_eV"][lev])
                d.l_qn[lev] = int(ionize["l"][lev])
            d.ionize_into = int(ionize["into"])
        keep = []
        ptrs = []
        on_dev = None
        n = len(x)
        for a in (x, y, z, ux, uy, uz, w, zq):
            if a is not None and (np.ndim(a) != 1 or len(a) != n):
                raise ValueError("particle arrays must be 1-D and of equal length")
            p, dev, k = _ptr_and_dev(a, np.float32)
            keep.append(k)
            ptrs.append(p)
            if a is not None:
                on_dev = dev if on_dev is None else on_dev
                if dev != on_dev:
                    raise ValueError("particle arrays must all be host or all be device memory")
        pid, dev, k = _ptr_and_dev(ids, np.uint64)
        keep.append(k)
        if ids is not None and dev != on_dev:
            raise ValueError("ids must live where the particle arrays live")
        d.n = int(len(x))
        d.tile_capacity = int(tile_capacity)
        d.ptr_on_device = int(bool(on_dev))
        d.x, d.y, d.z, d.ux, d.uy, d.uz, d.w, d.zq = ptrs
        d.ids = pid
        sid = C.c_int()
        check(self._lib.hyb_load_species(self._ctx, C.byref(d), C.byref(sid)))
        self.n_species += 1
        return sid.value

    def load_fluid(self, q, m, n, ux=None, uy=None, uz=None, n_floor=0.0, temperature_keV=0.0, gamma_ad=0.0,
                   n_ref=0.0):
        """Add a fluid species (node arrays shaped (nz, ny, nx)); returns its id.
        temperature_keV > 0 makes it warm: p = n_ref T (n / n_ref)^gamma_ad."""
        d = _abi.hyb_fluid_desc()
        d.q, d.m, d.n_floor = q, m, n_floor
        d.temperature_keV, d.gamma_ad, d.n_ref = temperature_keV, gamma_ad, n_ref
        keep = []
        ptrs = []
        on_dev = None
        for a in (n, ux, uy, uz):
            if a is not None and np.size(a) != self.N:
                raise ValueError("fluid arrays must hold nz*ny*nx values")
            p, dev, k = _ptr_and_dev(a, np.float32)
            keep.append(k)
            ptrs.append(p)
            if a is not None:
                on_dev = dev if on_dev is None else on_dev
                if dev != on_dev:
                    raise ValueError("fluid arrays must all be host or all be device memory")
        d.ptr_on_device = int(bool(on_dev))
        d.n, d.ux, d.uy, d.uz = ptrs
        fid = C.c_int()
        check(self._lib.hyb_load_fluid(self._ctx, C.byref(d), C.byref(fid)))
        return fid.value

    POLICIES = {"default": _abi.HYB_REGIME_DEFAULT, "union": _abi.HYB_REGIME_UNION,
                "all_kinetic": _abi.HYB_REGIME_ALL_KINETIC}

    def set_regime(self, a_thr=1.0, n_thr=1.0, c_thr=0.1, chi_thr=1e-3, dilate=2, k_sigma=1.0, ppc=8,
                   to_species=None, policy="default", quiet=False, reach=0):
        """Thresholds and conversion targets of hyb_classify; policy is
        "default" (classifier if given, else physics criterion), "union"
        (classifier or criterion) or "all_kinetic" (full PIC); quiet=True
        places converted particles on a sub-lattice of the node's dual cell;
        reach > 0 runs the classifier only within reach + dilate nodes (in x)
        of matter (exact when the next classification is at most reach - 1
        steps away)."""
        d = _abi.hyb_regime_desc()
        d.policy = self.POLICIES[policy]
        d.quiet = int(bool(quiet))
        d.reach = int(reach)
        d.a_thr, d.n_thr, d.c_thr, d.chi_thr = a_thr, n_thr, c_thr, chi_thr
        d.dilate, d.k_sigma, d.ppc = dilate, k_sigma, ppc
        ts = list(to_species or [])
        for f in range(_abi.HYB_MAX_FLUIDS):
            d.to_species[f] = int(ts[f]) if f < len(ts) else -1
        check(self._lib.hyb_set_regime(self._ctx, C.byref(d)))

    def classify(self, model=None, p_mean=None, p_std=None):
        """Recompute the regime mask (physics criterion, or the classifier
        `model`) and convert fluid <-> particles.  p_mean / p_std: optional
        torch CUDA tensors of nz*ny*nx FP32 values receiving the MC statistics."""
        ptr = lambda t: None if t is None else t.data_ptr()
        check(self._lib.hyb_classify(self._ctx, None if model is None else model.handle, ptr(p_mean), ptr(p_std),
                                     None))
        if (p_mean is not None or p_std is not None) and self.torch_stream is not None:
            # the outputs are written on the context's stream: order torch's
            # current stream (their consumer) after it
            torch = _torch()
            torch.cuda.current_stream().wait_stream(self.torch_stream)

    def node_fields(self, out=None):
        """The classifier's six input channels at the nodes, not normalised
        (hyb_node_fields): a torch CUDA tensor [6, nz, ny, nx]."""
        torch = _torch()
        if out is None:
            out = torch.empty((6,) + self.shape, dtype=torch.float32, device="cuda")
        check(self._lib.hyb_node_fields(self._ctx, out.data_ptr()))
        if self.torch_stream is not None:
            torch.cuda.current_stream().wait_stream(self.torch_stream)
        return out

    def node_state(self, out=None):
        """The surrogate's ten channels at the nodes (hyb_node_state): E, B,
        J averaged to the nodes and the charge density; a torch CUDA tensor
        [10, nz, ny, nx]."""
        torch = _torch()
        if out is None:
            out = torch.empty((10,) + self.shape, dtype=torch.float32, device="cuda")
        check(self._lib.hyb_node_state(self._ctx, out.data_ptr()))
        if self.torch_stream is not None:
            torch.cuda.current_stream().wait_stream(self.torch_stream)
        return out

    def get_regime(self):
        mask = np.empty(self.shape, np.uint8)
        rho_bg = np.empty(self.shape, np.float32)
        check(self._lib.hyb_get_regime(self._ctx, mask.ctypes.data, rho_bg.ctypes.data))
        return mask, rho_bg

    def get_fluid(self, fid):
        out = {k: np.empty(self.shape, np.float32) for k in ("n", "ux", "uy", "uz")}
        check(self._lib.hyb_get_fluid(self._ctx, int(fid), *[out[k].ctypes.data for k in ("n", "ux", "uy", "uz")]))
        return out

    def set_fields(self, E, B):
        pe, de, ke = _ptr_and_dev(E, np.float32)
        pb, db, kb = _ptr_and_dev(B, np.float32)
        if de != db:
            raise ValueError("E and B must both be host or both be device memory")
        check(self._lib.hyb_set_fields(self._ctx, pe, pb, int(de)))

    # ------------------------------------------------------------------ stepping
    def step(self, n=1):
        check(self._lib.hyb_step(self._ctx, int(n)))

    def set_profiling(self, on=True):
        check(self._lib.hyb_set_profiling(self._ctx, int(bool(on))))

    def phase_times(self):
        """Device milliseconds of each phase of the most recent step (synchronises)."""
        out = _abi.hyb_phase_times_t()
        check(self._lib.hyb_phase_times(self._ctx, C.byref(out)))
        return {name: out.ms[i] for i, name in enumerate(_abi.PHASES) if out.ms[i] > 0}

    def clear_status(self):
        check(self._lib.hyb_clear_status(self._ctx))

    def get_state(self):
        """The context's whole state as a byte image (hyb_get_state); a numpy uint8 array."""
        size = C.c_size_t()
        check(self._lib.hyb_get_state(self._ctx, None, 0, C.byref(size)))
        buf = np.empty(size.value, np.uint8)
        check(self._lib.hyb_get_state(self._ctx, buf.ctypes.data, buf.size, C.byref(size)))
        return buf

    def set_state(self, image):
        """Restore an image of get_state (hyb_set_state) into this context."""
        buf = np.ascontiguousarray(image, dtype=np.uint8)
        check(self._lib.hyb_set_state(self._ctx, buf.ctypes.data, buf.size))

    def set_auto_grow(self, on=True):
        """Turn the growth of full particle tiles on or off (hyb_set_auto_grow)."""
        check(self._lib.hyb_set_auto_grow(self._ctx, int(bool(on))))

    def selftest_wait_timeout(self, polls=4096):
        """Run the bounded-wait self-test (hyb_selftest_wait_timeout): latches HYB_ETIMEOUT."""
        check(self._lib.hyb_selftest_wait_timeout(self._ctx, int(polls)))

    # ------------------------------------------------------------------ read-back
    def diagnostics(self, raise_on_status=True):
        out = _abi.hyb_diag()
        code = self._lib.hyb_diagnostics(self._ctx, C.byref(out))
        if raise_on_status:
            check(code)
        ns = out.n_species
        return {"step": out.step, "time": out.time, "w_e": out.w_e, "w_b": out.w_b,
                "w_kin": [out.w_kin[i] for i in range(ns)], "count": [out.count[i] for i in range(ns)],
                "status": out.status, "launches_per_step": out.launches_per_step,
                "w_ionize": out.w_ionize, "n_ionize": out.n_ionize,
                "w_photon_untracked": out.w_photon_untracked, "w_pair_deficit": out.w_pair_deficit,
                "n_emit": out.n_emit, "n_pair": out.n_pair,
                "w_fluid": [out.w_fluid[i] for i in range(out.n_fluids)],
                "n_fluid": [out.n_fluid[i] for i in range(out.n_fluids)], "n_clamped": out.n_clamped,
                "launches_classify": out.launches_classify,
                "classified_cells": out.classified_cells,
                "fluid_cells": out.fluid_cells,
                "tile_capacity": [out.tile_capacity[i] for i in range(ns)]}

    def eval_qed(self, what, chi, r=None):
        """Evaluate the device QED tables (see hyb_eval_qed)."""
        ca = np.ascontiguousarray(chi, dtype=np.float32)
        ra = None if r is None else np.ascontiguousarray(r, dtype=np.float32)
        out = np.empty_like(ca)
        check(self._lib.hyb_eval_qed(self._ctx, int(what), ca.ctypes.data, None if ra is None else ra.ctypes.data,
                                     len(ca), out.ctypes.data))
        return out

    def eval_rate_table(self, table, species_id, level, x):
        """Evaluate a device rate table at the points x (see hyb_eval_rate_table)."""
        xa = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty_like(xa)
        check(self._lib.hyb_eval_rate_table(self._ctx, int(table), int(species_id), int(level),
                                            xa.ctypes.data, len(xa), out.ctypes.data))
        return out

    def get_fields(self):
        E = np.empty((3,) + self.shape, np.float32)
        B = np.empty((3,) + self.shape, np.float32)
        J = np.empty((3,) + self.shape, np.float32)
        check(self._lib.hyb_get_fields(self._ctx, E.ctypes.data, B.ctypes.data, J.ctypes.data))
        return E, B, J

    def get_species(self, sid, with_zq=False, max_n=None):
        if max_n is None:
            max_n = self.diagnostics(raise_on_status=False)["count"][sid]
        arrs = {k: np.empty(max_n, np.float32) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
        arrs["zq"] = np.empty(max_n, np.float32) if with_zq else None
        ids = np.empty(max_n, np.uint64)
        n = C.c_longlong()
        check(self._lib.hyb_get_species(
            self._ctx, sid, max_n, *[arrs[k].ctypes.data if arrs[k] is not None else None
                                     for k in ("x", "y", "z", "ux", "uy", "uz", "w", "zq")],
            ids.ctypes.data, C.byref(n)))
        out = {k: v[:n.value] for k, v in arrs.items() if v is not None}
        out["ids"] = ids[:n.value]
        return out


class Batch:
    """Independent Simulations advanced together (hyb_batch_*): one CUDA graph
    per step with one branch per simulation.  ``stream``: a torch CUDA stream
    or raw stream handle for the batch (default: the first simulation's)."""

    def __init__(self, sims, stream=None):
        self._lib = _abi.load()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s._ctx for s in self.sims])
        if stream is None:
            stream = self.sims[0].desc.stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        h = C.c_void_p()
        check(self._lib.hyb_batch_create(arr, len(self.sims), stream, C.byref(h)))
        self._b = h

    def step(self, n=1):
        check(self._lib.hyb_batch_step(self._b, int(n)))

    def close(self):
        if getattr(self, "_b", None):
            self._lib.hyb_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
