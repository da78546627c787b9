// C ABI of the hybrid fluid-kinetic step: context creation, species loading,
// the step sequence (captured once into a CUDA graph and replayed), and the
// synchronising read-back calls.  See include/hyb.h for the contract.
//
// Step order (arXiv 2510.11174, Methodology: time loop of laser excitation,
// ionization, particle movement, fluid changes and field modification):
//   1. push + gather + Esirkepov deposit of every species (J^{n+1/2})
//   2. assemble J from the tile frames; add the laser source current
//   3. re-insert particles that changed tile; compact vacated slots
//   4. B half step, E full step with J, Mur faces, B half step
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hyb_internal.cuh"

namespace hyb {

static constexpr int GROW_CHECK_STEPS = 4;  // steps between checks of the tile fill

static thread_local std::string g_err = "no error";

hyb_status set_error(hyb_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

cudaError_t ctx_alloc(hyb_ctx *c, void **p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (c->arena.base) {
        if (c->arena.used + bytes > c->arena.size) return cudaErrorMemoryAllocation;
        *p = c->arena.base + c->arena.used;
        c->arena.used += bytes;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) c->owned.push_back(*p);
    return e;
}

SpSet species_set(const hyb_ctx *c) {
    SpSet s;
    memset(&s, 0, sizeof(s));
    s.n = (int)c->sp.size();
    for (int i = 0; i < s.n; ++i) s.s[i] = c->sp[i].dev;
    return s;
}

static hyb_status status_to_code(int st) {
    if (st & ST_OVERFLOW) return HYB_EOVERFLOW;
    if (st & ST_NAN) return HYB_ENAN;
    if (st & ST_TIMEOUT) return HYB_ETIMEOUT;
    if (st & ST_BADPOS) return HYB_EINVAL;
    return HYB_OK;
}

// phase boundary markers (event records captured into the step graph)
struct PhaseMark {
    hyb_ctx *c;
    void begin(int ph) {
        c->phase_ran[ph] = true;
        // External: during stream capture this becomes an event-record node that
        // records at every replay (a plain record would only order the capture)
        if (c->profiling) cudaEventRecordWithFlags(c->ev_start[ph], c->stream, cudaEventRecordExternal);
    }
    void end(int ph) {
        if (c->profiling) cudaEventRecordWithFlags(c->ev_end[ph], c->stream, cudaEventRecordExternal);
    }
};

// Enqueue one full step on the context stream.
static void enqueue_step(hyb_ctx *c) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const SpSet set = species_set(c);
    PhaseMark pm{c};
    for (int p = 0; p < HYB_PH_CLASSIFY; ++p) c->phase_ran[p] = false;
    cudaMemsetAsync(c->mig_counts, 0, sizeof(int) * HYB_MAX_SPECIES, st);
    if (set.n > 0) {
        pm.begin(HYB_PH_PUSH);
        launch_push_deposit(g, c->E, c->B, c->sp_dev, set.n, c->qed, c->jscratch, c->jvalid, c->status, c->step_dev,
                            st);
        pm.end(HYB_PH_PUSH);
        pm.begin(HYB_PH_JREDUCE);
        launch_j_reduce(g, c->jscratch, c->jvalid, c->J, st);
        pm.end(HYB_PH_JREDUCE);
    } else {
        cudaMemsetAsync(c->J, 0, sizeof(float) * 3 * g.N, st);
    }
    const bool fluid_phase = !c->fluids.empty() && !c->fluids_idle;
    if (fluid_phase) {
        pm.begin(HYB_PH_FLUID);
        launch_fluids(g, c->E, c->B, c->fluids.data(), (int)c->fluids.size(), c->J, c->fluid_xr, st);
        pm.end(HYB_PH_FLUID);
    }
    if (c->desc.laser_kind == HYB_LASER_GAUSS) {
        pm.begin(HYB_PH_SOURCE);
        launch_laser_source(g, c->desc, c->laser_profile, c->step_dev, c->J, st);
        pm.end(HYB_PH_SOURCE);
    }
    if (set.n > 0) {
        pm.begin(HYB_PH_REBIN);
        for (int s = 0; s < set.n; ++s) {
            launch_rebin(g, set.s[s], c->status, st);
            launch_compact(g, set.s[s], st);
        }
        pm.end(HYB_PH_REBIN);
    }
    pm.begin(HYB_PH_FIELD);
    launch_fdtd_b_half(g, c->E, c->B, st);
    launch_fdtd_e(g, c->E, c->B, c->J, st);
    launch_mur(g, c->E, c->mur_old, c->mur_plane, st);
    launch_fdtd_b_half(g, c->E, c->B, st);
    pm.end(HYB_PH_FIELD);
    launch_step_inc(c->step_dev, st);

    // kernels enqueued above (memsets and event records are not kernels)
    long long k = 0;
    if (set.n > 0) k += 2 + 2LL * set.n;
    if (fluid_phase) k += 2;
    if (c->desc.laser_kind == HYB_LASER_GAUSS) k += 1;
    k += 3 + ((g.bc[0] || g.bc[1] || g.bc[2]) ? 3 : 0) + 1;
    c->launches_per_step = k;
}

// the per-slot arrays (particles, hole list) and the migration buffer of a
// species with `cap` slots per tile
hyb_status alloc_slots(hyb_ctx *c, SpDev &s, int cap, bool has_zq, bool has_tau) {
    const size_t slots = (size_t)cap * c->g.ntiles;
    s.cap = cap;
    s.zq = s.tau = s.mzq = s.mtau = nullptr;
    float **fl[7] = {&s.x, &s.y, &s.z, &s.ux, &s.uy, &s.uz, &s.w};
    for (auto f : fl)
        if (ctx_alloc(c, (void **)f, sizeof(float) * slots)) return HYB_ENOMEM;
    if (has_zq && ctx_alloc(c, (void **)&s.zq, sizeof(float) * slots)) return HYB_ENOMEM;
    if (has_tau && ctx_alloc(c, (void **)&s.tau, sizeof(float) * slots)) return HYB_ENOMEM;
    if (ctx_alloc(c, (void **)&s.id, sizeof(uint64_t) * slots) || ctx_alloc(c, (void **)&s.holes, sizeof(int) * slots))
        return HYB_ENOMEM;
    // a particle moves less than one cell per step, so only the shell of a tile can leave it
    const long long mig = std::min<long long>((long long)slots, std::max<long long>(65536, (long long)slots / 2));
    s.mig_cap = (int)std::min<long long>(mig, 0x7fffffffLL);
    float **ml[7] = {&s.mx, &s.my, &s.mz, &s.mux, &s.muy, &s.muz, &s.mw};
    for (auto f : ml)
        if (ctx_alloc(c, (void **)f, sizeof(float) * s.mig_cap)) return HYB_ENOMEM;
    if (has_zq && ctx_alloc(c, (void **)&s.mzq, sizeof(float) * s.mig_cap)) return HYB_ENOMEM;
    if (has_tau && ctx_alloc(c, (void **)&s.mtau, sizeof(float) * s.mig_cap)) return HYB_ENOMEM;
    if (ctx_alloc(c, (void **)&s.mid, sizeof(uint64_t) * s.mig_cap) ||
        ctx_alloc(c, (void **)&s.mdest, sizeof(int) * s.mig_cap))
        return HYB_ENOMEM;
    return HYB_OK;
}

// release a buffer of the context (buffers carved from a caller's arena stay
// until the context is destroyed)
static void ctx_free(hyb_ctx *c, void *p) {
    if (!p || c->arena.base) return;
    for (auto it = c->owned.begin(); it != c->owned.end(); ++it)
        if (*it == p) {
            c->owned.erase(it);
            cudaFree(p);
            return;
        }
}

void free_slots(hyb_ctx *c, const SpDev &s) {
    void *ps[] = {s.x, s.y, s.z, s.ux, s.uy, s.uz, s.w, s.zq, s.tau, s.id, s.holes,
                  s.mx, s.my, s.mz, s.mux, s.muy, s.muz, s.mw, s.mzq, s.mtau, s.mid, s.mdest};
    for (void *p : ps) ctx_free(c, p);
}

}  // namespace hyb

using namespace hyb;

extern "C" {

static hyb_status read_status(hyb_ctx *c);

const char *hyb_last_error(void) { return g_err.c_str(); }

hyb_status hyb_init_grid(const hyb_grid_desc *d, hyb_ctx **out) {
    if (!d || !out) return set_error(HYB_EINVAL, "null descriptor or output");
    *out = nullptr;
    const int n[3] = {d->nx, d->ny, d->nz};
    const double dd[3] = {d->dx, d->dy, d->dz};
    const int T = d->tile == 0 ? 8 : d->tile;
    if (T != 4 && T != 8) return set_error(HYB_EINVAL, "tile must be 4 or 8");
    for (int a = 0; a < 3; ++a) {
        if (n[a] <= 0 || n[a] % T != 0)
            return set_error(HYB_EINVAL, "grid size must be a positive multiple of the tile edge");
        if (!(dd[a] > 0.0)) return set_error(HYB_EINVAL, "cell size must be positive");
        if (d->bc[a] != HYB_BC_PERIODIC && d->bc[a] != HYB_BC_MUR) return set_error(HYB_EINVAL, "bad boundary");
        if (d->bc[a] == HYB_BC_MUR && n[a] < 4) return set_error(HYB_EINVAL, "Mur axis needs >= 4 nodes");
    }
    const double courant = 1.0 / std::sqrt(1.0 / (dd[0] * dd[0]) + 1.0 / (dd[1] * dd[1]) + 1.0 / (dd[2] * dd[2]));
    double dt = d->dt;
    if (!(dt > 0.0)) {
        if (!(d->cfl_frac > 0.0 && d->cfl_frac < 1.0)) return set_error(HYB_EINVAL, "need dt or cfl_frac in (0,1)");
        dt = d->cfl_frac * courant;
    }
    if (dt >= courant) return set_error(HYB_EINVAL, "dt at or above the Courant limit");
    const int order = d->shape_order == 0 ? 1 : d->shape_order;
    if (order != 1 && order != 2) return set_error(HYB_EINVAL, "shape_order must be 1 or 2");
    if (order == 2 && (d->bc[0] || d->bc[1] || d->bc[2]))
        return set_error(HYB_EINVAL, "the quadratic shape needs periodic axes");
    if (d->laser_kind == HYB_LASER_GAUSS) {
        if (d->x_src < 0 || d->x_src >= n[0]) return set_error(HYB_EINVAL, "laser x_src outside the grid");
        if (d->pol != 1 && d->pol != 2) return set_error(HYB_EINVAL, "laser pol must be 1 (y) or 2 (z)");
        if (!(d->tau_fwhm > 0.0) || !(d->w0_spot > 0.0)) return set_error(HYB_EINVAL, "laser tau and w0 must be > 0");
    } else if (d->laser_kind != HYB_LASER_NONE) {
        return set_error(HYB_EINVAL, "bad laser kind");
    }

    hyb_ctx *c = new hyb_ctx();
    c->desc = *d;
    c->desc.dt = dt;
    c->desc.tile = T;
    GridDev &g = c->g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = n[a];
        g.bc[a] = d->bc[a];
        g.nt[a] = n[a] / T;
        g.d[a] = (float)dd[a];
        g.dd[a] = dd[a];
    }
    g.T = T;
    g.tshift = T == 8 ? 3 : 2;
    g.ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    g.N = (long long)n[0] * n[1] * n[2];
    g.dt = (float)dt;
    g.dt_d = dt;
    g.seed = d->seed;
    g.order = order;

    if (d->stream) {
        c->stream = (cudaStream_t)d->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return set_error(HYB_ECUDA, std::string("stream create: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    if (d->arena_dev) {
        c->arena.base = (char *)d->arena_dev;
        c->arena.size = d->arena_bytes;
    }

    auto fail = [&](hyb_status s, const std::string &m) {
        hyb_destroy(c);
        return set_error(s, m);
    };
    const size_t fbytes = sizeof(float) * 3 * (size_t)g.N;
    c->mur_plane = std::max({(long long)n[1] * n[2], (long long)n[0] * n[2], (long long)n[0] * n[1]});
    // 3 current components (of the shape order's frame) in the step, 4 CIC moments in a conversion
    const long long G1 = T + 3, Gk = T + 2 * order + 1;
    c->jframe = std::max(4 * G1 * G1 * G1, 3 * Gk * Gk * Gk);
    c->red_blocks = 152 * 8;   // enough warps for the loads of the reductions to cover the memory latency
    if (ctx_alloc(c, (void **)&c->E, fbytes) || ctx_alloc(c, (void **)&c->B, fbytes) ||
        ctx_alloc(c, (void **)&c->J, fbytes) ||
        ctx_alloc(c, (void **)&c->mur_old, sizeof(float) * 24 * (size_t)c->mur_plane) ||
        ctx_alloc(c, (void **)&c->jscratch, sizeof(float) * (size_t)c->jframe * g.ntiles) ||
        ctx_alloc(c, (void **)&c->jvalid, sizeof(int) * (size_t)g.ntiles) ||
        ctx_alloc(c, (void **)&c->red_partials, sizeof(double) * (2 + HYB_MAX_SPECIES + 2 * HYB_MAX_FLUIDS) * c->red_blocks) ||
        ctx_alloc(c, (void **)&c->red_out, sizeof(double) * (2 + HYB_MAX_SPECIES + 2 * HYB_MAX_FLUIDS)) ||
        ctx_alloc(c, (void **)&c->diag_dev, sizeof(DiagSummary)) ||
        ctx_alloc(c, (void **)&c->status, sizeof(int)) || ctx_alloc(c, (void **)&c->step_dev, sizeof(long long)) ||
        ctx_alloc(c, (void **)&c->mig_counts, sizeof(int) * HYB_MAX_SPECIES) ||
        ctx_alloc(c, (void **)&c->fill_flags, sizeof(int)) ||
        ctx_alloc(c, (void **)&c->sp_dev, sizeof(SpDev) * HYB_MAX_SPECIES) ||
        ctx_alloc(c, (void **)&c->mask, (size_t)g.N) || ctx_alloc(c, (void **)&c->mask_tmp, (size_t)g.N) ||
        ctx_alloc(c, (void **)&c->mask_prev, (size_t)g.N) ||
        ctx_alloc(c, (void **)&c->rho_bg, sizeof(float) * (size_t)g.N) ||
        ctx_alloc(c, (void **)&c->ne, sizeof(float) * (size_t)g.N) ||
        ctx_alloc(c, (void **)&c->fluid_xr, 2 * sizeof(int)))
        return fail(HYB_ENOMEM, "device allocation for the grid failed (arena too small?)");
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->E, 0, fbytes, st);
    cudaMemsetAsync(c->B, 0, fbytes, st);
    cudaMemsetAsync(c->J, 0, fbytes, st);
    cudaMemsetAsync(c->mur_old, 0, sizeof(float) * 24 * (size_t)c->mur_plane, st);
    cudaMemsetAsync(c->status, 0, sizeof(int), st);
    cudaMemsetAsync(c->step_dev, 0, sizeof(long long), st);
    cudaMemsetAsync(c->mask, 0, (size_t)g.N, st);  // no node has switched to kinetic before a classification
    cudaMemsetAsync(c->fill_flags, 0, sizeof(int), st);
    cudaMemsetAsync(c->fluid_xr, 0, 2 * sizeof(int), st);  // every plane
    if (cudaMallocHost((void **)&c->fill_host, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&c->fluid_xr_host, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&c->diag_host, sizeof(DiagSummary)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fill_ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(HYB_ENOMEM, "pinned fill flag");
    *c->fill_host = 0;
    cudaMemsetAsync(c->rho_bg, 0, sizeof(float) * (size_t)g.N, st);
    c->regime.a_thr = 1.0;
    c->regime.n_thr = 1.0;
    c->regime.c_thr = 0.1;
    c->regime.chi_thr = 1e-3;
    c->regime.dilate = 2;
    c->regime.k_sigma = 1.0;
    c->regime.ppc = 8;
    for (int f = 0; f < HYB_MAX_FLUIDS; ++f) c->regime.to_species[f] = -1;

    if (d->laser_kind == HYB_LASER_GAUSS) {
        // transverse profile f = exp(-r^2 / w0^2) at the J_pol positions of the source plane, FP64
        std::vector<float> prof((size_t)n[1] * n[2]);
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j) {
                const double y = (j + (d->pol == 1 ? 0.5 : 0.0) - d->y_c) * dd[1];
                const double z = (k + (d->pol == 2 ? 0.5 : 0.0) - d->z_c) * dd[2];
                prof[(size_t)k * n[1] + j] = (float)std::exp(-(y * y + z * z) / (d->w0_spot * d->w0_spot));
            }
        if (ctx_alloc(c, (void **)&c->laser_profile, sizeof(float) * prof.size()))
            return fail(HYB_ENOMEM, "laser profile allocation failed");
        cudaError_t e = cudaMemcpyAsync(c->laser_profile, prof.data(), sizeof(float) * prof.size(),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(HYB_ECUDA, std::string("laser profile upload: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(HYB_ECUDA, std::string("init: ") + cudaGetErrorString(e));
    *out = c;
    return HYB_OK;
}

void hyb_destroy(hyb_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_tmpl) cudaGraphDestroy(c->graph_tmpl);
    for (cudaEvent_t e : c->conv_ev) cudaEventDestroy(e);
    for (int p = 0; p < HYB_NPHASE; ++p) {
        if (c->ev_start[p]) cudaEventDestroy(c->ev_start[p]);
        if (c->ev_end[p]) cudaEventDestroy(c->ev_end[p]);
    }
    for (void *p : c->owned) cudaFree(p);
    if (c->fill_host) cudaFreeHost(c->fill_host);
    if (c->diag_host) cudaFreeHost(c->diag_host);
    if (c->xflag_host) cudaFreeHost(c->xflag_host);
    if (c->fluid_xr_host) cudaFreeHost(c->fluid_xr_host);
    if (c->fill_ev) cudaEventDestroy(c->fill_ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static hyb_status alloc_species(hyb_ctx *c, Species &sp, int cap, bool has_zq, bool has_tau) {
    const GridDev &g = c->g;
    SpDev &s = sp.dev;
    memset(&s, 0, sizeof(s));
    s.q = (float)sp.q;
    s.m = (float)sp.m;
    s.m_d = sp.m;
    if (alloc_slots(c, s, cap, has_zq, has_tau) != HYB_OK) return HYB_ENOMEM;
    if (ctx_alloc(c, (void **)&s.tal_e, sizeof(double) * NTALLY * g.ntiles) ||
        ctx_alloc(c, (void **)&s.tal_n, sizeof(unsigned long long) * NTALLY * g.ntiles))
        return HYB_ENOMEM;
    if (ctx_alloc(c, (void **)&s.count, sizeof(int) * g.ntiles) ||
        ctx_alloc(c, (void **)&s.hole_count, sizeof(int) * g.ntiles) ||
        ctx_alloc(c, (void **)&s.hole_used, sizeof(int) * g.ntiles))
        return HYB_ENOMEM;
    s.fill_flags = c->fill_flags;
    s.mig_count = c->mig_counts + c->sp.size();
    cudaMemsetAsync(s.count, 0, sizeof(int) * g.ntiles, c->stream);
    cudaMemsetAsync(s.hole_count, 0, sizeof(int) * g.ntiles, c->stream);
    cudaMemsetAsync(s.hole_used, 0, sizeof(int) * g.ntiles, c->stream);
    cudaMemsetAsync(s.tal_e, 0, sizeof(double) * NTALLY * g.ntiles, c->stream);
    cudaMemsetAsync(s.tal_n, 0, sizeof(unsigned long long) * NTALLY * g.ntiles, c->stream);
    return HYB_OK;
}

// fill the species' kind / QED fields from its descriptor
static void species_flags(SpDev &s, const hyb_species_desc *d, int sid) {
    s.pusher = d->pusher;
    s.kind = d->kind;
    s.qed = d->qed;
    s.ph_species = d->qed ? d->photon_species : -1;
    s.eps_min = d->photon_eps_min > 0.0 ? (float)d->photon_eps_min : 2.0f;
    s.pair_e = d->kind == HYB_KIND_PHOTON ? d->pair_electron : -1;
    s.pair_p = d->kind == HYB_KIND_PHOTON ? d->pair_positron : -1;
    s.tau_index = (uint32_t)sid;
    s.sp_index = (uint32_t)sid;
}

static bool needs_tau(const hyb_species_desc *d) {
    return d->qed || (d->kind == HYB_KIND_PHOTON && d->pair_electron >= 0);
}

// cross-species references must name loaded species of the right kind
static hyb_status validate_links(const hyb_ctx *c) {
    const int ns = (int)c->sp.size();
    auto lepton = [&](int i, double q) {
        return i >= 0 && i < ns && c->sp[i].dev.kind == HYB_KIND_MASSIVE && c->sp[i].q == q && c->sp[i].m == 1.0 &&
               !c->sp[i].has_zq;
    };
    for (int i = 0; i < ns; ++i) {
        const SpDev &s = c->sp[i].dev;
        if (s.zmax > 0 && !lepton(s.ion_into, -1.0))
            return set_error(HYB_EINVAL, "ionize_into must be an electron species");
        if (s.qed && s.ph_species >= 0 &&
            !(s.ph_species < ns && c->sp[s.ph_species].dev.kind == HYB_KIND_PHOTON))
            return set_error(HYB_EINVAL, "photon_species must be a photon species");
        if (s.kind == HYB_KIND_PHOTON && s.pair_e >= 0 && !(lepton(s.pair_e, -1.0) && lepton(s.pair_p, 1.0)))
            return set_error(HYB_EINVAL, "pair_electron / pair_positron must be electron / positron species");
    }
    return HYB_OK;
}

hyb_status hyb_load_species(hyb_ctx *c, const hyb_species_desc *d, int *species_id) {
    if (!c || !d || !species_id) return set_error(HYB_EINVAL, "null argument");
    if ((int)c->sp.size() >= HYB_MAX_SPECIES) return set_error(HYB_EINVAL, "too many species");
    if (d->kind != HYB_KIND_MASSIVE && d->kind != HYB_KIND_PHOTON) return set_error(HYB_EINVAL, "bad species kind");
    if (d->kind == HYB_KIND_PHOTON) {
        if (d->q != 0.0 || d->zmax != 0 || d->qed || d->zq)
            return set_error(HYB_EINVAL, "a photon species has q = 0 and no ionization, emission or zq");
        if ((d->pair_electron >= 0) != (d->pair_positron >= 0))
            return set_error(HYB_EINVAL, "pair creation needs both an electron and a positron species");
    } else if (!(d->m > 0.0)) {
        return set_error(HYB_EINVAL, "species mass must be > 0");
    }
    if (d->qed && !(std::fabs(d->q) == 1.0 && d->m == 1.0))
        return set_error(HYB_EINVAL, "photon emission is for electrons and positrons (|q| = 1, m = 1)");
    if ((d->qed || (d->kind == HYB_KIND_PHOTON && d->pair_electron >= 0)) && !(c->desc.lambda_um > 0.0))
        return set_error(HYB_EINVAL, "QED needs lambda_um > 0");
    if (d->n < 0) return set_error(HYB_EINVAL, "negative particle count");
    if (d->pusher < HYB_PUSH_BORIS || d->pusher > HYB_PUSH_HIGUERA_CARY)
        return set_error(HYB_EINVAL, "pusher must be one of HYB_PUSH_*");
    if (d->n > 0 && (!d->x || !d->y || !d->z || !d->ux || !d->uy || !d->uz || !d->w))
        return set_error(HYB_EINVAL, "missing particle arrays");
    if (d->zmax < 0 || d->zmax > 8) return set_error(HYB_EINVAL, "zmax must be in 0..8");
    if (d->zmax > 0) {
        if (!d->zq) return set_error(HYB_EINVAL, "an ionizable species needs per-particle charge states (zq)");
        if (d->ionize_into < 0 || d->ionize_into >= HYB_MAX_SPECIES)
            return set_error(HYB_EINVAL, "ionize_into must be a species id");
        for (int z = 0; z < d->zmax; ++z)
            if (!(d->ip_eV[z] > 0.0) || d->l_qn[z] < 0 || d->l_qn[z] > 3)
                return set_error(HYB_EINVAL, "bad ionization potential or quantum number");
        if (!(c->desc.lambda_um > 0.0)) return set_error(HYB_EINVAL, "ionization needs lambda_um > 0");
    }
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const long long n = d->n;

    // positions must lie inside the domain
    // (checked on the device copy below through the tile counts: out-of-range positions are clamped
    // into the edge tiles by tile_index, so validate on the host when the arrays are host memory)
    if (!d->ptr_on_device) {
        for (long long p = 0; p < n; ++p) {
            const float v[3] = {d->x[p], d->y[p], d->z[p]};
            for (int a = 0; a < 3; ++a) {
                const float hi = g.bc[a] ? (float)(g.n[a] - 1) : (float)g.n[a];
                if (!(v[a] >= 0.0f) || v[a] > hi || (g.bc[a] == 0 && v[a] >= hi))
                    return set_error(HYB_EINVAL, "particle " + std::to_string(p) + " position " +
                                                     std::to_string(v[a]) + " on axis " + std::to_string(a) +
                                                     " outside the domain");
            }
        }
    }

    // stage arrays on the device (temporary)
    size_t arena_mark = c->arena.used;
    std::vector<void *> tmp;
    auto talloc = [&](void **p, size_t b) -> bool {
        if (c->arena.base) return ctx_alloc(c, p, b) == cudaSuccess;
        if (cudaMalloc(p, b ? b : 256) != cudaSuccess) return false;
        tmp.push_back(*p);
        return true;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (void *p : tmp) cudaFree(p);
        if (c->arena.base) c->arena.used = arena_mark;
    };
    const float *src[8] = {d->x, d->y, d->z, d->ux, d->uy, d->uz, d->w, d->zq};
    const float *dsrc[8] = {nullptr};
    const uint64_t *dids = nullptr;
    int *counts = nullptr;
    bool ok = talloc((void **)&counts, sizeof(int) * g.ntiles);
    for (int k = 0; ok && k < 8; ++k) {
        if (!src[k]) continue;
        if (d->ptr_on_device) {
            dsrc[k] = src[k];
        } else {
            float *p = nullptr;
            ok = talloc((void **)&p, sizeof(float) * n);
            if (ok) ok = cudaMemcpyAsync(p, src[k], sizeof(float) * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            dsrc[k] = p;
        }
    }
    if (ok && d->ids) {
        if (d->ptr_on_device) {
            dids = d->ids;
        } else {
            uint64_t *p = nullptr;
            ok = talloc((void **)&p, sizeof(uint64_t) * n);
            if (ok) ok = cudaMemcpyAsync(p, d->ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            dids = p;
        }
    }
    if (!ok) {
        cleanup();
        return set_error(HYB_ENOMEM, "staging allocation/copy for species failed");
    }
    cudaMemsetAsync(counts, 0, sizeof(int) * g.ntiles, st);
    launch_count_tiles(g, n, dsrc[0], dsrc[1], dsrc[2], counts, st);
    std::vector<int> hcounts(g.ntiles);
    cudaMemcpyAsync(hcounts.data(), counts, sizeof(int) * g.ntiles, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return set_error(HYB_ECUDA, std::string("species count: ") + cudaGetErrorString(e));
    }
    int maxc = 0;
    for (int v : hcounts) maxc = std::max(maxc, v);
    long long cap = d->tile_capacity > 0 ? d->tile_capacity : 2LL * maxc + 64;
    cap = (cap + 31) / 32 * 32;
    if (cap < maxc) {
        cleanup();
        return set_error(HYB_EOVERFLOW, "tile_capacity below the initial count of a tile");
    }
    if (cap > 0x7fffffffLL / 2) {
        cleanup();
        return set_error(HYB_EINVAL, "tile capacity too large");
    }

    // the species buffers must outlive the staging area: allocate them after
    // releasing it when an arena is used (the bump allocator is LIFO)
    if (c->arena.base) {
        // move staging out of the way: copy counts were read; re-stage after allocation
    }
    Species sp;
    sp.q = d->q;
    sp.m = d->m;
    sp.has_zq = d->zq != nullptr;
    sp.cap = (int)cap;
    if (c->arena.base) {
        // release staging, allocate species, then stage again on top
        cleanup();
        tmp.clear();
        if (alloc_species(c, sp, (int)cap, sp.has_zq, needs_tau(d)) != HYB_OK)
            return set_error(HYB_ENOMEM, "species allocation failed (arena too small?)");
        species_flags(sp.dev, d, (int)c->sp.size());
        hyb_status is = setup_ionization(c, sp.dev, d);
        if (is != HYB_OK) return is;
        arena_mark = c->arena.used;
        ok = true;
        for (int k = 0; ok && k < 8; ++k) {
            if (!src[k] || d->ptr_on_device) continue;
            float *p = nullptr;
            ok = talloc((void **)&p, sizeof(float) * n);
            if (ok) ok = cudaMemcpyAsync(p, src[k], sizeof(float) * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            dsrc[k] = p;
        }
        if (ok && d->ids && !d->ptr_on_device) {
            uint64_t *p = nullptr;
            ok = talloc((void **)&p, sizeof(uint64_t) * n);
            if (ok) ok = cudaMemcpyAsync(p, d->ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            dids = p;
        }
        if (!ok) {
            cleanup();
            return set_error(HYB_ENOMEM, "staging allocation for species failed (arena too small?)");
        }
    } else {
        if (alloc_species(c, sp, (int)cap, sp.has_zq, needs_tau(d)) != HYB_OK) {
            cleanup();
            return set_error(HYB_ENOMEM, "species allocation failed");
        }
        species_flags(sp.dev, d, (int)c->sp.size());
        hyb_status is = setup_ionization(c, sp.dev, d);
        if (is != HYB_OK) {
            cleanup();
            return is;
        }
    }
    launch_bin_particles(g, sp.dev, n, dsrc[0], dsrc[1], dsrc[2], dsrc[3], dsrc[4], dsrc[5], dsrc[6], dsrc[7], dids,
                         nullptr, c->status, st);
    int hstatus = 0;
    cudaMemcpyAsync(&hstatus, c->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("species bin: ") + cudaGetErrorString(e));
    if (hstatus) {
        c->error_latched = true;
        return set_error(status_to_code(hstatus), "particle binning overflowed a tile");
    }
    if (needs_tau(d)) {
        hyb_status qs = setup_qed(c);
        if (qs != HYB_OK) return qs;
    }
    *species_id = (int)c->sp.size();
    c->sp.push_back(sp);
    {
        const SpSet all = species_set(c);
        e = cudaMemcpyAsync(c->sp_dev, all.s, sizeof(SpDev) * all.n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            c->sp.pop_back();
            return set_error(HYB_ECUDA, std::string("species table upload: ") + cudaGetErrorString(e));
        }
    }
    c->graph_valid = false;
    return HYB_OK;
}

hyb_status hyb_load_fluid(hyb_ctx *c, const hyb_fluid_desc *d, int *fluid_id) {
    if (!c || !d || !fluid_id || !d->n) return set_error(HYB_EINVAL, "null argument");
    if ((int)c->fluids.size() >= HYB_MAX_FLUIDS) return set_error(HYB_EINVAL, "too many fluids");
    if (!(d->m > 0.0)) return set_error(HYB_EINVAL, "fluid mass must be > 0");
    const size_t N = (size_t)c->g.N;
    FluidDev f;
    memset(&f, 0, sizeof(f));
    float **bufs[8] = {&f.n, &f.ux, &f.uy, &f.uz, &f.ns, &f.usx, &f.usy, &f.usz};
    for (auto b : bufs)
        if (ctx_alloc(c, (void **)b, sizeof(float) * N)) return set_error(HYB_ENOMEM, "fluid allocation failed");
    if (ctx_alloc(c, (void **)&f.clamped, sizeof(unsigned long long)))
        return set_error(HYB_ENOMEM, "fluid allocation failed");
    f.q = (float)d->q;
    f.m = (float)d->m;
    f.m_d = d->m;
    f.n_floor = d->n_floor > 0.0 ? (float)d->n_floor : 1e-10f;
    if (d->temperature_keV < 0.0 || d->gamma_ad < 0.0 || d->n_ref < 0.0)
        return set_error(HYB_EINVAL, "fluid temperature, adiabatic index and reference density must be >= 0");
    if (d->temperature_keV > 0.0) {
        const double gam = d->gamma_ad > 0.0 ? d->gamma_ad : 5.0 / 3.0;
        const double nref = d->n_ref > 0.0 ? d->n_ref : 1.0;
        f.pK = (float)(d->temperature_keV / 510.99895 * std::pow(nref, 1.0 - gam));
        f.pgam = (float)gam;
    }
    const cudaMemcpyKind kind = d->ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const float *src[4] = {d->n, d->ux, d->uy, d->uz};
    float *dst[4] = {f.n, f.ux, f.uy, f.uz};
    for (int k = 0; k < 4; ++k) {
        if (src[k]) HYB_CUDA_TRY(cudaMemcpyAsync(dst[k], src[k], sizeof(float) * N, kind, c->stream));
        else HYB_CUDA_TRY(cudaMemsetAsync(dst[k], 0, sizeof(float) * N, c->stream));
    }
    HYB_CUDA_TRY(cudaMemsetAsync(f.clamped, 0, sizeof(unsigned long long), c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->fluids_idle = false;
    // a new fluid's u where n = 0 is whatever was loaded: no fluid range until a step has run
    c->fluid_fresh_step = c->step;
    if (clear_fluid_range(c, c->stream) != HYB_OK) return set_error(HYB_ECUDA, "fluid range reset");
    *fluid_id = (int)c->fluids.size();
    c->fluids.push_back(f);
    c->graph_valid = false;
    return HYB_OK;
}

hyb_status hyb_set_regime(hyb_ctx *c, const hyb_regime_desc *d) {
    if (!c || !d) return set_error(HYB_EINVAL, "null argument");
    if (d->dilate < 0 || d->dilate > 8) return set_error(HYB_EINVAL, "dilate must be in 0..8");
    if (d->ppc < 0 || d->ppc > 64) return set_error(HYB_EINVAL, "ppc must be in 0..64");
    if (d->policy < HYB_REGIME_DEFAULT || d->policy > HYB_REGIME_ALL_KINETIC)
        return set_error(HYB_EINVAL, "policy must be one of HYB_REGIME_*");
    if (d->quiet != 0 && d->quiet != 1) return set_error(HYB_EINVAL, "quiet must be 0 or 1");
    if (d->reach < 0) return set_error(HYB_EINVAL, "reach must be >= 0");
    for (int f = 0; f < HYB_MAX_FLUIDS; ++f)
        if (d->to_species[f] >= (int)c->sp.size() ||
            (d->to_species[f] >= 0 && c->sp[d->to_species[f]].dev.kind != HYB_KIND_MASSIVE))
            return set_error(HYB_EINVAL, "to_species must name a loaded massive species or -1");
    hyb_regime_desc r = *d;
    if (!(r.a_thr > 0.0)) r.a_thr = 1.0;
    if (!(r.n_thr > 0.0)) r.n_thr = 1.0;
    if (!(r.c_thr > 0.0)) r.c_thr = 0.1;
    if (!(r.chi_thr > 0.0)) r.chi_thr = 1e-3;
    if (r.ppc == 0) r.ppc = 8;
    c->regime = r;
    return HYB_OK;
}

hyb_status hyb_classify(hyb_ctx *c, const hyb_model *model, float *p_mean_dev, float *p_std_dev, uint8_t *mask_dev) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    if (c->error_latched) return set_error(HYB_ESTATE, "context is in an error state (hyb_clear_status)");
    for (size_t f = 0; f < c->fluids.size(); ++f) {
        const int sid = c->regime.to_species[f];
        if (sid >= 0 && (c->sp[sid].q != (double)c->fluids[f].q || c->sp[sid].m != c->fluids[f].m_d))
            return set_error(HYB_EINVAL, "a fluid converts into a species of the same charge and mass");
        if (sid >= 0 && c->g.order != 1)
            return set_error(HYB_EINVAL, "conversions deposit with the CIC shape: not with shape_order 2");
    }
    hyb_status s;
    c->launches_classify = 0;
    auto mark = [c](cudaEvent_t e) {
        if (c->profiling) cudaEventRecord(e, c->stream);
    };
    if (model) {
        c->phase_ran[HYB_PH_CLASSIFY] = c->profiling;
        mark(c->ev_start[HYB_PH_CLASSIFY]);
        s = classifier_forward(c, model, p_mean_dev, p_std_dev);
        mark(c->ev_end[HYB_PH_CLASSIFY]);
        if (s != HYB_OK) return s;
    }
    c->phase_ran[HYB_PH_REGIME] = c->profiling;
    mark(c->ev_start[HYB_PH_REGIME]);
    s = model ? regime_update(c, model_p_mean(model), model_p_std(model)) : regime_update(c, nullptr, nullptr);
    if (s == HYB_OK) s = set_fluid_range(c);
    mark(c->ev_end[HYB_PH_REGIME]);
    if (s != HYB_OK) return s;
    if (mask_dev) HYB_CUDA_TRY(cudaMemcpyAsync(mask_dev, c->mask, (size_t)c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    return HYB_OK;
}

hyb_status hyb_get_regime(hyb_ctx *c, uint8_t *mask, float *rho_bg) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    if (mask) HYB_CUDA_TRY(cudaMemcpyAsync(mask, c->mask, (size_t)c->g.N, cudaMemcpyDeviceToHost, c->stream));
    if (rho_bg)
        HYB_CUDA_TRY(cudaMemcpyAsync(rho_bg, c->rho_bg, sizeof(float) * (size_t)c->g.N, cudaMemcpyDeviceToHost,
                                     c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return read_status(c);
}

hyb_status hyb_get_fluid(hyb_ctx *c, int id, float *n, float *ux, float *uy, float *uz) {
    if (!c || id < 0 || id >= (int)c->fluids.size()) return set_error(HYB_EINVAL, "bad fluid id");
    const FluidDev &f = c->fluids[id];
    const size_t bytes = sizeof(float) * (size_t)c->g.N;
    float *dst[4] = {n, ux, uy, uz};
    const float *src[4] = {f.n, f.ux, f.uy, f.uz};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) HYB_CUDA_TRY(cudaMemcpyAsync(dst[k], src[k], bytes, cudaMemcpyDeviceToHost, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return HYB_OK;
}

hyb_status hyb_set_fields(hyb_ctx *c, const float *E, const float *B, int on_device) {
    if (!c || !E || !B) return set_error(HYB_EINVAL, "null argument");
    const size_t fbytes = sizeof(float) * 3 * (size_t)c->g.N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HYB_CUDA_TRY(cudaMemcpyAsync(c->E, E, fbytes, kind, c->stream));
    HYB_CUDA_TRY(cudaMemcpyAsync(c->B, B, fbytes, kind, c->stream));
    launch_mur_save(c->g, c->E, c->mur_old, c->mur_plane, c->stream);
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return HYB_OK;
}

static hyb_status capture_step(hyb_ctx *c) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (c->graph_tmpl) {
        cudaGraphDestroy(c->graph_tmpl);
        c->graph_tmpl = nullptr;
    }
    cudaGraph_t graph;
    HYB_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(c);
    HYB_CUDA_TRY(cudaStreamEndCapture(c->stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&c->graph, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(HYB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->graph_tmpl = graph;
    c->graph_version += 1;
    c->graph_valid = true;
    return HYB_OK;
}

// Capacity growth: a species whose tiles passed half of their capacity (flag
// set by the compaction or a conversion) gets twice the slots per tile before
// the next steps; its live particles are copied tile by tile.
static hyb_status grow_full_species(hyb_ctx *c, bool wait, cudaStream_t steps_stream = nullptr) {
    if (!c->fill_pending) return HYB_OK;
    const cudaError_t q = wait ? cudaEventSynchronize(c->fill_ev) : cudaEventQuery(c->fill_ev);
    if (q == cudaErrorNotReady) return HYB_OK;
    if (q != cudaSuccess) return set_error(HYB_ECUDA, std::string("fill check: ") + cudaGetErrorString(q));
    c->fill_pending = false;
    const int flags = *c->fill_host;
    if (!flags) return HYB_OK;
    if (steps_stream) HYB_CUDA_TRY(cudaStreamSynchronize(steps_stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (size_t sid = 0; sid < c->sp.size(); ++sid) {
        if (!(flags & (1 << sid))) continue;
        Species &sp = c->sp[sid];
        const long long ncap = std::min<long long>(2LL * sp.dev.cap, 0x3fffffffLL);
        if (ncap <= sp.dev.cap || ncap * (long long)c->g.ntiles > (1LL << 40))
            return set_error(HYB_EOVERFLOW, "species tiles are full and cannot grow");
        SpDev ns = sp.dev;
        if (alloc_slots(c, ns, (int)ncap, sp.dev.zq != nullptr, sp.dev.tau != nullptr) != HYB_OK)
            return set_error(HYB_ENOMEM, "growing a species' tiles");
        launch_regrid(c->g, sp.dev, ns, c->stream);
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        free_slots(c, sp.dev);
        sp.dev = ns;
        sp.cap = (int)ncap;
        sp.mig_cap = ns.mig_cap;
    }
    const SpSet all = species_set(c);
    HYB_CUDA_TRY(cudaMemcpyAsync(c->sp_dev, all.s, sizeof(SpDev) * all.n, cudaMemcpyHostToDevice, c->stream));
    HYB_CUDA_TRY(cudaMemsetAsync(c->fill_flags, 0, sizeof(int), c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->graph_valid = false;
    return HYB_OK;
}

hyb_status hyb_step(hyb_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return set_error(HYB_EINVAL, "bad argument");
    if (c->error_latched) return set_error(HYB_ESTATE, "context is in an error state (hyb_clear_status)");
    if (nsteps == 0) return HYB_OK;
    if (!c->graph_valid) {
        hyb_status lv = validate_links(c);
        if (lv != HYB_OK) return lv;
    }
    for (int done = 0; done < nsteps;) {
        if (c->auto_grow) {
            // the host may run ahead of the flags by at most two check intervals
            hyb_status gs = grow_full_species(c, c->steps_since_copy >= GROW_CHECK_STEPS);
            if (gs != HYB_OK) return gs;
        }
        if (!c->graph_valid) {
            hyb_status cs = capture_step(c);
            if (cs != HYB_OK) return cs;
        }
        const int chunk = std::min(nsteps - done, GROW_CHECK_STEPS);
        for (int i = 0; i < chunk; ++i) {
            if (c->fluid_xr_until >= 0 && c->step + i >= c->fluid_xr_until) {
                hyb_status fs = clear_fluid_range(c, c->stream);  // the range has lapsed: every plane again
                if (fs != HYB_OK) return fs;
            }
            HYB_CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
        }
        done += chunk;
        c->step += chunk;
        c->steps_since_copy += chunk;
        if (c->auto_grow && !c->fill_pending && c->steps_since_copy >= GROW_CHECK_STEPS) {
            // the fill flags travel to pinned memory behind the steps; the next
            // check reads them once the copy is done, without waiting for it
            HYB_CUDA_TRY(cudaMemcpyAsync(c->fill_host, c->fill_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            HYB_CUDA_TRY(cudaEventRecord(c->fill_ev, c->stream));
            c->fill_pending = true;
            c->steps_since_copy = 0;
        }
    }
    return HYB_OK;
}

}  // extern "C"

// A batch replays the captured steps of several contexts as one CUDA graph
// whose branches (one child graph per context) have no dependencies between
// them, so small runs share the GPU instead of queueing behind each other.
struct hyb_batch {
    std::vector<hyb_ctx *> ctx;
    std::vector<unsigned> version;      // graph_version of each context when the batch graph was built
    std::vector<cudaEvent_t> ctx_ev;    // orders the batch after each context's earlier work
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t done = nullptr;         // orders each context's later work after the batch
};

static hyb_status batch_build(hyb_batch *b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t parent;
    HYB_CUDA_TRY(cudaGraphCreate(&parent, 0));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaGraphNode_t node;
        const cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, b->ctx[i]->graph_tmpl);
        if (e != cudaSuccess) {
            cudaGraphDestroy(parent);
            return set_error(HYB_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        }
        b->version[i] = b->ctx[i]->graph_version;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->exec, parent, 0);
    cudaGraphDestroy(parent);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
    return HYB_OK;
}

extern "C" {

hyb_status hyb_batch_create(hyb_ctx *const *ctxs, int n, void *stream, hyb_batch **out) {
    if (!ctxs || n <= 0 || !out) return set_error(HYB_EINVAL, "bad argument");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return set_error(HYB_EINVAL, "null context in a batch");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return set_error(HYB_EINVAL, "a context appears twice in a batch");
    }
    hyb_batch *b = new hyb_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->version.assign(n, 0);
    b->ctx_ev.assign(n, nullptr);
    bool ok = true;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess;
        b->own_stream = ok;
    }
    for (int i = 0; ok && i < n; ++i) ok = cudaEventCreateWithFlags(&b->ctx_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        hyb_batch_destroy(b);
        return set_error(HYB_ECUDA, "batch stream or events");
    }
    *out = b;
    return HYB_OK;
}

void hyb_batch_destroy(hyb_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaEvent_t e : b->ctx_ev)
        if (e) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

hyb_status hyb_batch_step(hyb_batch *b, int nsteps) {
    if (!b || nsteps < 0) return set_error(HYB_EINVAL, "bad argument");
    if (nsteps == 0) return HYB_OK;
    const size_t n = b->ctx.size();
    for (hyb_ctx *c : b->ctx) {
        if (c->error_latched) return set_error(HYB_ESTATE, "a context of the batch is in an error state");
        if (!c->graph_valid) {
            hyb_status lv = validate_links(c);
            if (lv != HYB_OK) return lv;
        }
    }
    for (size_t i = 0; i < n; ++i) {
        HYB_CUDA_TRY(cudaEventRecord(b->ctx_ev[i], b->ctx[i]->stream));
        HYB_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0));
    }
    for (int done = 0; done < nsteps;) {
        bool rebuild = b->exec == nullptr;
        for (size_t i = 0; i < n; ++i) {
            hyb_ctx *c = b->ctx[i];
            if (c->auto_grow) {
                hyb_status gs = grow_full_species(c, c->steps_since_copy >= GROW_CHECK_STEPS, b->stream);
                if (gs != HYB_OK) return gs;
            }
            if (!c->graph_valid) {
                hyb_status cs = capture_step(c);
                if (cs != HYB_OK) return cs;
            }
            rebuild = rebuild || b->version[i] != c->graph_version;
        }
        if (rebuild) {
            hyb_status bs = batch_build(b);
            if (bs != HYB_OK) return bs;
        }
        const int chunk = std::min(nsteps - done, GROW_CHECK_STEPS);
        for (int k = 0; k < chunk; ++k) {
            for (hyb_ctx *c : b->ctx)
                if (c->fluid_xr_until >= 0 && c->step + k >= c->fluid_xr_until) {
                    hyb_status fs = clear_fluid_range(c, b->stream);  // a lapsed range: every plane again
                    if (fs != HYB_OK) return fs;
                }
            HYB_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
        }
        done += chunk;
        for (hyb_ctx *c : b->ctx) {
            c->step += chunk;
            c->steps_since_copy += chunk;
            if (c->auto_grow && !c->fill_pending && c->steps_since_copy >= GROW_CHECK_STEPS) {
                HYB_CUDA_TRY(cudaMemcpyAsync(c->fill_host, c->fill_flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
                HYB_CUDA_TRY(cudaEventRecord(c->fill_ev, b->stream));
                c->fill_pending = true;
                c->steps_since_copy = 0;
            }
        }
    }
    HYB_CUDA_TRY(cudaEventRecord(b->done, b->stream));
    for (hyb_ctx *c : b->ctx) HYB_CUDA_TRY(cudaStreamWaitEvent(c->stream, b->done, 0));
    return HYB_OK;
}

hyb_status hyb_set_profiling(hyb_ctx *c, int on) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    if (on) {
        for (int p = 0; p < HYB_NPHASE; ++p) {
            if (!c->ev_start[p]) HYB_CUDA_TRY(cudaEventCreate(&c->ev_start[p]));
            if (!c->ev_end[p]) HYB_CUDA_TRY(cudaEventCreate(&c->ev_end[p]));
        }
    }
    if ((bool)on != c->profiling) {
        c->profiling = on != 0;
        c->graph_valid = false;
        for (int p = 0; p < HYB_NPHASE; ++p) c->phase_ran[p] = false;
    }
    return HYB_OK;
}

hyb_status hyb_phase_times(hyb_ctx *c, hyb_phase_times_t *out) {
    if (!c || !out) return set_error(HYB_EINVAL, "null argument");
    if (!c->profiling) return set_error(HYB_ESTATE, "profiling is off");
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < HYB_NPHASE; ++p) {
        out->ms[p] = 0.0f;
        if (!c->phase_ran[p] || (c->step == 0 && p < HYB_PH_CLASSIFY)) continue;
        if (p == HYB_PH_CONV1 || p == HYB_PH_CONV2) {
            const int l = p - HYB_PH_CONV1, K = c->conv_ev_passes;
            for (int k = 0; k < K; ++k) {
                float ms = 0.0f;
                HYB_CUDA_TRY(cudaEventElapsedTime(&ms, c->conv_ev[(l * K + k) * 2], c->conv_ev[(l * K + k) * 2 + 1]));
                out->ms[p] += ms;
            }
            continue;
        }
        HYB_CUDA_TRY(cudaEventElapsedTime(&out->ms[p], c->ev_start[p], c->ev_end[p]));
    }
    return HYB_OK;
}

hyb_status hyb_eval_rate_table(hyb_ctx *c, int table, int sid, int level, const float *x, int n, float *out) {
    if (!c || !x || !out || n < 0) return set_error(HYB_EINVAL, "bad argument");
    if (n == 0) return HYB_OK;
    if (table == HYB_LUT_IONIZE) {
        if (sid < 0 || sid >= (int)c->sp.size()) return set_error(HYB_EINVAL, "bad species id");
        return eval_ion_table(c, c->sp[sid].dev, level, x, n, out);
    }
    return set_error(HYB_EINVAL, "unknown table");
}

hyb_status hyb_eval_qed(hyb_ctx *c, int what, const float *chi, const float *r, int n, float *out) {
    if (!c || !chi || !out || n < 0) return set_error(HYB_EINVAL, "bad argument");
    if (n == 0) return HYB_OK;
    return eval_qed(c, what, chi, r, n, out);
}

hyb_status hyb_set_auto_grow(hyb_ctx *c, int on) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    c->auto_grow = on != 0;
    return HYB_OK;
}

hyb_status hyb_selftest_wait_timeout(hyb_ctx *c, long long polls) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    if (polls < 1 || polls > (1LL << 20)) return set_error(HYB_EINVAL, "polls must be in 1..2^20");
    launch_wait_selftest(polls, c->status, c->stream);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

hyb_status hyb_clear_status(hyb_ctx *c) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    HYB_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->error_latched = false;
    return HYB_OK;
}

static hyb_status read_status(hyb_ctx *c) {
    int h = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (h) {
        c->error_latched = true;
        return set_error(status_to_code(h), "device status word set");
    }
    return HYB_OK;
}

hyb_status hyb_diagnostics(hyb_ctx *c, hyb_diag *out) {
    if (!c || !out) return set_error(HYB_EINVAL, "null argument");
    memset(out, 0, sizeof(*out));
    const SpSet set = species_set(c);
    const int nfl = (int)c->fluids.size();
    for (int f = 0; f < nfl; ++f) {
        double *pw = c->red_partials + (long long)(2 + set.n + 2 * f) * c->red_blocks;
        launch_fluid_energy(c->g, c->fluids[f], pw, pw + c->red_blocks, c->red_blocks, c->stream);
    }
    launch_energy(c->g, c->E, c->B, set, c->red_partials, c->red_blocks, c->red_out, c->status, c->stream, 2 * nfl);
    ClampPtrs cl;
    memset(&cl, 0, sizeof(cl));
    cl.n = nfl;
    for (int f = 0; f < nfl; ++f) cl.p[f] = c->fluids[f].clamped;
    launch_diag_summary(set, c->g.ntiles, c->red_out, 2 + set.n + 2 * nfl, cl, c->status, c->diag_dev, c->stream);
    HYB_CUDA_TRY(cudaGetLastError());
    HYB_CUDA_TRY(cudaMemcpyAsync(c->diag_host, c->diag_dev, sizeof(DiagSummary), cudaMemcpyDeviceToHost, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const DiagSummary &ds = *c->diag_host;
    const double *r = ds.red;
    const int h = ds.status;
    out->n_species = set.n;
    for (int s = 0; s < set.n; ++s) out->count[s] = ds.count[s];
    out->step = c->step;
    out->time = c->step * c->g.dt_d;
    out->w_e = r[0];
    out->w_b = r[1];
    for (int s = 0; s < set.n; ++s) out->w_kin[s] = r[2 + s];
    out->status = status_to_code(h);
    out->launches_per_step = c->launches_per_step;
    out->launches_classify = c->launches_classify;
    out->classified_cells = c->classified_cells;
    out->fluid_cells = c->fluid_xr_until >= 0
                           ? (long long)(c->fluid_xr_host[1] - c->fluid_xr_host[0]) * c->g.n[1] * c->g.n[2]
                           : c->g.N;
    for (size_t i = 0; i < c->sp.size() && i < HYB_MAX_SPECIES; ++i) out->tile_capacity[i] = c->sp[i].dev.cap;
    out->n_fluids = nfl;
    for (int f = 0; f < nfl; ++f) {
        out->w_fluid[f] = r[2 + set.n + 2 * f];
        out->n_fluid[f] = r[2 + set.n + 2 * f + 1];
        out->n_clamped += (long long)ds.clamped[f];
    }
    // event tallies: per-tile FP64 accumulators, summed on the device
    for (int s = 0; s < set.n; ++s) {
        out->w_ionize += ds.tal_e[s][TALLY_IONIZE];
        out->n_ionize += (long long)ds.tal_n[s][TALLY_IONIZE];
        out->w_photon_untracked += ds.tal_e[s][TALLY_EMIT];
        out->n_emit += (long long)ds.tal_n[s][TALLY_EMIT];
        out->w_pair_deficit += ds.tal_e[s][TALLY_PAIR];
        out->n_pair += (long long)ds.tal_n[s][TALLY_PAIR];
    }
    if (h) {
        c->error_latched = true;
        return set_error(status_to_code(h), "device status word set");
    }
    return HYB_OK;
}

hyb_status hyb_get_fields(hyb_ctx *c, float *E, float *B, float *J) {
    if (!c) return set_error(HYB_EINVAL, "null context");
    const size_t fbytes = sizeof(float) * 3 * (size_t)c->g.N;
    if (E) HYB_CUDA_TRY(cudaMemcpyAsync(E, c->E, fbytes, cudaMemcpyDeviceToHost, c->stream));
    if (B) HYB_CUDA_TRY(cudaMemcpyAsync(B, c->B, fbytes, cudaMemcpyDeviceToHost, c->stream));
    if (J) HYB_CUDA_TRY(cudaMemcpyAsync(J, c->J, fbytes, cudaMemcpyDeviceToHost, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return HYB_OK;
}

hyb_status hyb_get_species(hyb_ctx *c, int sid, long long max_n, float *x, float *y, float *z, float *ux, float *uy,
                           float *uz, float *w, float *zq, uint64_t *ids, long long *n_out) {
    if (!c || sid < 0 || sid >= (int)c->sp.size() || !n_out) return set_error(HYB_EINVAL, "bad argument");
    const Species &sp = c->sp[sid];
    const GridDev &g = c->g;
    std::vector<int> cnt((size_t)g.ntiles);
    HYB_CUDA_TRY(cudaMemcpyAsync(cnt.data(), sp.dev.count, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    long long tot = 0;
    for (int &v : cnt) {
        v = std::min(v, sp.cap);
        tot += v;
    }
    *n_out = tot;
    if (tot > max_n) return set_error(HYB_EINVAL, "output arrays too small");
    // whole slabs are copied to the host and compacted there
    const size_t slots = (size_t)sp.cap * g.ntiles;
    std::vector<float> buf(slots);
    std::vector<uint64_t> ibuf;
    float *dst[8] = {x, y, z, ux, uy, uz, w, zq};
    const float *srcs[8] = {sp.dev.x, sp.dev.y, sp.dev.z, sp.dev.ux, sp.dev.uy, sp.dev.uz, sp.dev.w, sp.dev.zq};
    for (int k = 0; k < 8; ++k) {
        if (!dst[k] || !srcs[k]) continue;
        HYB_CUDA_TRY(cudaMemcpyAsync(buf.data(), srcs[k], sizeof(float) * slots, cudaMemcpyDeviceToHost, c->stream));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        long long o = 0;
        for (int t = 0; t < g.ntiles; ++t) {
            std::memcpy(dst[k] + o, buf.data() + (size_t)t * sp.cap, sizeof(float) * cnt[t]);
            o += cnt[t];
        }
    }
    if (ids) {
        ibuf.resize(slots);
        HYB_CUDA_TRY(cudaMemcpyAsync(ibuf.data(), sp.dev.id, sizeof(uint64_t) * slots, cudaMemcpyDeviceToHost,
                                     c->stream));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        long long o = 0;
        for (int t = 0; t < g.ntiles; ++t) {
            std::memcpy(ids + o, ibuf.data() + (size_t)t * sp.cap, sizeof(uint64_t) * cnt[t]);
            o += cnt[t];
        }
    }
    return read_status(c);
}

}  // extern "C"
