// Internal declarations of the hybrid fluid-kinetic step library (arXiv 2510.11174).
// Shared by the CUDA translation units of libhyb; not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/hyb.h"

namespace hyb {

// ---------------------------------------------------------------- grid view passed to kernels
// Yee staggering: E_x (i+1/2, j, k), E_y (i, j+1/2, k), E_z (i, j, k+1/2),
// B_x (i, j+1/2, k+1/2), B_y (i+1/2, j, k+1/2), B_z (i+1/2, j+1/2, k);
// J with E; index i holds the value at i (integer) or i+1/2 (half-integer).
// Arrays are component-major: F[c * N + i + nx * (j + ny * k)].
struct GridDev {
    int n[3];          // nx, ny, nz
    int bc[3];         // 0 periodic, 1 Mur / reflecting
    int T;             // tile edge (cells), a power of two
    int tshift;        // log2 T
    int nt[3];         // tiles per axis
    int ntiles;
    long long N;       // cells
    float d[3];        // dx, dy, dz
    float dt;
    double dd[3];      // dx, dy, dz in FP64 (reductions)
    double dt_d;       // the same step in FP64 (laser phase, time)
    uint32_t seed;     // Philox key word 0
    int order;         // particle shape: 1 CIC, 2 quadratic (periodic axes only)
};

__host__ __device__ inline long long cidx(const GridDev &g, int i, int j, int k) {
    return (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * (long long)k);
}

#ifdef __CUDACC__
// Kinetic-energy terms of the FP64 reductions in double-float arithmetic: a
// value is an unevaluated sum hi + lo of two FP32 numbers (about 48 mantissa
// bits).  FP64 arithmetic runs at a small fraction of the FP32 rate on this
// part, so the per-particle and per-cell terms are formed on the FP32 units
// with error-free transformations -- two-sum (Knuth), two-product by fused
// multiply-add (Dekker's exact product) -- and only block partials are
// converted to FP64.  Relative error of a term: a few units of 2^-48.
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.h, b.h);
    return ff_fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    const ff p = ff_two_prod(a.h, b);
    return ff_fast_two_sum(p.h, fmaf(a.l, b, p.l));
}
// square root of a > 0: the correctly rounded FP32 root s plus the Newton
// correction (a - s^2) / (2 s); a.h - s^2 is exact by the fused multiply-add
__device__ __forceinline__ ff ff_sqrt(ff a) {
    const float s = sqrtf(a.h);
    const float r = fmaf(-s, s, a.h) + a.l;
    return ff_fast_two_sum(s, r * (0.5f / s));
}
// a / b (b > 0): FP32 quotient q0, then the quotient of the exact residual
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float rc = __frcp_rn(b.h);
    const float q0 = a.h * rc;
    const ff pb = ff_mulf(b, -q0);
    const ff r = ff_add(a, pb);
    return ff_fast_two_sum(q0, r.h * rc);
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }
// u^2 = ux^2 + uy^2 + uz^2 of FP32 components (each square exact)
__device__ __forceinline__ ff ff_u2(float ux, float uy, float uz) {
    return ff_add(ff_add(ff_two_prod(ux, ux), ff_two_prod(uy, uy)), ff_two_prod(uz, uz));
}
// gamma - 1 = u^2 / (gamma + 1) (no cancellation for slow particles)
__device__ __forceinline__ ff ff_gamma_minus_one(ff u2) {
    const ff g = ff_sqrt(ff_add(u2, ff{1.0f, 0.0f}));
    return ff_div(u2, ff_add(g, ff{1.0f, 0.0f}));
}
// |u| for photons (0 at u = 0)
__device__ __forceinline__ ff ff_norm(ff u2) { return u2.h > 0.0f ? ff_sqrt(u2) : ff{0.0f, 0.0f}; }

// Position of v on a grid uniform in log2 v with npo points per octave that
// starts at 2^e0.  The octave comes from the binary exponent (exact) and the
// in-octave position from log2 of the mantissa, so the coordinate keeps the
// mantissa's precision however many octaves the grid spans.
__device__ __forceinline__ void log2_grid(float v, int e0, int npo, int &i, float &f) {
    int e;
    const float m = frexpf(v, &e);           // v = m 2^e, m in [0.5, 1)
    const float lm = log2f(m) * (float)npo;  // in [-npo, 0)
    const float fl = floorf(lm);
    i = (e - e0) * npo + (int)fl;
    f = lm - fl;
}
#endif

// ---------------------------------------------------------------- particle species on the device
// SoA FP32 in fixed-capacity tiles: slot s of tile t lives at t * cap + s.
// x, y, z are cell units; a dead slot (awaiting compaction) has x = -1.
struct SpDev {
    float *x, *y, *z, *ux, *uy, *uz, *w, *zq;  // zq may be null
    uint64_t *id;
    int *count;        // live slots per tile
    int *holes;        // per tile: slots vacated by leavers this step
    int *hole_count, *hole_used;
    int cap;           // slots per tile
    float q, m;
    double m_d;        // mass in FP64 for the energy reductions
    // migration buffer: particles that left their tile this step
    float *mx, *my, *mz, *mux, *muy, *muz, *mw, *mzq;
    uint64_t *mid;
    int *mdest;
    int *mig_count;
    int mig_cap;
    // field ionization (zmax = 0: none)
    int zmax;
    int ion_into;          // species index of the electrons
    uint32_t sp_index;     // Philox key word 1
    const float *lnw;      // [zmax][ION_NL] ln of the rate [1/atomic time] on the log2 F grid
    float e_ratio;         // |E| (normalised) -> F (atomic units)
    float dt_au;           // dt in atomic units
    double ip_mc2[8];      // Ip of state Z in m_e c^2 (energy tally)
    // strong-field QED
    int pusher;            // HYB_PUSH_* (momentum update of massive species)
    int kind;              // 0 massive, 1 photon (moves at c, no charge)
    int qed;               // lepton emits photons
    int ph_species;        // receiving photon species (-1: tally only)
    float eps_min;         // tracking threshold of emitted photons [m c^2]
    int pair_e, pair_p;    // photon species: receiving electron / positron species (-1: none)
    float *tau, *mtau;     // optical depth per slot / per migrant (QED leptons, photons)
    uint32_t tau_index;    // Philox key word 1 for the initial optical depth
    // per-tile accumulated tallies, TALLY_* entries per tile
    double *tal_e;
    unsigned long long *tal_n;
    // bit sp_index is set when a tile of this species passed half of its capacity
    int *fill_flags;
};

// tallies per tile: energies (FP64) and event counts
enum { TALLY_IONIZE = 0, TALLY_EMIT = 1, TALLY_PAIR = 2, NTALLY = 3 };

// cold fluid species on the nodes (state + per-step scratch)
struct FluidDev {
    float *n, *ux, *uy, *uz;       // state: density, u = gamma beta
    float *ns, *usx, *usy, *usz;   // scratch: density and u* after the Lorentz step
    float q, m, n_floor;
    float pK, pgam;                // adiabatic pressure p = pK n^pgam (pK = 0: cold)
    double m_d;
    unsigned long long *clamped;   // accumulated clamp count
};

// device QED tables (see qed.cuh)
struct QedDev {
    const float *em_lnh;    // ln h(chi) on the emission chi grid
    const float *em_cdf;    // cumulative emission spectrum rows over mu
    const float *pair_lnT;  // ln T(chi) on the pair chi grid
    const float *pair_cdf;  // cumulative pair spectrum rows over xi
    float kappa;            // hbar w0 / m c^2
    float pref;             // alpha / kappa
};

// ionization table grid: uniform in log2 F over F = 2^-14 .. 2^10 atomic units
static constexpr int ION_E0 = -14, ION_E1 = 10, ION_NPO = 2048;
static constexpr int ION_NL = (ION_E1 - ION_E0) * ION_NPO + 1;

struct SpSet {
    int n;
    SpDev s[HYB_MAX_SPECIES];
};

// launch shape of the one-thread-per-node kernels: blocks of whole warps
// along x, grid (x blocks, ny, nz), so that a kernel takes (i, j, k) from the
// block and thread indices instead of dividing the linear index
inline dim3 node_block(const GridDev &g) { return dim3(g.n[0] >= 256 ? 256 : 32 * ((g.n[0] + 31) / 32)); }
inline dim3 node_grid(const GridDev &g) {
    const unsigned bx = node_block(g).x;
    return dim3((unsigned)((g.n[0] + bx - 1) / bx), (unsigned)g.n[1], (unsigned)g.n[2]);
}

// what hyb_diagnostics reads back, gathered on the device so that one small
// copy and one synchronisation serve the call
struct DiagSummary {
    double red[2 + HYB_MAX_SPECIES + 2 * HYB_MAX_FLUIDS];  // the energy reductions' results
    long long count[HYB_MAX_SPECIES];                      // live particles per species
    double tal_e[HYB_MAX_SPECIES][NTALLY];                 // event tallies summed over tiles
    unsigned long long tal_n[HYB_MAX_SPECIES][NTALLY];
    unsigned long long clamped[HYB_MAX_FLUIDS];            // fluid nodes clamped to n >= 0
    int status;                                            // device status word
};
struct ClampPtrs {
    const unsigned long long *p[HYB_MAX_FLUIDS];
    int n;
};

// device status bits (latched; read by the synchronising calls)
enum : int {
    ST_OVERFLOW = 1,   // tile or migration capacity exceeded
    ST_NAN = 2,        // non-finite field value
    ST_TIMEOUT = 4,
    ST_BADPOS = 8,     // particle outside its tile or non-finite position (skipped)
};

// ---------------------------------------------------------------- host-side context
struct Species {
    double q, m;
    int has_zq;
    int cap;
    SpDev dev;
    long long mig_cap;
};

struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
};

}  // namespace hyb

struct hyb_ctx {
    hyb_grid_desc desc;
    hyb::GridDev g;
    cudaStream_t stream;
    bool own_stream = false;
    bool error_latched = false;  // set when a synchronising call saw a device error
    hyb::Arena arena;
    std::vector<void *> owned;  // cudaMalloc'd buffers when no arena is given

    float *E = nullptr, *B = nullptr, *J = nullptr;  // 3 * N each
    float *mur_old = nullptr;                        // saved boundary planes for Mur
    long long mur_plane = 0;                         // max plane size
    float *jscratch = nullptr;                       // per-tile J frames
    int *jvalid = nullptr;                           // per tile: 1 when its frame was written this step
    long long jframe = 0;                            // floats per tile of the frame scratch (4 * G^3)
    double *red_partials = nullptr;                  // FP64 block partials of reductions
    int red_blocks = 0;
    double *red_out = nullptr;                       // reduction results
    hyb::DiagSummary *diag_dev = nullptr;            // device summary of hyb_diagnostics
    hyb::DiagSummary *diag_host = nullptr;           // its pinned host copy
    int *status = nullptr;                           // device status word
    long long *step_dev = nullptr;                   // device step counter (read by graph replays)
    int *mig_counts = nullptr;                       // HYB_MAX_SPECIES migration counters
    int *fill_flags = nullptr;                       // device: species whose tiles passed half of their capacity
    int *fill_host = nullptr;                        // pinned copy of fill_flags (read without a sync)
    cudaEvent_t fill_ev = nullptr;                   // marks the copy into fill_host
    bool fill_pending = false;                       // a copy into fill_host was enqueued
    long long steps_since_copy = 0;                  // steps enqueued since that copy
    bool auto_grow = true;                           // hyb_step grows full species

    std::vector<hyb::Species> sp;
    hyb::SpDev *sp_dev = nullptr;  // device copy of the species descriptors (HYB_MAX_SPECIES)

    std::vector<hyb::FluidDev> fluids;

    // regime switching
    hyb_regime_desc regime = {};
    uint8_t *mask = nullptr, *mask_tmp = nullptr;  // 1 = kinetic
    uint8_t *mask_prev = nullptr;                  // the mask before the current classification
    float *rho_bg = nullptr;                       // residual background charge
    float *ne = nullptr;                           // electron density scratch
    uint32_t epoch = 0;                            // conversion counter (Philox counter word)
    int *xflag = nullptr, *xflag_host = nullptr;   // x-planes holding matter (device, pinned copy; nx each)
    // the fluid kernels' x-range [lo, hi) (device; hi <= lo: every plane), set by a
    // classification with a reach and valid for the steps before fluid_xr_until
    int *fluid_xr = nullptr, *fluid_xr_host = nullptr;
    long long fluid_xr_until = -1;                 // -1: no range in force
    long long fluid_fresh_step = 0;                // the step of the latest fluid load or state restore
    bool fluids_idle = false;                      // every fluid was converted by an all-kinetic classification

    // LCFA QED tables (built on first use)
    bool qed_ready = false;
    hyb::QedDev qed = {};
    double *airy_ai = nullptr, *airy_aip = nullptr, *airy_aint = nullptr;
    long long step = 0;

    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_tmpl = nullptr;               // the captured step (kept for batches)
    unsigned graph_version = 0;                     // bumped at every capture
    bool graph_valid = false;

    // phase profiling: events recorded at the start of every phase and at the end
    bool profiling = false;
    cudaEvent_t ev_start[HYB_NPHASE] = {};
    cudaEvent_t ev_end[HYB_NPHASE] = {};
    bool phase_ran[HYB_NPHASE] = {};
    std::vector<cudaEvent_t> conv_ev;               // profiling: [layer 1, 2][pass][start, end]
    int conv_ev_passes = 0;                         // passes recorded by the most recent classification
    long long launches_per_step = 0;
    long long launches_classify = 0;               // kernels the most recent hyb_classify launched
    long long classified_cells = 0;                // nodes the most recent classifier pass computed

    // laser transverse profile (FP32, ny*nz) when a Gaussian source is set
    float *laser_profile = nullptr;
};

namespace hyb {

// allocation from the caller's arena (bump) or cudaMalloc
cudaError_t ctx_alloc(hyb_ctx *c, void **p, size_t bytes);

// error plumbing
hyb_status set_error(hyb_status s, const std::string &msg);
#define HYB_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return ::hyb::set_error(HYB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ---------------------------------------------------------------- launchers (one per kernel family)
void launch_fdtd_b_half(const GridDev &g, const float *E, float *B, cudaStream_t st);
void launch_fdtd_e(const GridDev &g, float *E, const float *B, const float *J, cudaStream_t st);
void launch_mur(const GridDev &g, float *E, float *mur_old, long long plane, cudaStream_t st);
void launch_mur_save(const GridDev &g, const float *E, float *mur_old, long long plane, cudaStream_t st);
void launch_laser_source(const GridDev &g, const hyb_grid_desc &d, const float *profile,
                         const long long *step_dev, float *J, cudaStream_t st);
void launch_step_inc(long long *step_dev, cudaStream_t st);
void launch_wait_selftest(long long polls, int *status, cudaStream_t st);

size_t push_smem_bytes(int T, int order);
void launch_push_deposit(const GridDev &g, const float *E, const float *B, const SpDev *sps_dev, int nsp,
                         const QedDev &qd, float *jscratch, int *jvalid, int *status, const long long *step_dev,
                         cudaStream_t st);
hyb_status setup_qed(hyb_ctx *c);  // builds the QED tables once per context
hyb_status regime_update(hyb_ctx *c, const float *p_mean, const float *p_std);
// the x-range [*xa, *xb) of nodes within `reach` nodes (along x) of an
// x-plane holding matter (fluid above its floor, or particles); empty
// (*xa == *xb) without matter.  Synchronises the context stream.
hyb_status matter_x_range(hyb_ctx *c, int reach, int *xa, int *xb);
// after a classification with a reach: restrict the fluid kernels to the
// x-planes within the reach of nonzero fluid density for the next `reach` steps
hyb_status set_fluid_range(hyb_ctx *c);
// back to every plane (stream-ordered)
hyb_status clear_fluid_range(hyb_ctx *c, cudaStream_t st);
hyb_status classifier_forward(hyb_ctx *c, const hyb_model *m, float *p_mean_dev, float *p_std_dev);
const float *model_p_mean(const hyb_model *m);
const float *model_p_std(const hyb_model *m);
void launch_fluids(const GridDev &g, const float *E, const float *B, const FluidDev *f, int nf, float *J,
                   const int *xr, cudaStream_t st);
// FP64 partials of sum n m (gamma-1) (into p_w) and sum n (into p_n), nblocks each
void launch_fluid_energy(const GridDev &g, const FluidDev &f, double *p_w, double *p_n, int nblocks,
                         cudaStream_t st);
hyb_status eval_qed(hyb_ctx *c, int what, const float *chi, const float *r, int n, float *out);
hyb_status setup_ionization(hyb_ctx *c, SpDev &s, const hyb_species_desc *d);
hyb_status eval_ion_table(hyb_ctx *c, const SpDev &s, int Z, const float *x_host, int n, float *out_host);
void launch_j_reduce(const GridDev &g, const float *jscratch, const int *jvalid, float *J, cudaStream_t st);
void launch_rebin(const GridDev &g, const SpDev &s, int *status, cudaStream_t st);
void launch_compact(const GridDev &g, const SpDev &s, cudaStream_t st);
void launch_regrid(const GridDev &g, const SpDev &from, const SpDev &to, cudaStream_t st);
void launch_bin_particles(const GridDev &g, const SpDev &s, long long n, const float *x, const float *y,
                          const float *z, const float *ux, const float *uy, const float *uz, const float *w,
                          const float *zq, const uint64_t *ids, const float *tau, int *status,
                          cudaStream_t st);
void launch_tiles_to_arrays(const GridDev &g, const SpDev &s, const long long *offsets, float *x, float *y, float *z,
                            float *ux, float *uy, float *uz, float *w, float *zq, float *tau, uint64_t *ids,
                            cudaStream_t st);
// species slot storage (abi.cu): allocate / release the per-slot arrays of a species
hyb_status alloc_slots(hyb_ctx *c, SpDev &s, int cap, bool has_zq, bool has_tau);
void free_slots(hyb_ctx *c, const SpDev &s);
SpSet species_set(const hyb_ctx *c);
void launch_count_tiles(const GridDev &g, long long n, const float *x, const float *y, const float *z,
                        int *counts, cudaStream_t st);

// FP64 reductions; results written to out[]: [0] = sum E^2 dV / 2, [1] = sum B^2 dV / 2,
// [2 + s] = kinetic energy of species s; also sets ST_NAN on non-finite fields.
void launch_diag_summary(const SpSet &set, int ntiles, const double *red, int nred, const ClampPtrs &cl,
                         const int *status, DiagSummary *out, cudaStream_t st);
void launch_energy(const GridDev &g, const float *E, const float *B, const SpSet &set,
                   double *partials, int nblocks, double *out, int *status, cudaStream_t st, int n_extra);


// ---------------------------------------------------------------- network training helpers (classifier.cu)
// out[o] = sum_k part[k][o], k in increasing order
__global__ void k_sum_parts(const float *__restrict__ part, int nchunks, int nout, float *__restrict__ out);
// one Adam step on FP32 masters (c1, c2: the bias corrections 1 - beta^t)
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2);

// dropout p as the threshold on 16-bit Philox fields (p is used as
// round(p 2^16) / 2^16) and the inverted-dropout scale of kept values
inline uint32_t dropout_threshold(double p) {
    const long t = std::lround(p * 65536.0);
    return (uint32_t)(t < 0 ? 0 : (t > 65535 ? 65535 : t));
}
inline float dropout_scale(uint32_t thr) { return (float)(65536.0 / (65536.0 - (double)thr)); }

// charge density at the nodes (particles by CIC, fluids, rho_bg) into rho [nz][ny][nx] (regime.cu)
hyb_status charge_density(hyb_ctx *c, float *rho);

// ---------------------------------------------------------------- layer activations (surrogate.cu)
// dropout of one layer on the classifier's Philox stream: counter (cell %
// V, cell / V, layer << 16 | channel / 8, pass), key (seed, 0xD0); a channel
// keeps when its 16-bit field is >= thr (thr = 0: no dropout)
struct DropArgs {
    uint32_t thr, seed, pass, layer;
    float scale;
};
// a = relu(s + b) [dropout] [+ res]: one thread per cell and 8-channel group;
// BF16 out (out) or FP32 out (outf); cells = B V
__global__ void k_act_finish(const float *__restrict__ s, const float *__restrict__ bias, int cop, int relu,
                             const __nv_bfloat16 *__restrict__ res, int cres, DropArgs dr, int B, long long V,
                             __nv_bfloat16 *__restrict__ out, float *__restrict__ outf);
// dz = bf16(G [s + b > 0] keep / (1 - p)): the data gradient at a layer's pre-activation
__global__ void k_act_dz(const float *__restrict__ G, const float *__restrict__ s, const float *__restrict__ bias,
                         int cop, int relu, DropArgs dr, int B, long long V, __nv_bfloat16 *__restrict__ dz);
// classifier loss pieces (classifier.cu): field energy density of [B][>=6][V]
// inputs with FP64 block partials; energy-weighted BCE with its gradient
__global__ void k_energy_density(const float *__restrict__ x, int B, long long V, float *__restrict__ e,
                                 double *__restrict__ part);
__global__ void k_loss(const float *__restrict__ logit, const float *__restrict__ y, const float *__restrict__ e,
                       float inv_emean, float lam, long long n, float *__restrict__ dlogit, double *__restrict__ part);

// ---------------------------------------------------------------- weight gradients on the tensor cores (wgrad_tc.cu)
// dW[co0 + co][ci0 + ci][t] = sum over cells of dZ[cell][co0 + co] X[cell + s(t)][ci0 + ci]
// for a 3x3x3 convolution (taps = 27, zero outside the volume) or a dense
// layer (taps = 1); co_n <= 32 (conv) or <= 128 (dense), ci_n <= 32 (conv) or
// <= 256 (dense).  gw has the layout [co][ci_tot][taps]; gb (optional) gets
// sum over cells of dZ.  dZ is BF16 channels-last [cells][dz_pitch], or FP32
// [cells] with one channel (dz_f32, conv only).  Deterministic.
struct WgradJob {
    const __nv_bfloat16 *x;  // [cells][x_pitch]
    int x_pitch, ci0, ci_n, ci_tot;
    const __nv_bfloat16 *dz;  // [cells][dz_pitch]
    const float *dz_f32;
    int dz_pitch, co0, co_n;
    int B, D, H, W;           // dense: B = D = H = 1, W = rows
    int taps;
    float *gw, *gb;
    int *status;
};
struct WgradScratch {
    void *buf = nullptr;
    long long bytes = 0;
    float *part = nullptr;
    long long pbytes = 0;
    ~WgradScratch() {
        if (buf) cudaFree(buf);
        if (part) cudaFree(part);
    }
};
hyb_status wgrad_tc(const WgradJob &j, WgradScratch &ws, cudaStream_t st);

}  // namespace hyb
