/*
 * hyb.h -- C ABI of the GB300-native hybrid fluid-kinetic laser-plasma step
 * (arXiv 2510.11174, "Machine Learning-Integrated Hybrid Fluid-Kinetic
 * Framework for Quantum Electrodynamic Laser-Plasma Simulations").
 *
 * The library advances, on one GPU, the paper's time step (Methodology): a
 * 3D Yee FDTD field update with first-order Mur boundaries and a Gaussian
 * laser source, a relativistic cold fluid in quiet cells, and a
 * particle-in-cell update (relativistic Boris push, charge-conserving
 * Esirkepov deposition, blended ADK/multiphoton ionization, Monte Carlo
 * radiation reaction and pair production from Airy-function rates) in the
 * cells a convolutional regime classifier flags as kinetic.
 *
 * Units (laser-normalised, wavelength lambda): length c/w0, time 1/w0,
 * momentum u = gamma*beta (p / m c), E in m_e c w0 / e, B in m_e w0 / e,
 * density in n_c = eps0 m_e w0^2 / e^2, charge in e, mass in m_e.  Particle
 * positions are in cell units (x / dx), domain [0, n) on periodic axes and
 * [0, n-1] on absorbing axes.
 *
 * Conventions common to every entry point:
 *  - every call returns hyb_status; no C++ exception crosses the ABI;
 *  - descriptors are caller-owned and copied during the call;
 *  - pointers named *_host are host memory; pointers named *_dev are device
 *    memory on the context's device; arrays passed to a call are borrowed for
 *    the duration of that call only;
 *  - calls are ordered on the context's CUDA stream and asynchronous, except
 *    hyb_diagnostics and the hyb_get_* calls, which synchronise that stream;
 *  - errors raised on the device (particle-capacity overflow, non-finite
 *    fields) are latched in a device status word and returned by the next
 *    synchronising call; a context in that state rejects hyb_step with
 *    HYB_ESTATE until hyb_clear_status;
 *  - hyb_last_error returns a human-readable message for the last failure.
 */
#ifndef HYB_H
#define HYB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYB_OK = 0,
    HYB_EINVAL = 1,     /* invalid argument or descriptor */
    HYB_ENOMEM = 2,     /* device allocation or caller arena too small */
    HYB_ECUDA = 3,      /* CUDA runtime error */
    HYB_EOVERFLOW = 4,  /* a particle tile or migration buffer overflowed */
    HYB_ENAN = 5,       /* non-finite value in fields */
    HYB_ETIMEOUT = 6,   /* a bounded device wait gave up */
    HYB_ESTATE = 7      /* context is in an error state */
} hyb_status;

enum { HYB_BC_PERIODIC = 0, HYB_BC_MUR = 1 };  /* per axis: Mur fields + reflecting particles */
enum { HYB_LASER_NONE = 0, HYB_LASER_GAUSS = 1 };

typedef struct hyb_ctx hyb_ctx;  /* opaque, library-owned */

/*
 * Grid, time step, boundaries and laser (paper, Methodology: uniform
 * Cartesian grid; constant dt from the Courant limit; first-order Mur
 * absorbers; Gaussian pulse with temporal and spatial envelopes).
 */
typedef struct {
    int nx, ny, nz;           /* cells (= nodes) per axis; multiples of `tile` */
    double dx, dy, dz;        /* cell size [c/w0] */
    double dt;                /* time step [1/w0]; if <= 0, cfl_frac * Courant limit */
    double cfl_frac;          /* used when dt <= 0 (e.g. 0.95) */
    int bc[3];                /* HYB_BC_* per axis */
    double lambda_um;         /* laser wavelength, fixes the physical scales */
    /* Gaussian soft source: current sheet J_pol on the plane x = x_src
     * (node index), field amplitude a0, intensity FWHM tau_fwhm [1/w0],
     * 1/e^2 intensity radius w0_spot [c/w0], centre (y_c, z_c) [cells],
     * peak time t_peak [1/w0]; pol 1 = y, 2 = z. */
    int laser_kind;
    double a0, tau_fwhm, w0_spot, t_peak, y_c, z_c;
    int x_src, pol;
    uint32_t seed;            /* Philox key word 0 */
    int tile;                 /* tile edge in cells (4 or 8; 0 = 8) */
    void *stream;             /* cudaStream_t the context runs on (NULL = legacy default) */
    void *arena_dev;          /* optional caller-provided device arena (e.g. a torch tensor) */
    size_t arena_bytes;       /* its size; all library buffers come from it when non-NULL */
    /* Particle shape of the gather and the Esirkepov deposition: 1 (or 0) the
     * linear CIC shape, 2 the quadratic TSC shape (Esirkepov's scheme for any
     * shape order; smoother, less grid noise).  The quadratic shape needs
     * periodic axes (its stencil reaches past an absorbing wall) and a context
     * without fluid <-> particle conversions (those deposit with CIC);
     * HYB_EINVAL otherwise. */
    int shape_order;
} hyb_grid_desc;

/*
 * A macro-particle species (paper, Methodology: PIC macro-particles weighted
 * by density-volume fraction; electrons, ions and positrons).
 * Initial particles are passed explicitly as SoA FP32 arrays (positions in
 * cell units, u = gamma*beta, weight in n_c (c/w0)^3), either host or device
 * memory as `ptr_on_device` says.  ids (uint64) identify particles across
 * tile migrations and key their random streams; NULL assigns 0..n-1.
 */
typedef struct {
    double q, m;              /* charge [e], mass [m_e] */
    long long n;              /* initial particle count */
    long long tile_capacity;  /* slots per tile; 0 = 2 x max initial count per tile + 64 */
    int ptr_on_device;        /* 1: arrays below are device pointers */
    const float *x, *y, *z, *ux, *uy, *uz, *w;
    const float *zq;          /* per-particle charge state (ions, q_p = q * zq) or NULL */
    const uint64_t *ids;      /* or NULL */
    /* Field ionization (paper, Methodology: ADK tunnelling and multiphoton
     * rates blended by a sigmoid at Keldysh parameter ~1.5).  zmax > 0 makes
     * the species ionizable up to charge state zmax (zq required); ip_eV[Z]
     * and l_qn[Z] are the ionization potential and orbital quantum number of
     * the electron removed in Z -> Z+1; new electrons join species
     * ionize_into (already loaded, charge -1, mass 1).  Rates come from an
     * FP64-built table on the device; events use Philox with key (seed,
     * species id) and counter (id, step, 1). */
    int zmax;
    double ip_eV[8];
    int l_qn[8];
    int ionize_into;
    /* Strong-field QED (paper, Methodology: radiation reaction and pair
     * production from Airy-function rates with the local field).  kind =
     * HYB_KIND_PHOTON makes a photon species (q = 0, u holds the momentum k
     * in m c, moves at c).  qed = 1 on a lepton species turns on photon
     * emission with recoil (optical-depth Monte Carlo, LCFA spectrum);
     * photons of energy >= photon_eps_min [m c^2] (0 = 2) join species
     * photon_species (-1: their energy is only tallied).  On a photon
     * species, pair_electron / pair_positron (-1: none) receive Breit-Wheeler
     * pairs.  Rates and spectra come from FP64-built tables on the device;
     * events use Philox counters (id, step, 2) for emission and (id, step, 3)
     * for pairs. */
    int kind;
    int qed;
    int photon_species;
    double photon_eps_min;
    int pair_electron, pair_positron;
    /* Momentum update (paper, Methodology: relativistic particle pusher):
     * HYB_PUSH_BORIS (Boris, the default), HYB_PUSH_VAY (Vay 2008) or
     * HYB_PUSH_HIGUERA_CARY (Higuera & Cary 2017); the last two move a
     * particle at the relativistic E x B drift velocity without spurious force. */
    int pusher;
} hyb_species_desc;

enum { HYB_KIND_MASSIVE = 0, HYB_KIND_PHOTON = 1 };
enum { HYB_PUSH_BORIS = 0, HYB_PUSH_VAY = 1, HYB_PUSH_HIGUERA_CARY = 2 };

/*
 * A cold relativistic fluid species on the nodes (paper, Methodology: fluid
 * continuity and momentum equations with relativistic gamma factors for the
 * bulk plasma in stable regions; clamping against instability).  n is the
 * density [n_c] and u = gamma beta, each an array of nz*ny*nx values at the
 * nodes (x fastest); ux/uy/uz may be NULL (u = 0).  Host or device memory as
 * ptr_on_device says.  Transport is first-order donor cell on the node
 * control volumes; the face fluxes times q are added to J on the Yee edges,
 * so charge is conserved exactly.  Where the new density is below n_floor
 * (0 = 1e-10) u is set to 0; negative densities are clamped to 0 and counted.
 */
typedef struct {
    double q, m;
    int ptr_on_device;
    const float *n, *ux, *uy, *uz;
    double n_floor;
    /* Warm fluid (the paper's fluid model carries an adiabatic pressure):
     * temperature_keV > 0 adds the pressure p = n_ref T (n / n_ref)^gamma_ad
     * (gamma_ad 0 = 5/3, n_ref 0 = 1 n_c) to the momentum equation, -grad p / m,
     * applied with the Lorentz force before the transport with central face
     * pressures (a wall reflects the pressure).  0 keeps the fluid cold. */
    double temperature_keV, gamma_ad, n_ref;
} hyb_fluid_desc;

/* Diagnostics: FP64 energy reductions (paper, Methodology: total energy from
 * electromagnetic, kinetic and thermal components) and device status. */
#define HYB_MAX_SPECIES 8
#define HYB_MAX_FLUIDS 4
typedef struct {
    long long step;
    double time;                           /* [1/w0] */
    double w_e, w_b;                       /* field energy (1/2) sum E^2 dV, (1/2) sum B^2 dV */
    double w_kin[HYB_MAX_SPECIES];         /* sum w m (gamma - 1) per species */
    long long count[HYB_MAX_SPECIES];      /* live macro-particles per species */
    int n_species;
    int status;                            /* latched device status (hyb_status) */
    long long launches_per_step;           /* kernels one step launches */
    double w_ionize;                       /* energy spent on ionization so far, sum w Ip */
    long long n_ionize;                    /* ionization events so far */
    double w_photon_untracked;             /* energy of emitted photons below the tracking threshold */
    double w_pair_deficit;                 /* pair energy below m c^2 that could not become momentum */
    long long n_emit;                      /* photon emission events so far */
    long long n_pair;                      /* pair creation events so far */
    int n_fluids;
    double w_fluid[HYB_MAX_FLUIDS];        /* sum n m (gamma - 1) dV per fluid */
    double n_fluid[HYB_MAX_FLUIDS];        /* sum n dV per fluid */
    long long n_clamped;                   /* fluid nodes clamped from negative density so far */
    long long launches_classify;           /* kernels the most recent hyb_classify launched */
    long long tile_capacity[HYB_MAX_SPECIES];  /* current slots per tile of each species */
    long long classified_cells;            /* nodes whose statistics the most recent classification with a
                                              model computed (all of them unless hyb_regime_desc.reach
                                              restricted it) */
    long long fluid_cells;                 /* nodes the fluid update covers now (all of them unless a
                                              classification with a reach restricted it) */
} hyb_diag;

/* Create a context: validates the descriptor, allocates fields on the
 * context's stream and zeroes them.  Returns HYB_EINVAL for a bad descriptor
 * (grid not a multiple of the tile, fewer than 4 nodes on a Mur axis, dt above
 * the Courant limit, ...), HYB_ENOMEM when the arena is too small. */
hyb_status hyb_init_grid(const hyb_grid_desc *desc, hyb_ctx **out);
void hyb_destroy(hyb_ctx *ctx);

/* Add a species; writes its id (0, 1, ...) to *species_id.  Particles are
 * binned into tiles on the device.  HYB_EOVERFLOW if a tile exceeds its
 * capacity. */
hyb_status hyb_load_species(hyb_ctx *ctx, const hyb_species_desc *desc, int *species_id);

/*
 * Regime switching (paper, Methodology: fluid in stable regions, PIC where
 * SwitchNet flags instability; charge and energy checked at switches).  The
 * paper does not define the instability criterion; the physics criterion
 * marks a node kinetic when |E| >= a_thr, or the electron density (fluid +
 * CIC of electron macro-particles) >= n_thr [n_c], or dt div v_e <= -c_thr
 * (electron fluid), or kappa gamma |E| >= chi_thr; the mask is then dilated by
 * `dilate` nodes.  With a classifier, a node is kinetic when
 * p_mean + k_sigma p_std >= 0.5 (same dilation).  Conversions: fluid f at
 * nodes that switch to kinetic (kinetic now, fluid at the previous
 * classification; every node counts as fluid before the first one) becomes
 * ppc macro-particles of species to_species[f]
 * (Philox-uniform in the node's dual cell, the fluid's u, weight n dV / ppc);
 * particles of species to_species[f] whose nearest node is fluid are
 * deposited (CIC) into fluid f.  A residual background charge keeps
 * div E - rho - rho_bg unchanged across conversions.  to_species[f] = -1:
 * fluid f is not converted.
 */
typedef struct {
    double a_thr, n_thr, c_thr, chi_thr;  /* 0 = defaults 1, 1, 0.1, 1e-3 */
    int dilate;                           /* nodes (e.g. 2) */
    double k_sigma;                       /* classifier decision: p_mean + k_sigma p_std >= 0.5 */
    int ppc;                              /* macro-particles per node created from fluid */
    int to_species[HYB_MAX_FLUIDS];
    int policy;                           /* HYB_REGIME_* below */
    int quiet;                            /* 1: quiet start -- the ppc particles of a converted node sit
                                             at the centres of an lx x ly x lz sub-lattice of its dual
                                             cell (lx >= ly >= lz, lz the largest divisor of ppc not
                                             above its cube root, ly the largest divisor of ppc / lz not
                                             above its square root), the same in every run, so that a
                                             uniform fluid becomes particles without shot noise;
                                             0: Philox-uniform positions */
    int reach;                            /* 0: the classifier runs on every node.  r > 0: it runs only on
                                             the nodes whose x lies within r + dilate nodes of an x-plane
                                             holding matter (a fluid above its n_floor at a node of the
                                             plane, or a particle with floor(x) in it); p_mean = p_std = 0
                                             on the other nodes.  Fluid moves at most one node per step and
                                             particles less, so with r at least the number of steps to the
                                             next classification plus one (a particle's CIC node) the
                                             decision differs from the whole-grid one only where no matter
                                             can be before then, and the run (conversions, fields,
                                             particles) is the same.  hyb_classify then synchronises the
                                             context stream to read the matter's x-extent, and, once a step
                                             has run since the fluids were loaded, restricts the fluid
                                             update of the next r steps to the planes within r of nonzero
                                             fluid density (fluid spreads one node per step; the planes
                                             left out stay empty): also exact; hyb_step lifts the
                                             restriction when it lapses. */
} hyb_regime_desc;
/* Which decision hyb_classify takes.  DEFAULT: the classifier when a model is
 * given, else the physics criterion.  UNION: a node is kinetic when the
 * classifier or the physics criterion says so (the thresholds act as prior
 * knowledge the network can only add to).  ALL_KINETIC: every node is
 * kinetic, i.e. all fluid becomes macro-particles (the full-PIC run, the
 * reference for the hybrid's error). */
#define HYB_REGIME_DEFAULT 0
#define HYB_REGIME_UNION 1
#define HYB_REGIME_ALL_KINETIC 2
hyb_status hyb_set_regime(hyb_ctx *ctx, const hyb_regime_desc *desc);

/* Recompute the regime mask and convert (stream-ordered).  model = NULL uses
 * the physics criterion; otherwise the classifier runs mc_passes MC-dropout
 * passes (see hyb_model_*).  Optional device outputs of nz*ny*nx values:
 * p_mean_dev, p_std_dev (NULL with the physics criterion) and mask_dev
 * (1 = kinetic). */
typedef struct hyb_model hyb_model;
hyb_status hyb_classify(hyb_ctx *ctx, const hyb_model *model, float *p_mean_dev, float *p_std_dev,
                        uint8_t *mask_dev);

/*
 * Regime classifier (paper, Methodology and Results: a convolutional network
 * on per-channel normalised fields decides fluid vs PIC; Monte Carlo dropout
 * gives its uncertainty; training uses a physics-informed energy term).  The
 * network is a 3D CNN 6 -> 32 -> 32 -> 16 -> 1 with 3x3x3 kernels, zero
 * "same" padding, ReLU and dropout(p) after each hidden layer and a sigmoid
 * output; input channels are E_x, E_y, E_z, B_x, B_y, B_z at the nodes,
 * normalised per channel as (x - mean_c) / std_c.  Weights are kept in FP32
 * (Adam master copy) and used in BF16 with FP32 accumulation; activations
 * between layers are BF16.  Dropout masks come from Philox (key (seed,
 * 0xD0), counter (cell, batch, layer << 16 | channel / 8, pass)): channel c
 * is kept when 16-bit field c % 8 of the output (word (c % 8) / 2, low half
 * for even c) is >= round(p 2^16); p is used as round(p 2^16) / 2^16.
 */
typedef struct {
    double dropout;            /* p (e.g. 0.2) */
    int mc_passes;             /* MC-dropout passes at classification (e.g. 16) */
    uint32_t seed;             /* initialisation and dropout streams */
    float mean[6], std[6];     /* per-channel normalisation of the input */
    double lr, beta1, beta2, eps;  /* Adam (0 = 1e-3, 0.9, 0.999, 1e-8) */
    double energy_weight;      /* lambda of the energy-weighted BCE (e.g. 0.1) */
    void *stream;              /* cudaStream_t (NULL: own stream) */
} hyb_model_desc;
hyb_status hyb_model_create(const hyb_model_desc *desc, hyb_model **out);
void hyb_model_destroy(hyb_model *model);

/* Weights as FP32 host arrays in the layout [c_out][c_in][kz][ky][kx] (x
 * fastest), biases [c_out]; layers 0..3 have (c_in, c_out) = (6, 32),
 * (32, 32), (32, 16), (16, 1).  hyb_model_create initialises them
 * He-uniform from the seed. */
hyb_status hyb_model_set_layer(hyb_model *model, int layer, const float *w_host, const float *b_host);
hyb_status hyb_model_get_layer(hyb_model *model, int layer, float *w_host, float *b_host);

/* One forward pass over patches x_dev (device FP32, [batch][6][D][H][W]):
 * writes the logits (device FP32, [batch][D][H][W]).  pass >= 0 applies the
 * dropout masks of that pass; pass < 0 disables dropout.  W % 8 == 0 and
 * H % 16 == 0.  Stream-ordered. */
hyb_status hyb_model_forward(hyb_model *model, const float *x_dev, int batch, int D, int H, int W, int pass,
                             float *logits_dev);

/*
 * One training step (paper, Methodology: the network is trained on data the
 * simulation generates, with a physics-informed energy-conservation term in
 * the loss).  patches_dev: device FP32 [batch][6][D][H][W] (E, B);
 * labels_dev: device FP32 [batch][D][H][W] in {0, 1} (1 = kinetic).  The loss
 * is the energy-weighted binary cross-entropy
 *   L = (1/N) sum_c w_c BCE(sigmoid(logit_c), y_c),
 *   w_c = 1 + energy_weight * e_c / mean(e),  e_c = (|E|^2 + |B|^2)/2 at c,
 * so cells holding more field energy weigh more (the reading of the paper's
 * energy term for a regime label).  Dropout is on with the masks of pass =
 * the step index; gradients flow through the same BF16 tensor-core
 * convolutions (data gradient = convolution with the transposed, flipped
 * kernel), weight gradients are tensor-core contractions over the cells
 * (BF16 operands, among them bf16(dL/dlogit) for the last layer, FP32
 * accumulation, partial sums of the SMs added in a fixed order), and Adam
 * updates the FP32 master weights.  Synchronises; fills *out.
 */
typedef struct {
    double loss;       /* L above */
    double bce;        /* unweighted mean BCE */
    double accuracy;   /* fraction of cells with (p >= 0.5) == y */
    long long step;    /* Adam step count after this update */
} hyb_train_stats;
hyb_status hyb_train_step(hyb_model *model, const float *patches_dev, const float *labels_dev, int batch, int D,
                          int H, int W, hyb_train_stats *out);

/* Gradients of the last training step (FP32 host arrays in the layout of
 * hyb_model_get_layer). */
hyb_status hyb_model_get_grad(hyb_model *model, int layer, float *gw_host, float *gb_host);

/* The classifier's input channels at the nodes, as the classification forms
 * them but not normalised: E_x, E_y, E_z averaged over the two Yee edges that
 * meet at the node, B_x, B_y, B_z over the four faces around it (zero outside
 * an absorbing axis), written to out_dev (device FP32, [6][nz][ny][nx]).  The
 * paper trains its networks on data the simulation generates (Methodology):
 * this is where training patches are cut from a run.  Stream-ordered. */
hyb_status hyb_node_fields(hyb_ctx *ctx, float *out_dev);

/* The plasma state at the nodes (the field surrogate's channels): E_x, E_y,
 * E_z and B_x, B_y, B_z as hyb_node_fields forms them, J_x, J_y, J_z of the
 * last step averaged over the two Yee edges that meet at the node (zero
 * outside an absorbing axis), and the charge density rho at the node: the
 * CIC deposit of every charged particle species (q w / dV, times the charge
 * state where a species has one), plus q n of every fluid, plus the residual
 * background charge of the regime conversions.  out_dev: device FP32
 * [10][nz][ny][nx].  The paper's predictor takes E, B, J and rho (Results:
 * state transitions of normalised E, B, J and rho).  Stream-ordered. */
hyb_status hyb_node_state(hyb_ctx *ctx, float *out_dev);

/*
 * Field surrogate: the paper's StatePredictor (Results, Table 2), a 3D CNN
 * that maps the normalised state of a patch (10 channels: E, B, J, rho) to
 * the state a fixed number of steps later.  Layers (3x3x3 convolutions, zero
 * "same" padding, BF16 weights and activations, FP32 accumulation):
 *   a1 = bf16(relu(conv(x; 10 -> 13)) + pad(x))
 *   a2 = bf16(dropout(relu(conv(a1; 13 -> 32))) + pad(a1))      dropout p
 *   a3 = bf16(relu(conv(a2; 32 -> 64)) + pad(a2))
 *   a4 = bf16(relu(conv(a3; 64 -> 128)))
 *   a5 = bf16(relu(conv(a4; 128 -> 32)))
 *   y  = conv(a5; 32 -> 10)                                      (FP32)
 * "pad" is the identity shortcut with the missing channels zero (Table 2's
 * residuals between layers of different width).  x = (s - mean_c) / std_c
 * per channel; y is the change of the state over the lead time in units
 * dstd_c (the spread of that change, std_c when not given), and the
 * prediction is s_c + dstd_c y_c (a residual forecast: with every weight zero
 * it is the input state).
 * Dropout uses the classifier's Philox stream (key (seed, 0xD0), counter
 * (cell, batch, 1 << 16 | channel / 8, pass)).
 * Training loss (Table 2: Huber with delta = 0.01 and 0.1 on the energy
 * violation): L = (1/N) sum huber_delta(y - t) + energy_weight v^2, t the
 * target change (target - s) / dstd_c, N the number of values, and v the relative violation
 * of the batch's total field energy, v = (sum_b W(pred_b) - sum_b
 * W(target_b)) / sum_b W(target_b), W = (1/2) sum over a patch of |E|^2 +
 * |B|^2 of the de-normalised channels 0..5 (a batch without field energy
 * has no energy term).  Adam on FP32 master weights.  Patches need
 * W % 8 == 0 and H % 16 == 0.
 */
typedef struct hyb_surrogate hyb_surrogate;
typedef struct {
    uint32_t seed;             /* He-uniform initialisation and dropout stream */
    double dropout;            /* p after layer 1 (Table 2: 0.1) */
    int mc_passes;             /* passes of hyb_surrogate_mc */
    double lr, beta1, beta2, eps;  /* Adam */
    double huber_delta;        /* 0.01 */
    double energy_weight;      /* 0.1 */
    float mean[10], std[10];   /* per-channel normalisation of the input state */
    float dstd[10];            /* unit of the predicted change per channel (its spread); 0: std */
    void *stream;              /* cudaStream_t (NULL: own stream) */
} hyb_surrogate_desc;
hyb_status hyb_surrogate_create(const hyb_surrogate_desc *desc, hyb_surrogate **out);
void hyb_surrogate_destroy(hyb_surrogate *s);
/* Layers 0..5 in the layout [c_out][c_in][kz][ky][kx], biases [c_out];
 * (c_in, c_out) = (10, 13), (13, 32), (32, 64), (64, 128), (128, 32), (32, 10). */
hyb_status hyb_surrogate_set_layer(hyb_surrogate *s, int layer, const float *w_host, const float *b_host);
hyb_status hyb_surrogate_get_layer(hyb_surrogate *s, int layer, float *w_host, float *b_host);
/* Prediction for states x_dev (device FP32 [batch][10][D][H][W]) into y_dev
 * (same layout, de-normalised).  pass >= 0 applies that pass's dropout masks,
 * pass < 0 none.  Stream-ordered. */
hyb_status hyb_surrogate_forward(hyb_surrogate *s, const float *x_dev, int batch, int D, int H, int W, int pass,
                                 float *y_dev);
/* Monte Carlo dropout: mc_passes passes (pass index 0 .. mc_passes - 1);
 * mean and population standard deviation of the de-normalised prediction
 * per value (device FP32, layout of x).  Stream-ordered. */
hyb_status hyb_surrogate_mc(hyb_surrogate *s, const float *x_dev, int batch, int D, int H, int W, float *mean_dev,
                            float *std_dev);
typedef struct {
    double loss;       /* L above */
    double huber;      /* mean Huber term */
    double energy;     /* v^2 */
    long long step;    /* Adam step count after this update */
} hyb_surrogate_stats;
/* One training step on states x_dev and targets t_dev (device FP32,
 * [batch][10][D][H][W], not normalised); dropout masks of pass = the step
 * index.  Synchronises; fills *out. */
hyb_status hyb_surrogate_train_step(hyb_surrogate *s, const float *x_dev, const float *t_dev, int batch, int D,
                                    int H, int W, hyb_surrogate_stats *out);
/* Gradients of the last training step, in the layout of hyb_surrogate_get_layer. */
hyb_status hyb_surrogate_get_grad(hyb_surrogate *s, int layer, float *gw_host, float *gb_host);

/*
 * SwitchNet: the paper's per-cell regime classifier (Table 1; Results: AUC
 * against the convolutional classifier).  Input: the ten node channels of
 * hyb_node_state for every cell, x = (s - mean_c) / std_c.  Layers (BF16
 * weights and activations, FP32 accumulation):
 *   h1 = bf16(relu(W0 x + b0) + pad(x))                        10 -> 128
 *   h2 = bf16(dropout(relu(W1 h1 + b1)) + pad(h1))             128 -> 256, p
 *   v  = bf16(Wv h2 + bv),  o = bf16(Wo v + bo)                 the attention layer
 *   logit = w4 . o + b4,  p = sigmoid(logit)
 * The attention layer (4 heads, 256 -> 256) sees one feature vector per cell,
 * a sequence of one token: its softmax over the single key is 1, so it is the
 * value projection followed by the output projection.  "pad" is the identity
 * shortcut with the missing channels zero.  Dropout uses the classifier's
 * Philox stream (layer index 1, counter (cell, 0, 1 << 16 | channel / 8,
 * pass)).  Training: the classifier's energy-weighted BCE (w_c = 1 +
 * energy_weight e_c / mean(e), e_c = (|E|^2 + |B|^2) / 2 of the raw
 * features), Adam on FP32 masters.
 */
typedef struct hyb_switchnet hyb_switchnet;
typedef struct {
    uint32_t seed;             /* He-uniform initialisation and dropout stream */
    double dropout;            /* p after layer 1 (Table 1: 0.2) */
    int mc_passes;             /* passes of hyb_switchnet_mc */
    double lr, beta1, beta2, eps;  /* Adam */
    double energy_weight;      /* lambda of the energy-weighted BCE */
    float mean[10], std[10];   /* per-channel normalisation */
    void *stream;              /* cudaStream_t (NULL: own stream) */
} hyb_switchnet_desc;
hyb_status hyb_switchnet_create(const hyb_switchnet_desc *desc, hyb_switchnet **out);
void hyb_switchnet_destroy(hyb_switchnet *s);
/* Layers 0..4: W [c_out][c_in] and b [c_out] with (c_in, c_out) = (10, 128),
 * (128, 256), (256, 256) value, (256, 256) output projection, (256, 1). */
hyb_status hyb_switchnet_set_layer(hyb_switchnet *s, int layer, const float *w_host, const float *b_host);
hyb_status hyb_switchnet_get_layer(hyb_switchnet *s, int layer, float *w_host, float *b_host);
/* Logits of n cells, x_dev device FP32 [10][n]; pass >= 0 applies that
 * pass's dropout.  Stream-ordered. */
hyb_status hyb_switchnet_forward(hyb_switchnet *s, const float *x_dev, long long n, int pass, float *logit_dev);
/* MC dropout: mean and population standard deviation of sigmoid(logit) over
 * mc_passes passes (device FP32 [n] each).  Stream-ordered. */
hyb_status hyb_switchnet_mc(hyb_switchnet *s, const float *x_dev, long long n, float *p_mean_dev, float *p_std_dev);
/* One Adam step on n cells: features x_dev [10][n], labels y_dev [n] in {0, 1};
 * dropout masks of pass = the step index.  Synchronises; fills *out. */
hyb_status hyb_switchnet_train_step(hyb_switchnet *s, const float *x_dev, const float *y_dev, long long n,
                                    hyb_train_stats *out);
/* Gradients of the last training step, in the layout of hyb_switchnet_get_layer. */
hyb_status hyb_switchnet_get_grad(hyb_switchnet *s, int layer, float *gw_host, float *gb_host);

/* Copy the current mask (uint8, 1 = kinetic) and the residual background
 * charge rho_bg (FP32) to host arrays of nz*ny*nx values (either may be NULL;
 * synchronises). */
hyb_status hyb_get_regime(hyb_ctx *ctx, uint8_t *mask_host, float *rho_bg_host);

/* Add a cold fluid species; writes its id (0, 1, ...) to *fluid_id. */
hyb_status hyb_load_fluid(hyb_ctx *ctx, const hyb_fluid_desc *desc, int *fluid_id);

/* Copy a fluid back (synchronises): n, ux, uy, uz host arrays of nz*ny*nx
 * values (any may be NULL). */
hyb_status hyb_get_fluid(hyb_ctx *ctx, int fluid_id, float *n, float *ux, float *uy, float *uz);

/* Replace the fields E, B (each: 3 contiguous FP32 arrays of nz*ny*nx
 * values, x fastest, Yee-staggered as documented in the library).  Host or
 * device memory as on_device says. */
hyb_status hyb_set_fields(hyb_ctx *ctx, const float *E, const float *B, int on_device);

/* Advance n steps (stream-ordered; the step sequence is captured once into a
 * CUDA graph and replayed).  Tiles have a fixed number of slots per species;
 * every 4 steps the compaction's fill flags travel to the host behind the
 * steps (the host never runs more than 4 steps ahead of the last flags it
 * read), and once a species' tiles have passed half of their slots hyb_step
 * synchronises and doubles that species' slots per tile (its particles are
 * copied tile by tile) before the next steps.  A tile that overflows before
 * that drops particles and latches HYB_EOVERFLOW. */
hyb_status hyb_step(hyb_ctx *ctx, int nsteps);

/* Batches of independent runs (many laser and plasma parameters, uneven grids,
 * advanced together).  A batch replays the captured step of each of its
 * contexts as one CUDA graph whose branches do not depend on each other, so
 * the GPU runs small grids side by side.  hyb_batch_step(b, n) advances every
 * context by n steps on the batch's stream (`stream`, or a stream of its own
 * when NULL): it first waits for the work already queued on each context's
 * stream and leaves each context's stream waiting for the batch, so calls on
 * a context before and after stay ordered.  Capacity growth works as in
 * hyb_step.  Contexts must be distinct and on the current device; a context
 * may belong to several batches but must not be stepped by two at once.  The
 * batch does not own its contexts: destroy it before them. */
typedef struct hyb_batch hyb_batch;
hyb_status hyb_batch_create(hyb_ctx *const *ctxs, int n, void *stream, hyb_batch **out);
hyb_status hyb_batch_step(hyb_batch *batch, int nsteps);
void hyb_batch_destroy(hyb_batch *batch);

/* Synchronises; fills *out. */
hyb_status hyb_diagnostics(hyb_ctx *ctx, hyb_diag *out);

/* Copy fields back (synchronises): E, B, J each 3*nz*ny*nx floats (host). */
hyb_status hyb_get_fields(hyb_ctx *ctx, float *E_host, float *B_host, float *J_host);

/* Copy a species back in tile order (synchronises).  Arrays of `max_n`
 * entries; *n_out receives the live count (HYB_EINVAL if > max_n).
 * zq may be NULL. */
hyb_status hyb_get_species(hyb_ctx *ctx, int species_id, long long max_n, float *x, float *y,
                           float *z, float *ux, float *uy, float *uz, float *w, float *zq,
                           uint64_t *ids, long long *n_out);

/* Checkpoint (paper, Methodology: runs are kept reproducible through stored
 * parameters, data and fixed random streams).
 * hyb_get_state writes the whole state of the context -- the fields E, B, J,
 * the Mur history planes, the regime mask, the previous mask and the residual
 * background charge, every species' particles (positions, momenta, weights,
 * charge states, optical depths, ids), per-tile event tallies and tile
 * capacity, every fluid with its clamp count, the step and conversion
 * counters, the regime settings and the device status word -- into the host
 * buffer buf_host of `cap` bytes, and its size into *size_out.  With buf_host
 * NULL only the size is reported; a `cap` below the size gives HYB_EINVAL
 * (with the size reported).  The image holds no pointers and no classifier
 * (hyb_model_get_layer saves a network).  Synchronises.
 * hyb_set_state restores such an image into a context created with the same
 * grid descriptor (grid, cell size, time step, boundaries, seed, tile) and
 * loaded with the same species (charge, mass, kind, ionization and QED
 * flags) and fluids, in the same order; anything else returns HYB_EINVAL
 * before the context is changed.  Particles are binned into their tiles again
 * (their slot order inside a tile may differ; nothing the step computes
 * depends on it), tile capacities become the saved ones and the step graph is
 * captured again at the next hyb_step.  Random events draw from streams keyed
 * by particle id and step, and the current deposition does not depend on the
 * particle order, so N steps, a save, a restore into a fresh context and M
 * more steps give the fields and particles of N + M uninterrupted steps bit
 * for bit.  Temporary device memory for the particles comes from the arena
 * when the context has one.  Synchronises. */
hyb_status hyb_get_state(hyb_ctx *ctx, void *buf_host, size_t cap, size_t *size_out);
hyb_status hyb_set_state(hyb_ctx *ctx, const void *buf_host, size_t size);

/* Resets the latched device status word. */
hyb_status hyb_clear_status(hyb_ctx *ctx);

/* Failure detection (paper, Methodology: the stability of the run is checked,
 * values are clamped and unstable steps are skipped).  The device latches
 * overflow, non-finite fields and wait timeouts; these two calls let a caller
 * exercise those paths without faulting the GPU.
 * hyb_set_auto_grow(ctx, 0) turns off the growth of full particle tiles
 * (on by default): a tile that overflows then drops the particles it cannot
 * hold and latches HYB_EOVERFLOW.
 * hyb_selftest_wait_timeout(ctx, polls) enqueues one kernel that waits, with
 * the same bounded mbarrier wait as the tensor-core pipelines, on a barrier
 * that nothing completes; after `polls` polls (1..2^20, HYB_EINVAL outside) it
 * gives up and latches HYB_ETIMEOUT, which the next synchronising call
 * returns.  The context stays usable; hyb_clear_status resets it. */
hyb_status hyb_set_auto_grow(hyb_ctx *ctx, int on);
hyb_status hyb_selftest_wait_timeout(hyb_ctx *ctx, long long polls);

/* Per-phase timing of a step.  With profiling on, the captured step graph
 * records a CUDA event (on the context's stream) at every phase boundary;
 * hyb_phase_times synchronises and returns the device time of each phase of
 * the most recent step in milliseconds (0 for phases the step does not run);
 * the two hyb_classify phases report the most recent classification.
 * Turning profiling on or off rebuilds the step graph. */
enum {
    HYB_PH_PUSH = 0,      /* gather + Boris + move + Esirkepov into tile frames */
    HYB_PH_JREDUCE = 1,   /* fixed-order sum of tile frames into J */
    HYB_PH_SOURCE = 2,    /* laser soft source */
    HYB_PH_REBIN = 3,     /* migration + compaction of particle tiles */
    HYB_PH_FIELD = 4,     /* B half, E, Mur, B half */
    HYB_PH_FLUID = 5,     /* cold fluid Lorentz step, transport, face currents */
    HYB_PH_CLASSIFY = 6,  /* hyb_classify: classifier forward over the MC-dropout passes */
    HYB_PH_REGIME = 7,    /* hyb_classify: decision, dilation, conversions */
    HYB_PH_CONV1 = 8,     /* hyb_classify: the 32 -> 32 convolutions, summed over the MC passes */
    HYB_PH_CONV2 = 9,     /* hyb_classify: the 32 -> 16 convolutions, summed over the MC passes */
    HYB_NPHASE = 10
};
typedef struct {
    float ms[HYB_NPHASE];
} hyb_phase_times_t;
hyb_status hyb_set_profiling(hyb_ctx *ctx, int on);
hyb_status hyb_phase_times(hyb_ctx *ctx, hyb_phase_times_t *out);

/* Evaluate a device rate table the way the step does, for n field values.
 * table = HYB_LUT_IONIZE: the ionization rate w [1/atomic time] of species
 * `species_id`, charge state `level`, at field strengths x_host[i] given in
 * atomic units.  Host arrays of n values; synchronises. */
enum { HYB_LUT_IONIZE = 0 };
hyb_status hyb_eval_rate_table(hyb_ctx *ctx, int table, int species_id, int level, const float *x_host, int n,
                               float *out_host);

/* Evaluate the device QED tables the way the step does, for n points:
 * what = HYB_QED_H: h(chi) (photon emission rate = alpha/kappa * h / gamma);
 * HYB_QED_T: T(chi) (pair rate = alpha/kappa * T / eps); HYB_QED_EM_SAMPLE:
 * the photon energy fraction xi drawn for (chi, r); HYB_QED_PAIR_SAMPLE: the
 * electron energy fraction for (chi, r).  chi_host, r_host (r only for the
 * samplers) and out_host hold n values; synchronises.  The tables are built
 * on first use (or by a QED species load). */
enum { HYB_QED_H = 0, HYB_QED_T = 1, HYB_QED_EM_SAMPLE = 2, HYB_QED_PAIR_SAMPLE = 3 };
hyb_status hyb_eval_qed(hyb_ctx *ctx, int what, const float *chi_host, const float *r_host, int n, float *out_host);

/* Field energy without any device allocation.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc -- code that must
 * not synchronise the device mid-loop (cudaMalloc/cudaFree can), code whose
 * device memory is all owned by another allocator, code with a memory budget
 * fixed at start-up.  It computes what hyb_diagnostics reports as w_e and w_b,
 * out_dev[0] = (1/2) sum E^2 dV and out_dev[1] = (1/2) sum B^2 dV (FP64,
 * deterministic), for E_dev, B_dev laid out like the context's fields (3
 * component-major FP32 arrays of n_cells values each) and out_dev pointing to 2
 * doubles, all device memory of the current device; the work is enqueued on
 * `stream` (cudaStream_t, NULL = legacy default) and the call returns without
 * waiting.  Block partial sums live in a fixed file-scope device array of
 * 64 KiB that every GPU loading the library holds until exit, so n_cells is
 * limited to HYB_NOALLOC_MAX_CELLS (HYB_EINVAL beyond it).  The first call on a
 * device looks up that array's device address (make it before any stream
 * capture) and keeps it for the life of the process: after cudaDeviceReset, or
 * anything else that destroys the device's primary context, that address is
 * stale, so do not call this entry point again in that process.  Every call overwrites the partial sums it reads, so nothing needs
 * clearing, but all calls share the array: calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised
 * by the caller.  No cudaMalloc, cudaFree or allocating library routine is
 * called. */
#define HYB_NOALLOC_MAX_CELLS 22369621LL
hyb_status hyb_field_energy_noalloc(const float *E_dev, const float *B_dev, long long n_cells, double dx, double dy,
                                    double dz, double *out_dev, void *stream);

/* Message for the last failing call on this thread (never NULL). */
const char *hyb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HYB_H */
