/*
 * FP64 CPU oracle for the hybrid fluid-kinetic laser-plasma step of
 * arXiv 2510.11174 ("Machine Learning-Integrated Hybrid Fluid-Kinetic Framework
 * for Quantum Electrodynamic Laser-Plasma Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code; only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * The paper prints no equations.  Every routine here is the plain textbook
 * algorithm that the paper names (Methodology section), written as scalar
 * loops in double precision so that it can be checked against the cited
 * source by eye.  Units are laser-normalised: length c/w0, time 1/w0,
 * momentum u = p/(m_e c) = gamma*beta, fields in m_e c w0 / e, density in n_c,
 * charge in e, mass in m_e.  In these units Maxwell's equations read
 * dB/dt = -curl E, dE/dt = curl B - J, div E = rho.
 *
 * Particle positions are stored in cell units (xi = x/dx) so that the CIC
 * shape of a particle needs no division.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- grid ---------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    int bc[3];               /* 0 = periodic, 1 = first-order Mur fields + reflecting particles */
    int order;               /* particle shape: 1 (CIC, also 0) or 2 (quadratic, TSC) */
} orc_grid;

/* field component staggering (Yee 1966): offset of each component in cell units */
enum { ORC_EX = 0, ORC_EY, ORC_EZ, ORC_BX, ORC_BY, ORC_BZ };

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);  /* ((x>>9)+0.5)*2^-23, exactly representable in FP32 */

/* ---- FDTD --------------------------------------------------------------- */
void orc_fdtd_b_half(const orc_grid *g, const double *E[3], double *B[3]);
void orc_fdtd_e(const orc_grid *g, double *E[3], const double *B[3], const double *J[3]);

/* ---- laser ------------------------------------------------------------- */
void orc_laser_source(const orc_grid *g, int x_src, int pol, double a0, double tau, double t_peak,
                      double w0, double y_c, double z_c, long step, double *J[3]);

/* ---- particles ---------------------------------------------------------- */
typedef struct {
    double q, m;             /* charge (e) and mass (m_e) of the species */
    long n;
    double *x, *y, *z;       /* cell units */
    double *ux, *uy, *uz;    /* gamma*beta */
    double *w;               /* weight: real particles per macro particle, units n_c (c/w0)^3 */
    double *zq;              /* per-particle charge state (ions) or NULL: q_p = q * zq[p] when set */
    uint64_t *id;            /* particle ids (keys of the random streams) */
    double *eb;              /* optional output of the push: E^n, B^n at x^n, 6 per particle */
    int pusher;              /* ORC_PUSH_BORIS, ORC_PUSH_VAY or ORC_PUSH_HC */
} orc_species;

enum { ORC_PUSH_BORIS = 0, ORC_PUSH_VAY = 1, ORC_PUSH_HC = 2 };

void orc_gather(const orc_grid *g, const double *E[3], const double *B[3],
                double xi, double yi, double zi, double e[3], double b[3]);
void orc_boris(double qm_dt_half, const double e[3], const double b[3], double u[3]);
void orc_vay(double qm_dt_half, const double e[3], const double b[3], double u[3]);
void orc_higuera_cary(double qm_dt_half, const double e[3], const double b[3], double u[3]);
void orc_esirkepov(const orc_grid *g, double qw, double x0, double y0, double z0,
                   double x1, double y1, double z1, double *J[3]);
double orc_tsc(double d);
void orc_esirkepov2(const orc_grid *g, double qw, double x0, double y0, double z0,
                    double x1, double y1, double z1, double *J[3]);
void orc_push_deposit(const orc_grid *g, const double *E[3], const double *B[3],
                      double *J[3], orc_species *s);
void orc_gather_species(const orc_grid *g, const double *E[3], const double *B[3], orc_species *s);

/* ---- ionization ----------------------------------------------------------- */
double orc_adk_rate(double F, double Ip, double Z, int l, int m);
double orc_keldysh(double F, double Ip, double w0);
double orc_mpi_rate(double F, double Ip, double Z, int l, double w0);
double orc_blend_weight(double gamma);
double orc_ionization_rate(double F, double Ip, double Z, int l, double w0);
long orc_ionize(orc_species *ions, const double *eb, int zmax, const double *Ip_au, const int *lq,
                double w0_au, double Eref_over_Ea, double dt_au, uint32_t seed, uint32_t sp_index, long step,
                orc_species *out, long cap, double *energy_au);

/* ---- Airy functions (z >= 0) and LCFA QED rates ---------------------------- */
double orc_bessel_k(double nu, double x);
double orc_bessel_k_int(double nu, double x);
double orc_airy_ai(double z);
double orc_airy_aip(double z);
double orc_airy_int(double z);
double orc_qed_em_density(double chi, double xi);
double orc_qed_pair_density(double chi, double xi);
double orc_qed_h(double chi);
double orc_qed_power(double chi);
double orc_qed_T(double chi);
double orc_qed_em_sample(double chi, double r);
double orc_qed_pair_sample(double chi, double r);
double orc_chi(double kappa, const double e[3], const double b[3], const double u[3], int photon);
uint64_t orc_splitmix64(uint64_t x);
uint64_t orc_derived_id(uint64_t id, long step, unsigned tag);
double orc_qed_tau0(uint64_t id, uint32_t seed, uint32_t sp_index);
long orc_qed_emit(orc_species *s, double *tau, double kappa, double dt, double eps_min, uint32_t seed,
                  uint32_t sp_index, long step, orc_species *ph, double *ph_tau, long cap, double *tallies);
void orc_photon_move(const orc_grid *g, orc_species *s);
long orc_qed_pairs(orc_species *s, double *tau, unsigned char *alive, double kappa, double dt, uint32_t seed,
                   uint32_t sp_index, long step, orc_species *el, double *el_tau, orc_species *po, double *po_tau,
                   long cap, double *tallies);

/* ---- cold relativistic fluid ----------------------------------------------- */
void orc_node_fields(const orc_grid *g, const double *E[3], const double *B[3], int i, int j, int k,
                     double e[3], double b[3]);
long orc_fluid_step(const orc_grid *g, const double *E[3], const double *B[3], double *J[3], double q, double m,
                    double *n, double *u[3], double n_floor, double K, double gam);
double orc_fluid_energy(const orc_grid *g, double m, const double *n, const double *u[3]);

/* ---- regime criterion and conversions ---------------------------------------- */
void orc_regime_criterion(const orc_grid *g, const double *E[3], const double *B[3], const double *ne,
                          const double *fu[3], double kappa, double a_thr, double n_thr, double c_thr,
                          double chi_thr, int dilate, unsigned char *mask);
long orc_fluid_to_particles(const orc_grid *g, const unsigned char *mask, double q, double *n, double *u[3],
                            double n_floor, int ppc, uint32_t seed, uint32_t sp_index, uint32_t epoch,
                            orc_species *out, long cap, double *rho_bg, int quiet);
long orc_particles_to_fluid(const orc_grid *g, const unsigned char *mask, orc_species *s, double *n,
                            double *u[3], double n_floor, unsigned char *alive);

/* ---- classifier dropout masks ----------------------------------------------- */
void orc_dropout_mask(unsigned char *keep, int B, int C, long V, uint32_t seed, uint32_t pass, uint32_t layer,
                      double p);
void orc_dropout_mask_cells(unsigned char *keep, int B, int C, long V, const long *cells, uint32_t seed,
                            uint32_t pass, uint32_t layer, double p);

/* ---- diagnostics --------------------------------------------------------- */
void orc_energy_fields(const orc_grid *g, const double *E[3], const double *B[3], double out[2]);
double orc_energy_particles(const orc_species *s);
void orc_charge_density(const orc_grid *g, const orc_species *s, double *rho);
void orc_div_e(const orc_grid *g, const double *E[3], double *div);
void orc_plasma_scales(double n_m3, double out[5]);
void orc_laser_scales(double lambda_m, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
