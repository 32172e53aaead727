/*
 * oracle.h -- plain FP64 CPU oracle for the 1D electrostatic PIC/MCC method of
 * Wang, Sun, Jiang & Kong, "On the energy conservation electrostatic PIC/MC
 * simulating: benchmark and application to the radio frequency discharges"
 * (Chinese Physics B).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the CUDA path: its own
 * constants, its own Philox, its own deposit, field solve and push.
 *
 * Units are SI throughout.  Positions are kept in cell units (xi = x / dx) so
 * that a position given as (integer cell, FP32 offset) is held exactly.
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_EC3_EXPLICIT: the explicit EC scheme with m = 3 in Eq. (2)-(3) (cubic
   S_3 charge assignment, S_2 force interpolation from the cell centres), the
   "larger m" Sec. 2 allows. */
enum { ORC_EC_EXPLICIT = 0, ORC_MC_EXPLICIT = 1, ORC_EC_IMPLICIT = 2, ORC_MC_IMPLICIT = 3, ORC_EC3_EXPLICIT = 4 };

typedef struct orc_params {
    /* grid and geometry (Sec. 3: planar gap between two electrodes) */
    int32_t n_cells;
    int32_t periodic;        /* 0: electrodes (x=0 driven, x=L grounded); 1: periodic box */
    int32_t scheme;          /* ORC_EC_EXPLICIT / ORC_MC_EXPLICIT / ORC_EC_IMPLICIT / ORC_MC_IMPLICIT (Sec. 2), ORC_EC3_EXPLICIT */
    int32_t mcc;             /* 1: null-collision Monte Carlo on */
    int32_t ions_mobile;     /* 0: ions replaced by a frozen uniform background */
    int32_t quantized;       /* 1: offset quantisation (16 bits; 12 for m = 3), int64 sums; 0: exact FP64 weights */
    int32_t diag_period;     /* heating profile and EEDF sampled every diag_period steps (0: never) */
    int32_t eedf_bins;
    uint32_t seed, run;      /* Philox key */
    double length;           /* gap [m] */
    double dt;               /* time step [s] */
    double rf_freq, rf_volt; /* V(t) = rf_volt sin(2 pi rf_freq t) on the x=0 electrode */
    double n0;               /* density that np_init macro-particles represent [m^-3] */
    double np_init;          /* macro-particles per species at load (sets the macro weight) */
    double bg_density;       /* frozen ion density [m^-3] when ions_mobile == 0 */
    double te_ev, ti_ev;     /* load temperatures [eV] */
    double ion_mass_amu;
    double gas_density;      /* [m^-3] */
    double gas_temp;         /* [K] */
    double sig_el;           /* e- elastic, constant [m^2] */
    double exc_thr, exc_ramp_end, sig_exc_max;  /* excitation: 0 below thr, linear to max at ramp_end */
    double iz_thr, sig_iz_peak;                 /* ionisation: peak value at e*thr */
    double sig_cx;           /* ion charge exchange, constant [m^2] */
    double eps_cap;          /* eV: energy up to which the e- collision frequency bound holds */
    double cx_vmax;          /* V: ion energy up to which the CX bound holds */
    double eedf_max_ev;
    /* collision model options (bits): ORC_IZ_OPAL shares the ionisation
       excess by the Opal-Pollock-Wagner law of width iz_split_b [eV] (else
       equally); ORC_SCATTER_VS scatters electrons by the Vahedi-Surendra
       anisotropic law (else isotropically) */
    int32_t coll_model;
    int32_t reserved;
    double iz_split_b;
    /* Non-uniform grid, the multi-scale grid Sec. 4 proposes: the widths [m]
       of the n_cells cells, summing to `length`; NULL for the uniform grid of
       width length / n_cells.  Positions stay in cell units (cell index plus
       the fraction of that cell's width); the EC schemes (explicit with m = 2
       or 3, direct implicit) with mobile ions are the ones defined on it
       (orc_sim_create refuses the momentum-conserving ones). */
    const double *cell_width;
} orc_params;
enum { ORC_IZ_OPAL = 1, ORC_SCATTER_VS = 2 };

/* Philox4x32-10: key (2 words), counter (4 words) -> 4 words. */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]);
/* n consecutive blocks with counter (c0 + k, c1, c2, c3); out has 4n words. */
void orc_philox_stream(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t c3, int64_t n, uint32_t *out);

/* Derived constants (computed from params alone). */
typedef struct orc_derived {
    double dx, weight, q[2], m[2], vth[2], vth_gas;
    double nu_max_e, nu_max_i, p_null_e, p_null_i;
    uint32_t thr_e, thr_i;   /* P_null on the 24-bit scale (nonzero: the species collides) */
    double g_max_i;
    uint32_t wait_thr[2][3][64]; /* [species][digit c, b, a][j - 1]: waiting-time thresholds */
} orc_derived;
void orc_derive(const orc_params *p, orc_derived *d);
/* Steps to the next null-collision selection of particle `id` of a species,
   drawn at `step` (sub 0: after a selection, 1: on entering the run), with
   bit 30 set when the count ends in a fresh draw rather than a selection. */
uint32_t orc_wait_draw(const orc_params *p, const orc_derived *d, int species, uint32_t id,
                       int64_t step, uint32_t sub);
void orc_wait_draws(const orc_params *p, int species, int64_t n, const uint32_t *id, int64_t step,
                    uint32_t sub, uint32_t *out);

/* ---- stand-alone pieces used by the pin tests ---- */
/* S_2 charge assignment of n particles to nodes, in units of 2^-33 particle
   charge (quantized) or in particle units (fp64 array).  Walls fold the ghost
   node onto the wall node; periodic wraps.  out has n_cells+1 entries. */
void orc_deposit_s2_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out);
void orc_deposit_s2_fp64(const orc_params *p, int64_t n, const double *xi, double *out);
/* S_1 charge assignment to nodes (momentum-conserving scheme), units 2^-33. */
void orc_deposit_s1_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out);
/* S_3 (cubic B-spline) charge assignment, m = 3: four nodes per particle.
   Fixed point: 12-bit offset code F, units of 2^-36/6 particle charge (each
   particle assigns exactly 6 * 2^36).  Ghost nodes fold / wrap as for S_2. */
void orc_deposit_s3_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out);
void orc_deposit_s3_fp64(const orc_params *p, int64_t n, const double *xi, double *out);
/* Integer node charge of one particle charge in the units of the scheme's
   fixed-point assignment: 2^33, or 6 * 2^36 for m = 3. */
int64_t orc_charge_unit(const orc_params *p);
/* Dirichlet tridiagonal solve of -(phi[g-1]-2phi[g]+phi[g+1])/dx^2 = rho[g]/eps0
   with phi[0]=v_left, phi[N]=0, coefficient (1+chi) on each cell face when chi
   is given (NULL: plain Poisson). Thomas algorithm. */
void orc_solve_dirichlet(int n_cells, double dx, const double *rho, const double *chi,
                         double v_left, double *phi);
/* Periodic solve (mean charge removed, gauge phi[0]=0). */
void orc_solve_periodic(int n_cells, double dx, const double *rho, const double *chi,
                        double *phi);
/* Fields from the node potential: cell-centred E[c] = (phi[c]-phi[c+1])/dx and
   the node field of the momentum-conserving scheme (centred, one-sided at walls). */
void orc_fields(const orc_params *p, const double *phi, double *e_cc, double *e_node);
/* EC force interpolation: E at particle from cell-centred E (ghost cells E=0). */
double orc_gather_ec(const orc_params *p, const double *e_cc, double xi);
double orc_gather_mc(const orc_params *p, const double *e_node, double xi);
/* m = 3: S_2 from the three nearest cell centres (ghost cells E = 0). */
double orc_gather_ec3(const orc_params *p, const double *e_cc, double xi);

/* ---- non-uniform grid (cell widths h[0..N-1], nodes x[0..N]) ----
   The EC scheme there keeps Eq. (2)-(3) in the cell coordinate xi: the S_2
   assignment of xi to the nodes and the S_1 interpolation between cell
   centres are those of the uniform grid.  The particle's potential energy
   q sum_g phi_g S_2(xi(x) - g) then has the x-derivative
   -(q / h_c) sum_c (phi_c - phi_{c+1}) S_1(xi - c - 1/2) inside cell c, which
   is the force; the Poisson equation is the Gauss law on the physical node
   spacing.  Node positions: x[0] = 0, x[g+1] = x[g] + h[g]. */
void orc_grid_nodes(int n_cells, const double *h, double *x);
/* The cell holding the physical position x (x[c] <= x < x[c+1]) and the
   fraction off = (x - x[c]) / h[c] in [0, 1); returns 0 inside, -1 below x[0],
   1 at or beyond x[N]. */
int orc_locate(int n_cells, const double *x_nodes, const double *h, double x, int64_t *cell,
               double *off);
/* Gauss law eps0 [(1+chi_g)(phi_g - phi_{g+1})/h_g - (1+chi_{g-1})(phi_{g-1} -
   phi_g)/h_{g-1}] = q_g for the interior nodes, node charges q_g per unit
   area [C/m^2], the implicit susceptibility chi of each cell (NULL: none),
   phi[0] = v_left, phi[N] = 0 (Thomas algorithm). */
void orc_solve_dirichlet_h(int n_cells, const double *h, const double *q_node, const double *chi,
                           double v_left, double *phi);
/* Periodic: the net charge is spread over the nodes in proportion to their
   lengths (h_{g-1} + h_g) / 2, gauge phi[0] = phi[N] = 0. */
void orc_solve_periodic_h(int n_cells, const double *h, const double *q_node, const double *chi,
                          double *phi);
/* Field at the particle [V/m] from the voltage drops u[c] = phi_c - phi_{c+1}
   of the cells (ghost cells 0 beyond the walls, wrapped in a periodic box). */
double orc_gather_ec_h(const orc_params *p, const double *u_cc, double xi);
/* The same for m = 3: S_2 interpolation of the voltage drops from the three
   nearest cell centres over the particle's own cell width. */
double orc_gather_ec3_h(const orc_params *p, const double *u_cc, double xi);

/* Isotropic scattering rotation used by the collision routines (exposed for tests). */
void orc_rotate(const double d[3], double cos_chi, double phi, double out[3]);
/* Vahedi & Surendra (1995) anisotropic electron scattering: cos chi for an
   electron of energy eps [eV] from a uniform u in (0, 1). */
double orc_vs_cos_chi(double eps, double u);
/* Opal, Pollock & Wagner (1971): energy [eV] the secondary electron of an
   ionisation takes out of the excess eps - I, from a uniform u in (0, 1). */
double orc_opal_secondary(double excess, double b, double u);

/* ---- whole simulation ---- */
typedef struct orc_diag {
    int64_t count[2];
    int64_t wall_count[2][2];        /* [species][wall 0 = x=0, 1 = x=L] */
    double  wall_energy_ev[2][2];
    int64_t coll[5];                 /* elastic, excitation, ionisation, charge exchange, null-selected */
    int64_t overflow[2];             /* collision-bound overflows per species */
    int64_t births;
    double  ke_x[2];                 /* time-centred x kinetic energy [J/m^2] of the last step */
    double  ke_perp[2];              /* current (vy^2+vz^2) kinetic energy [J/m^2] */
    double  field_energy;            /* 1/2 eps0 sum E^2 dx at the current field [J/m^2] */
    double  field_energy_push;       /* the same for the field the last step's push used */
    double  power[2];                /* sum q w E v over the last step [W/m^2] */
    int64_t step;
    int64_t n_avg;                   /* steps accumulated in the time averages */
    int64_t n_diag;                  /* diagnostic samples in heating / EEDF */
} orc_diag;

typedef struct orc_sim orc_sim;

orc_sim *orc_sim_create(const orc_params *p, int64_t cap_e, int64_t cap_i);
void     orc_sim_free(orc_sim *s);
/* uniform load of n_e electrons and n_i ions (ids 0..n-1) followed by the t=0 field */
int      orc_sim_load(orc_sim *s, int64_t n_e, int64_t n_i);
/* inject a state: positions in cell units, velocities in m/s, ids; abar may be NULL.
   next_id: first id given to a particle born later.  wait: the steps to each
   particle's next null-collision selection (as orc_sim_get returns them), or
   NULL to draw them as for particles entering the run at the current step. */
int      orc_sim_set(orc_sim *s, int species, int64_t n, const double *xi, const double *vx,
                     const double *vy, const double *vz, const uint32_t *id, const double *abar,
                     uint32_t next_id, const uint32_t *wait);
/* deposit + field solve for the current state (and abar = a^0 for the implicit scheme) */
void     orc_sim_init_field(orc_sim *s, int set_abar);
int64_t  orc_sim_count(const orc_sim *s, int species);
void     orc_sim_get(const orc_sim *s, int species, double *xi, double *vx, double *vy,
                     double *vz, uint32_t *id, double *abar, uint32_t *wait);
int      orc_sim_step(orc_sim *s, int64_t nsteps);
void     orc_sim_set_step(orc_sim *s, int64_t step);
void     orc_sim_diag(const orc_sim *s, orc_diag *d);
/* grids: rho_q[species][N+1] int64 (units of orc_charge_unit), phi[N+1], e_cc[N], chi[N] */
void     orc_sim_grids(const orc_sim *s, int64_t *rho_q_e, int64_t *rho_q_i, double *phi,
                       double *e_cc, double *chi);
/* time averages: n_e, n_i, phi at nodes [N+1]; heating per cell and species [2][N]; eedf [bins+1] */
void     orc_sim_averages(const orc_sim *s, double *ne, double *ni, double *phi,
                          double *heat_e, double *heat_i, int64_t *eedf);
void     orc_sim_reset_averages(orc_sim *s);

/* ---- collisionless EC explicit run and its discrete adjoint (adjoint.c) ---- */
/* Electrons (charge -e, mass m_e, weight particles/m^2 each) on a frozen
   uniform ion background; no collisions; K = nsteps leapfrog steps of the EC
   scheme from time level step0.  Objective J = c_power <P> + c_flux <Gamma>,
   time averages over the K steps of P^n = sum q w E_p vbar_p and
   Gamma^n = sum w vbar_p S_1(xi_p - 1/2)/dx, vbar = (v^{n-1/2} + v^{n+1/2})/2. */
typedef struct orc_adj_problem {
    int32_t n_cells;
    int32_t periodic;        /* 0: electrodes (x=0 driven, x=L grounded, absorbing); 1: periodic */
    int64_t nsteps;
    int64_t step0;           /* time level of the initial state (RF phase) */
    double length, dt, rf_freq, rf_volt;
    double weight;           /* electrons per m^2 represented by one macro-particle */
    double bg_density;       /* frozen ion density [m^-3] */
    double c_power, c_flux;
} orc_adj_problem;

/* Forward run: time-averaged P and Gamma; final state (may be NULL);
   absorbed_at[p] = step in which particle p was absorbed, -1 if never (may be NULL). */
int orc_adj_forward(const orc_adj_problem *pb, int64_t np, const double *xi0, const double *vx0,
                    double *power_avg, double *flux_avg, double *xi_end, double *vx_end,
                    int64_t *absorbed_at);
/* J and its gradient with respect to the initial velocities v^{-1/2} [n],
   the initial positions in cell units [n] (may be NULL) and rf_volt. */
int orc_adj_gradient(const orc_adj_problem *pb, int64_t np, const double *xi0, const double *vx0,
                     double *j_out, double *dj_dvx0, double *dj_dxi0, double *dj_dv0);

#ifdef __cplusplus
}
#endif
#endif
