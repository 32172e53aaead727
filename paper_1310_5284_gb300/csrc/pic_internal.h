// pic_internal.h -- data layout shared by the host runtime and the kernels of
// libpic.so.  Nothing here is part of the public ABI (include/pic.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include <string>

#include "pic.h"

namespace pic {

// Launch shape of the particle kernels (build-time knobs; the defaults are
// the ones the autotuning sweep picked on GB300).
#ifndef PIC_THREADS
#define PIC_THREADS 256
#endif
#ifndef PIC_UNROLL
#define PIC_UNROLL 4
#endif
#ifndef PIC_MIN_BLOCKS
#define PIC_MIN_BLOCKS 4
#endif

constexpr int kMaxCells = 1024;          // grid lives in shared memory
constexpr int kThreads = PIC_THREADS;    // block size of the particle kernels
constexpr int kUnroll = PIC_UNROLL;      // particles per thread per tile
constexpr int kMinBlocks = PIC_MIN_BLOCKS;
constexpr int kMaxEedfBins = 4096;

enum Mode : int {
    kExplicitEC = 0,   // gather/push/absorb/collide/deposit S_2, field solve
    kExplicitMC = 1,   // same with the momentum-conserving S_1 weighting
    kDepositEC = 2,    // deposit only (initial field, injected state)
    kDepositMC = 3,
    kImplicit1 = 4,    // direct implicit pass 1: predictor, deposit rho~ and chi
    kImplicit2 = 5,    // direct implicit pass 2: corrector, absorb, collide
    kImplicit1MC = 6,  // the same two passes with S_1 weighting and node fields
    kImplicit2MC = 7,
    kExplicitEC3 = 8,  // explicit EC with m = 3: S_3 assignment, S_2 interpolation
    kDepositEC3 = 9,
    kExplicitNU = 10,  // explicit EC on a non-uniform grid (cell widths h_c)
    kImplicit1NU = 11, // direct implicit pass 1 on a non-uniform grid
    kImplicit2NU = 12, // direct implicit pass 2 on a non-uniform grid
    kExplicitEC3NU = 13, // explicit EC with m = 3 on a non-uniform grid
};

// The cell word of a particle.  A hole left by an absorbed particle is -1.
// A live particle holds its cell in bits 0..10 and, in runs with collisions,
// the steps left to its next null-collision selection in bits 11..29 (at most
// kWaitCap), with bit 30 set when that count ends in a fresh draw of the wait
// instead of a selection.  Runs without collisions hold the plain cell.
constexpr int kCellBits = 11;
constexpr uint32_t kCellMask = (1u << kCellBits) - 1u;
constexpr uint32_t kWaitCap = 262144u;          // 64^3 steps: the longest wait one draw gives
constexpr uint32_t kRedrawBit = 0x40000000u;    // in a drawn wait and in the cell word alike
constexpr uint32_t kWaitOne = 1u << kCellBits;  // one step of the count in the cell word

// One species' particle arrays (structure of arrays).
struct Species {
    int32_t *cell;
    float *off;
    float *vx, *vy, *vz;
    uint32_t *id;
    float *abar;
};

// An ionisation event recorded by the push, placed by the step's tail.
struct Birth {
    uint32_t pid;
    int32_t cell;
    float off;
    float abar_e;
    float ve[3];
    float vi[3];
};

// Mutable per-run state, resident in the arena.
struct DevState {
    long long step;
    long long n_slots[2];          // slots in use (live + holes left by absorption)
    long long n_live[2];
    unsigned int next_id[2];
    unsigned int parity;           // which of the two particle buffers is current
    unsigned int status;           // sticky PIC_STATUS_* bits
    unsigned int blocks_done;      // last-block detection of the particle kernels
    unsigned int n_births;         // births recorded in the current step
    unsigned int sort_blocks_done;
    unsigned int next_item;        // work-item claim counter of the running particle launch
    unsigned long long absorbed_step[2];
    double ke_x_acc[2], power_acc[2];
    double ke_x[2], power[2];
    double field_energy, field_energy_push;
    double v_left;                 // electrode voltage of the current field
    double v_sum;                  // running sum of v_left over the averaged steps
    double ke_perp[2];
    unsigned long long wall_count[2][2];
    double wall_energy[2][2];
    unsigned long long coll[5];
    unsigned long long overflow[2];
    unsigned long long births_total;
    long long n_avg, n_diag;
    // Work a particle launch's tail leaves to the next launch (or to the
    // finalize kernel before the host reads diagnostics): bit 0 accumulate
    // the running averages of the newest field and charges, bit 1 convert the
    // newest field to FP64 and sum its energy.
    unsigned int pending;
    unsigned int check;            // pic_set_particles: nonzero if an uploaded particle is off the grid
    double fe_acc;                 // sum of E_c^2 of the field the next push uses
    // Electrode voltage of the field the running particle launch's tail
    // solves (one block stores it at launch start; the tail reads it), with
    // its double-word split.
    double volt_v;
    float volt_hi, volt_lo;
};

// State of a batched launch sequence (one per batch, in its arena).
struct BatchState {
    unsigned int next_item;    // work-item claim counter of the running launch
    unsigned int blocks_done;  // arrival counter of the running launch
    unsigned int status;
    unsigned int pad;
    long long launches;
};

// Constants and pointers of one run, passed to kernels by value.
struct Run {
    int n_cells, periodic, scheme, mcc, ions_mobile, diag_period, eedf_bins, sort_period;
    uint32_t seed, run;
    uint32_t rk0[10], rk1[10];   // Philox round keys of (seed, run)
    long long capacity[2];
    long long births_cap;
    // geometry / field (FP64, host-derived)
    double dx, inv_dx, dt, rf_freq, rf_volt, weight;
    double kappa;        // E jump per 2^-33 macro charge: e w 2^-33 / eps0
    double kappa_bg;     // E jump per interior node from the frozen ion density
    double chi_coef[2];  // dt^2/2 q^2 w / (m eps0 dx) * 2^-16
    double dens_scale;   // density per 2^-33 macro charge: w 2^-33 / dx
    double half_m_w[2];  // kinetic energy per (m/s)^2 per macro-particle
    double eps0_dx_half; // field energy factor eps0 dx / 2
    // the same constants as double-word FP32 pairs (hi, lo) for the tail
    float kappa_ff[2], kbg_ff[2], inv_n_ff[2], inv_ndx_ff[2];
    // push (FP32)
    float qm_dt[2];        // (q/m) dt
    float qm[2];
    float mq[2];           // m/q
    float dt_dx;           // dt / dx
    float half_dt;         // dt / 2
    float half_dt2_dx;     // dt^2 / (2 dx)
    float half_dt2;        // dt^2 / 2 (the corrector's move on a non-uniform grid)
    float qw[2];           // q w: power per particle per (V/m * m/s)
    float half_m_over_e[2];// 0.5 m / e: energy [eV] per (m/s)^2
    // collisions (FP32)
    uint32_t thr[2];       // nonzero: the species collides (P_null > 0)
    double p_null[2];      // null-collision probability per step (host-derived)
    // waiting-time thresholds [species][digit c, b, a][j - 1] of the geometric
    // law of the steps between selections (draw_wait), in the arena
    const uint32_t *wait_tab;
    float nu_max_e, nu_max_i, n_g;
    float sig_el, exc_thr, exc_ramp_end, exc_slope, sig_exc_max, iz_thr, sig_iz_k, sig_cx;
    float eps_cap, g_max_i, two_m_over_M, two_e_over_me, vth_gas;
    float abar_ion_over_e; // (q_i/m_i) / (q_e/m_e)
    int iz_opal, scatter_vs; // collision-model options (PIC_IZ_OPAL, PIC_SCATTER_VS)
    float iz_b;            // Opal-Pollock-Wagner width B [eV]
    float eedf_inv_width;
    // pointers into the arena
    Species buf[2][2];     // [parity][species]
    unsigned long long *acc_cnt[2], *acc_a[2], *acc_b[2];   // [species][n_cells + 1]
    unsigned long long *acc_c[2];                           // [species][n_cells + 1] sum F^3 (m = 3)
    unsigned int *cursor[2];                                // [species][n_cells + 1]
    float *e_gather;       // [n_cells + 2]
    double *e_cc, *chi;                                     // [n_cells], [n_cells]
    float *e_hi, *e_lo;    // [n_cells] newest field as a double-word pair (deferred conversion)
    long long *rho_q[2];   // [species][n_cells + 1] last assembled node charge, 2^-33 units (2^-36/6 for m = 3)
    double *avg_ne, *avg_ni, *avg_e, *heat[2];   // sums over steps (charge units, V/m)
    unsigned long long *eedf;
    Birth *births;
    DevState *st;
    // non-uniform grid (stretched != 0; the pointers are in the arena)
    int stretched;
    float dt_f;            // dt (FP32)
    float len_f;           // L (FP32)
    double eps0_half;      // eps0 / 2 (field energy sum_c h_c E_c^2)
    float inv_len_ff[2];   // 1 / L as a double-word pair
    const float2 *hw;      // [n_cells] (h_c, 1/h_c) in FP32 for the push
    const double *h64;     // [n_cells] h_c
    const double *xnode;   // [n_cells + 1] node positions, x_0 = 0
    const float2 *hdw;     // [n_cells] h_c as a double-word pair
    const float2 *wdw;     // [n_cells] periodic box: share of the net charge on nodes 0..c (double-word)
};

// Byte offsets of one run's buffers inside its arena.
struct Layout {
    size_t state;
    size_t sp[2][2][7];  // [parity][species][field] offsets (cell, off, vx, vy, vz, id, abar)
    size_t acc_cnt[2], acc_a[2], acc_b[2], acc_c[2], cursor[2], rho_q[2];
    size_t e_gather, e_cc, chi, avg_ne, avg_ni, avg_e, heat[2], eedf, births, e_hi, e_lo, wait_tab;
    size_t hw, h64, xnode, hdw, wdw;  // non-uniform grid tables (0 bytes on the uniform grid)
    size_t total;
};

// Arguments of the adjoint kernels (collisionless EC explicit step).
struct AdjSlot {
    int32_t *cell;
    float *off;
    float *vx;
};

struct AdjFwd {
    AdjSlot in, out;       // time levels n and n+1 (distinct arrays)
    const float *e_in;     // gather table of level n [n_cells + 2]
    float *e_out;          // gather table of level n+1, written by the tail
    double *obj;           // [2]: P^n, G^n
    long long np;
    long long level;       // time level of e_out
};

struct AdjRev {
    AdjSlot lo, hi;        // time levels n and n+1
    const float *e;        // gather table of level n
    const float *lam_in;   // Lambda of level n+1 (nullptr: level n+1 is the last)
    float *lam_out;        // Lambda of level n, written by the tail
    float *lx, *lv;        // adjoints of x (level n+1 -> n) and v (v^{n+1/2} -> v^{n-1/2})
    double *le;            // [n_cells + 2] scattered sensitivities (zero between launches)
    double *dv0;           // accumulated dJ/dV0
    long long np;
    long long level;       // n
    int a_part;            // 0: only finish level n+1 (the last launch, n+1 = 0)
    float c_pw;            // c_power / K
    float c_fl;            // c_flux / K
    float w_dx;            // w / dx
    double lam_scale;      // e w / eps0
};

// ---- shared host helpers (pic_capi.cu) ----
inline bool implicit_scheme(const pic_config &c) {
    return c.scheme == PIC_EC_IMPLICIT || c.scheme == PIC_MC_IMPLICIT;
}
Layout make_run_layout(const pic_config &c);
int validate_run_config(const pic_config *c);  // PIC_* code; message via pic_last_error
void derive_run(const pic_config &c, const Layout &L, unsigned char *arena, Run &R);
Mode push_mode_of(const pic_config &c);
Mode deposit_mode_of(const pic_config &c);
// diagnostics and particle read-back of one run (synchronise stream s)
int run_diag(const Run &R, const pic_config &c, const Layout &L, unsigned char *arena, cudaStream_t s,
             pic_diag_t *out, int reset_avg, std::string *err);
int run_get_particles(const Run &R, cudaStream_t s, int species, pic_host_particles *out, std::string *err);
// time-averaged profiles of one run (as pic_profiles)
int run_profiles(const Run &R, const pic_config &c, cudaStream_t s, double *ne, double *ni, double *phi,
                 double *heat_e, double *heat_i, uint64_t *eedf, std::string *err);
// zero a run's arena, load its particles, assign charge, solve, sort
int init_run_state(const pic_config &c, const Run &R, unsigned char *arena, size_t arena_bytes, int grid,
                   cudaStream_t s, std::string *err);

// ---- launchers (pic_kernels.cu) ----
int block_smem_bytes(const Run &r);
cudaError_t launch_load(const Run &r, int species, long long n, float vth, cudaStream_t s);
cudaError_t launch_particles(const Run &r, Mode m, int grid, cudaStream_t s);
cudaError_t launch_sort(const Run &r, int grid, cudaStream_t s);
cudaError_t sort_grid(int *grid);
cudaError_t launch_set_abar(const Run &r, cudaStream_t s);
// flag |= 1 if any of the n particles has a cell outside [0, n_cells) or an
// offset outside [0, 1)
cudaError_t launch_check_particles(const int32_t *cell, const float *off, long long n, int n_cells,
                                   unsigned int *flag, cudaStream_t s);
cudaError_t launch_perp_energy(const Run &r, cudaStream_t s);
// (with collisions, each particle draws its first wait at the run's step)
cudaError_t launch_apply_particles(const Run &r, const Species &dst, const Species &src, long long n,
                                   bool abar_given, const unsigned int *flag, int S, unsigned int next_id,
                                   cudaStream_t s);
cudaError_t launch_finalize(const Run &r, cudaStream_t s);
cudaError_t launch_philox_fill(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                               uint32_t c3, long long n, uint32_t *out, cudaStream_t s);
cudaError_t occupancy_grid(const Run &r, Mode m, int *grid);
// batched runs
size_t batch_smem_bytes(int max_cells, int max_bins, int nruns, int *table_off);
cudaError_t batch_prepare(int smem, int *grid);
cudaError_t launch_batch(int phase, const Run *runs, int nruns, long long *work, BatchState *bs,
                         long long chunk, int grid, int smem, int table_off, cudaStream_t s);
// adjoint of the collisionless EC explicit step
int adj_fwd_smem_bytes(int n_cells);
int adj_rev_smem_bytes(int n_cells);
cudaError_t adj_prepare(int n_cells, int *grid);
cudaError_t launch_adj_fwd(const Run &r, const AdjFwd &a, bool push, int grid, cudaStream_t s);
cudaError_t launch_adj_rev(const Run &r, const AdjRev &a, int grid, cudaStream_t s);
// message returned by pic_last_error(NULL) (pic_capi.cu)
void set_last_error(const char *msg);

}  // namespace pic
