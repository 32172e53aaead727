/*
 * pic.h -- C ABI of the GB300 energy-conserving PIC/MCC library (libpic.so).
 *
 * The library advances the 1D electrostatic particle-in-cell / Monte Carlo
 * collision model of Wang, Sun, Jiang & Kong ("On the energy conservation
 * electrostatic PIC/MC simulating: benchmark and application to the radio
 * frequency discharges"): a planar gap between an RF-driven and a grounded
 * electrode filled with electrons and ions (Sec. 3), charge assignment by the
 * quadratic spline S_2 (Eq. 2), force interpolation by S_1 from cell-centred
 * fields (Eq. 3), explicit leapfrog or direct-implicit push (Sec. 2, schemes
 * (1)-(4)), absorbing electrodes and null-collision Monte Carlo with
 * ionisation (Sec. 3).
 *
 * Conventions for every entry point:
 *  - Return value: PIC_OK (0) on success, a negative PIC_E* code otherwise;
 *    pic_last_error() then holds a one-line message.  Nothing is partially
 *    applied when validation fails.
 *  - Device memory is owned by the caller: pic_required_sizes() states how
 *    many bytes the library needs; the caller allocates one device buffer
 *    (the "arena", 256-byte aligned, e.g. a torch uint8 tensor) and passes it
 *    to pic_init().  The handle keeps the pointer and never frees it; the
 *    arena must outlive the handle.  The library allocates no device memory.
 *  - Work is enqueued on the CUDA stream given to pic_init() (a cudaStream_t
 *    passed as void*, NULL = legacy default stream).  pic_step() is
 *    asynchronous; calls that return data to the host synchronise that
 *    stream first.
 *  - Host buffers passed in or out are owned by the caller and only read or
 *    written during the call.
 *  - A handle is not thread-safe; separate handles on separate streams are
 *    independent.
 *  - The device keeps a sticky status word (particle or birth capacity
 *    exceeded, collision bound exceeded).  It is read by pic_status() and
 *    pic_diag().
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 3

/* Error codes. */
#define PIC_OK 0
#define PIC_EINVAL (-1)     /* invalid argument or configuration */
#define PIC_EUNSTABLE (-2)  /* strict mode: omega_p dt >= 2, Eq. (1) leapfrog limit */
#define PIC_ENOMEM (-3)     /* arena too small or misaligned */
#define PIC_EOVERFLOW (-4)  /* particle / birth capacity or fixed-point headroom exceeded */
#define PIC_ECUDA (-5)      /* a CUDA call failed; message in pic_last_error */
#define PIC_ETIMEOUT (-6)   /* a bounded device-side wait gave up */

/* Device status bits (pic_diag_t.status, pic_status). */
#define PIC_STATUS_CAPACITY 0x1u    /* particles dropped: slot capacity exhausted */
#define PIC_STATUS_BIRTHS 0x2u      /* births dropped: per-step birth buffer full */
#define PIC_STATUS_TIMEOUT 0x4u     /* a bounded device wait ran out (about a second; the launch
                                       ended its stream early: the step is incomplete) */
#define PIC_STATUS_QUEUE 0x8u       /* a selected collision found the collision queue full
                                       (drains keep room for a whole tile: not expected) */

/* Schemes (Sec. 2): (2) EC explicit, (1) momentum-conserving explicit, (4) EC
   direct implicit, (3) momentum-conserving direct implicit (S_1 charge and
   susceptibility, the susceptibility's node sums averaged onto the faces of
   the modified Poisson equation, force from the node field). */
#define PIC_EC_EXPLICIT 0
#define PIC_MC_EXPLICIT 1
#define PIC_EC_IMPLICIT 2
#define PIC_MC_IMPLICIT 3
/* The explicit EC scheme with m = 3 in Eq. (2)-(3) (Sec. 2 allows m > 2):
   cubic S_3 charge assignment to four nodes, quadratic S_2 force
   interpolation from the three nearest cell centres (zero field in the ghost
   cells beyond an electrode).  Charges are assigned in fixed point from a
   12-bit offset code, F = floor(off * 2^12), in units of 2^-36/6 particle
   charge (pic_grids() returns rho_q in these units for this scheme).  Single
   runs only (pic_batch_init and pic_deposit_noalloc reject it); capacity per
   species below 2^23 (int64 headroom of the node charges). */
#define PIC_EC3_EXPLICIT 4

/* Boundaries: electrodes at x=0 (driven, V(t) = rf_volt sin(2 pi rf_freq t))
   and x=L (grounded), both absorbing (Sec. 3); or a periodic box. */
#define PIC_BC_ELECTRODES 0
#define PIC_BC_PERIODIC 1

/* Collision-model options (bits of pic_config.collision_model; 0 is the
   equal ionisation split and isotropic scattering).  PIC_IZ_OPAL: the
   secondary electron of an ionisation takes eps_s of the excess eps - I from
   the Opal-Pollock-Wagner spectrum 1 / (1 + (eps_s / B)^2) on [0, (eps - I)/2]
   (B = iz_split_b), the primary the rest.  PIC_SCATTER_VS: electrons scatter
   by the Vahedi-Surendra anisotropic law cos chi = (2 + eps - 2 (1 + eps)^u)
   / eps (eps in eV), at the incident energy for elastic scattering and at the
   energy each electron leaves with after excitation or ionisation (the
   secondary turned from the incident direction).  Sec. 3 takes its collision
   model from its MCC reference; these are the published forms. */
#define PIC_IZ_OPAL 1
#define PIC_SCATTER_VS 2

typedef struct pic_config {
    int32_t scheme;          /* PIC_EC_EXPLICIT / PIC_MC_EXPLICIT / PIC_EC_IMPLICIT / PIC_MC_IMPLICIT /
                                PIC_EC3_EXPLICIT */
    int32_t boundary;        /* PIC_BC_ELECTRODES / PIC_BC_PERIODIC */
    int32_t n_cells;         /* 2 .. 1024 */
    int32_t mcc;             /* 1: null-collision Monte Carlo on */
    int32_t ions_mobile;     /* 0: no ion particles; frozen uniform ion density bg_density */
    int32_t strict;          /* 1: reject explicit runs with omega_p dt >= 2 (Eq. 1) */
    int32_t sort_period;     /* steps between counting sorts of the particles (0: never) */
    int32_t diag_period;     /* heating profile / EEDF sampled every diag_period steps (0: never) */
    int32_t eedf_bins;       /* EEDF bins over [0, eedf_max_ev), plus one overflow bin */
    uint32_t seed;           /* Philox key word 0 */
    uint32_t run;            /* Philox key word 1 (run index in a batch) */
    int32_t collision_model; /* PIC_IZ_OPAL | PIC_SCATTER_VS bits (0: equal split, isotropic) */
    int64_t np_init;         /* macro-particles per species placed by pic_init (uniform load) */
    int64_t capacity[2];     /* particle slots per species (electrons, ions) */
    int64_t births_capacity; /* ionisation events one step can record */
    double length;           /* gap [m] */
    double dt;               /* time step [s] */
    double rf_freq;          /* [Hz] */
    double rf_volt;          /* amplitude [V] */
    double n0;               /* density represented by np_init macro-particles [m^-3] */
    double bg_density;       /* frozen ion density [m^-3] when ions_mobile == 0 */
    double te_ev, ti_ev;     /* load temperatures [eV] */
    double ion_mass_amu;
    double pressure_mtorr;   /* neutral gas pressure */
    double gas_temp;         /* neutral gas temperature [K] */
    double sig_el;           /* e- elastic, constant [m^2] */
    double exc_thr;          /* excitation threshold [eV] */
    double exc_ramp_end;     /* energy at which excitation reaches its maximum [eV] */
    double sig_exc_max;      /* [m^2] */
    double iz_thr;           /* ionisation threshold I [eV] */
    double sig_iz_peak;      /* ionisation peak value (at e*I) [m^2] */
    double sig_cx;           /* ion charge exchange, constant [m^2] */
    double eps_cap;          /* e- energy up to which the collision bound holds [eV] */
    double cx_vmax;          /* ion energy up to which the charge-exchange bound holds [V] */
    double eedf_max_ev;
    double iz_split_b;       /* Opal-Pollock-Wagner width B [eV] (PIC_IZ_OPAL) */
    /* Non-uniform grid, the multi-scale grid Sec. 4 proposes for resolving
       the sheaths without resolving the bulk: NULL for the uniform grid of
       width length / n_cells, else a host array of n_cells cell widths [m],
       each positive, summing to `length` within 1e-9 relative.  pic_init
       copies it (the caller keeps ownership).  Taken by the EC schemes
       (PIC_EC_EXPLICIT, PIC_EC_IMPLICIT, PIC_EC3_EXPLICIT) with mobile ions,
       in single runs (pic_batch_init rejects it).  The
       paper gives no form of Eq. (2)-(3) for unequal cells; this library's:
       a particle's position stays (cell, offset in [0, 1) of that cell's
       width); the charge assignment and the interpolation weights are those
       of the uniform grid in that cell coordinate; the force is the
       x-derivative of the particle's potential energy, the interpolated
       voltage drop divided by the particle's own cell width; the field
       solve is the Gauss law on the physical node spacing, with sum_c h_c
       E_c = V(t) between electrodes, and in a periodic box zero with the
       net charge spread over the nodes in proportion to (h_{g-1} + h_g)/2.
       Energy conservation (Sec. 2) carries over.  The direct-implicit
       scheme moves the predicted and corrected positions the same way, takes
       a cell's susceptibility from its S_1-weighted count over its own
       width, and solves (1 + chi_c) E_c in the same Gauss law.  With m = 3
       the S_3 assignment and the S_2 interpolation of the voltage drops are
       those of the uniform grid in the cell coordinate, the force again over
       the particle's own cell width.  pic_profiles divides a
       node's charge by (h_{g-1} + h_g)/2, and the heating of a cell by its
       width. */
    const double *cell_width;
} pic_config;

typedef struct pic_sizes {
    size_t arena_bytes;      /* device bytes pic_init needs */
    size_t snapshot_bytes;   /* host bytes pic_save writes */
} pic_sizes;

typedef struct pic_buffers {
    void *arena;             /* device pointer, 256-byte aligned */
    size_t arena_bytes;
} pic_buffers;

/* One species' particles in the device storage form: cell index, offset in
   [0,1) within the cell (position x = (cell + off) * dx), velocity [m/s],
   id, and the implicit push's time-averaged acceleration abar [m/s^2]
   (may be NULL: zero).  Host arrays of length count. */
typedef struct pic_host_particles {
    int64_t count;
    int32_t *cell;
    float *off;
    float *vx, *vy, *vz;
    uint32_t *id;
    float *abar;
    uint32_t next_id;        /* set: first id given to particles born later; get: current */
} pic_host_particles;

typedef struct pic_diag_t {
    int64_t step;
    int64_t count[2];                 /* live particles per species */
    uint64_t wall_count[2][2];        /* [species][0: x=0 electrode, 1: x=L electrode] */
    double wall_energy_ev[2][2];      /* summed kinetic energy of absorbed particles [eV] */
    uint64_t coll[5];                 /* elastic, excitation, ionisation, charge exchange, null */
    uint64_t overflow[2];             /* selected particles above the collision bound */
    uint64_t births;
    double ke_x[2];                   /* time-centred x kinetic energy of the last step [J/m^2] */
    double ke_perp[2];                /* current (vy,vz) kinetic energy [J/m^2] */
    double field_energy;              /* 1/2 eps0 sum E^2 dx of the current field [J/m^2] */
    double field_energy_push;         /* the same for the field the last push used */
    double power[2];                  /* sum_p q w E v of the last step [W/m^2] */
    int64_t n_avg;                    /* steps in the running time averages */
    int64_t n_diag;                   /* samples in the heating profile / EEDF */
    uint32_t status;                  /* PIC_STATUS_* bits */
    uint32_t reserved;
} pic_diag_t;

typedef struct pic_handle pic_handle;

/* Library version (PIC_ABI_VERSION) and a build description string. */
int pic_version(void);
const char *pic_build_info(void);

/* Bytes of device memory (arena) and host snapshot a configuration needs.
   Validates the configuration (Eq. (1) in strict mode, capacities,
   fixed-point headroom: capacity < 2^30 per species). */
int pic_required_sizes(const pic_config *cfg, pic_sizes *out);

/* Create a run in caller-owned device memory and place np_init electrons and
   ions uniformly between the electrodes with Maxwellian velocities (Sec. 3:
   uniform initial plasma), ids 0..np_init-1, then assign charge and solve for
   the t = 0 field (and abar = a^0 for the implicit scheme).  stream: a
   cudaStream_t as void* (NULL = default stream). */
int pic_init(const pic_config *cfg, const pic_buffers *bufs, void *stream, pic_handle **out);

/* Enqueue n steps (Sec. 2: gather, push, absorb, collide, assign charge,
   solve) on the handle's stream.  Asynchronous. */
int pic_step(pic_handle *h, int64_t n);

/* Synchronise and read the diagnostics.  reset_avg != 0 clears the running
   time averages (densities, potential, heating, EEDF) after reading.
   Returns PIC_ETIMEOUT (with *out filled) once the sticky status holds
   PIC_STATUS_TIMEOUT. */
int pic_diag(pic_handle *h, pic_diag_t *out, int reset_avg);

/* Time-averaged profiles since the last reset, each may be NULL:
   ne, ni, phi [n_cells+1] at the nodes; heat_e, heat_i [n_cells] power
   density J.E [W/m^3] per cell; eedf [eedf_bins+1] counts. */
int pic_profiles(pic_handle *h, double *ne, double *ni, double *phi, double *heat_e,
                 double *heat_i, uint64_t *eedf);

/* Current grid state, each may be NULL: rho_q_e, rho_q_i [n_cells+1] charge
   assigned per node in units of 2^-33 macro-particle charges (2^-36/6 for
   PIC_EC3_EXPLICIT; int64, exact);
   phi [n_cells+1]; e_cc [n_cells] cell-centred field; chi [n_cells]
   susceptibility of the last implicit field solve. */
int pic_grids(pic_handle *h, int64_t *rho_q_e, int64_t *rho_q_i, double *phi, double *e_cc,
              double *chi);

/* Live particle counts per species (synchronises). */
int pic_count(pic_handle *h, int64_t *n_e, int64_t *n_i);

/* Copy one species' live particles to host arrays of length out->count
   (at least the live count); out->count is set to the number written. */
int pic_get_particles(pic_handle *h, int species, pic_host_particles *out);

/* Replace one species' particles by host arrays (count <= capacity).  The
   arrays are uploaded into the run's idle second particle buffer and checked
   there on the device (cell in [0, n_cells), offset in [0, 1)); if any
   particle is off the grid the call returns PIC_EINVAL and the run is
   unchanged.  Synchronous.  The field is not recomputed: call
   pic_init_field() after setting both species. */
int pic_set_particles(pic_handle *h, int species, const pic_host_particles *in);

/* Both species at once, as pic_set_particles does one: the uploads, both
   checks and then both moves into the current buffer run back to back on the
   run's stream with one synchronisation at the end; if a particle of either
   species is off the grid the call returns PIC_EINVAL and neither species
   changes.  PIC_EINVAL for a NULL argument. */
int pic_set_state(pic_handle *h, const pic_host_particles *electrons, const pic_host_particles *ions);

/* Assign charge for the current particles and solve for the field at the
   current time level; set_abar != 0 also sets abar = (q/m) E(x) for the
   implicit scheme. */
int pic_init_field(pic_handle *h, int set_abar);

/* Set the step counter (time level n: V(t_n), Philox counter). */
int pic_set_step(pic_handle *h, int64_t step);

/* Synchronise and return the device status word (PIC_STATUS_* bits). */
int pic_status(pic_handle *h, uint32_t *status);

/* Snapshot the whole run state into a host buffer of snapshot_bytes, and
   restore it.  Philox streams are keyed on (id, step), so a restored run
   continues exactly as the original would have. */
int pic_save(pic_handle *h, void *host_buf, size_t nbytes);
int pic_load(pic_handle *h, const void *host_buf, size_t nbytes);

/* Self-test of the bounded device waits.  Every wait of the particle
   launches (a staged copy landing in shared memory) gives up after about a
   second, sets PIC_STATUS_TIMEOUT and lets the launch end, so a copy that
   never lands cannot hang the GPU.  This call runs that same wait once, in a
   one-thread launch, on a barrier that nothing completes (no copy is issued)
   with the given limit, and returns PIC_ETIMEOUT with *status =
   PIC_STATUS_TIMEOUT and *waited_s the time the wait took; the context stays
   usable.  limit_ns in 0 .. 1e10; PIC_EINVAL otherwise or for a NULL output;
   PIC_ECUDA if the launch fails.  Synchronous on `stream`. */
int pic_selftest_wait(int64_t limit_ns, uint32_t *status, double *waited_s, void *stream);

/* Fill a device buffer with n Philox4x32-10 blocks: key (k0, k1), counter
   (c0 + i, c1, c2, c3) for block i; out receives 4n uint32 words. */
int pic_philox_fill(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                    uint32_t c3, int64_t n, uint32_t *out_device, void *stream);

/* ---- Batched runs ----
   Many independent discharges (different grids, particle counts, pressures,
   voltages, schemes) in one caller-owned arena, advanced together by
   persistent launches over all runs: each step is one launch for the
   explicit runs and the implicit predictor, one for the implicit corrector,
   and one counting sort every sort period, replayed from a captured CUDA
   graph.  Each run gives bit-identical particles to the same configuration
   run alone with pic_init/pic_step (charge sums are integers and draws are
   keyed on (particle id, step, run)); the paper's sweeps of grid spacing,
   time step and pressure (Sec. 3) are the use case. */
typedef struct pic_batch pic_batch;

/* Arena bytes for nruns configurations (1..1024), each validated as in
   pic_required_sizes; PIC_EINVAL for a PIC_EC3_EXPLICIT configuration. */
int pic_batch_required_sizes(const pic_config *cfgs, int32_t nruns, pic_sizes *out);
/* Create the batch in a caller-owned device arena (256-byte aligned) and load
   every run (uniform load, t = 0 field, one sort).  The batch sort period is
   the smallest positive sort_period of the configurations (16 if none). */
int pic_batch_init(const pic_config *cfgs, int32_t nruns, const pic_buffers *bufs, void *stream,
                   pic_batch **out);
/* Enqueue n steps of every run (asynchronous). */
int pic_batch_step(pic_batch *b, int64_t n);
/* Diagnostics and particles of one run (synchronising; as pic_diag and
   pic_get_particles). */
int pic_batch_diag(pic_batch *b, int32_t run, pic_diag_t *out, int reset_avg);
int pic_batch_get_particles(pic_batch *b, int32_t run, int species, pic_host_particles *out);
/* Time-averaged profiles of one run (synchronising; as pic_profiles: the
   averages since the run's last reset through pic_batch_diag(..., 1)). */
int pic_batch_profiles(pic_batch *b, int32_t run, double *ne, double *ni, double *phi, double *heat_e,
                       double *heat_i, uint64_t *eedf);
/* Work-item size (particles per item, 256..2^24) and sort period (0: never)
   of the batched launches.  Results do not depend on them. */
int pic_batch_set_schedule(pic_batch *b, int64_t chunk, int32_t sort_period);
/* Time whole sort cycles of at least trial_steps steps for each candidate
   schedule (work items of 4096..65536 particles, sort periods 4..32), keep
   the fastest and report it.  The trial steps are ordinary steps of the runs
   (every schedule gives the same particles), so the runs advance by them. */
int pic_batch_autotune(pic_batch *b, int32_t trial_steps, int64_t *chunk, int32_t *sort_period,
                       double *ms_per_step);
/* OR of the runs' device status words (synchronising). */
int pic_batch_status(pic_batch *b, uint32_t *status);
void pic_batch_free(pic_batch *b);

/* Charge assignment of one species for callers that cannot allocate device
   memory where they need a density (code inside another framework's memory
   pool, allocation-free real-time loops, tools that hold only particle
   arrays).  The paper has no counterpart: this is a library convenience
   beside the run API.
   cell, off: device arrays of n particles in the storage form (cell index,
   offset in [0,1)); entries with a cell outside [0, n_cells) or an offset
   outside [0, 1) (NaN included) assign nothing.
   rho_q_out: device array of n_cells+1 int64 receiving the node charge in
   units of 2^-33 macro-particle charges, quadratic S_2 weights (EC schemes)
   or linear S_1 (PIC_MC_EXPLICIT, PIC_MC_IMPLICIT), electrodes or periodic as `boundary` -
   the same numbers pic_grids() returns for a run holding these particles.
   The per-node sums live in a static device array of the library sized for
   n_cells <= 1024 (about 25 KB on every GPU that loads the library, held
   until the process exits); no other memory is used and nothing is
   allocated.  The first call on a device looks up that array's device
   address; make it before any stream capture on that device.  The address
   is kept for the life of the process, so cudaDeviceReset() between calls
   is not supported (the reset unloads the module that holds the array).
   All calls on one device share the array: calls that overlap on the GPU
   race (calls on one stream are ordered); each call clears it first.
   Asynchronous on `stream`.  Returns PIC_OK; PIC_EINVAL for n_cells outside
   2..1024, n outside 0..2^29-1, an unknown scheme or boundary
   (PIC_EC3_EXPLICIT included), or a NULL array; PIC_ECUDA if a CUDA call
   fails (message in pic_last_error(NULL)). */
int pic_deposit_noalloc(int32_t scheme, int32_t boundary, int32_t n_cells, const int32_t *cell,
                        const float *off, int64_t n, int64_t *rho_q_out, void *stream);

/* ---- Adjoint of the collisionless EC explicit step ----
   Reverse-mode derivative of a run of the explicit energy-conserving scheme
   (Sec. 2, scheme (2): S_2 charge assignment Eq. 2, S_1 force interpolation
   Eq. 3, leapfrog) for electrons on a frozen uniform ion background, with no
   collisions.  Between electrodes (x = 0 driven by V(t) = rf_volt
   sin(2 pi rf_freq t), x = L grounded, both absorbing, Sec. 3) or in a
   periodic box.  The paper computes no derivatives; the objectives are the
   time averages over the run's K steps of
     P^n = sum_p q w E_p vbar_p                 power absorbed by the electrons [W/m^2]
     G^n = sum_p w vbar_p S_1(xi_p - 1/2) / dx  electron current density at the centre
                                                of the first cell [1/(m^2 s)]
   with vbar = (v^{n-1/2} + v^{n+1/2})/2, and J = c_power <P> + c_flux <G>.
   Absorptions are events the derivative holds fixed; the offset quantisation
   of the charge assignment is differentiated as the smooth spline.  The
   forward run stores a checkpoint every checkpoint_every steps; the backward
   run recomputes each segment from its checkpoint and runs one reverse
   launch per step. */
typedef struct pic_adj_config {
    int32_t boundary;          /* PIC_BC_ELECTRODES / PIC_BC_PERIODIC */
    int32_t n_cells;           /* 2 .. 1024 */
    int32_t checkpoint_every;  /* >= 1 steps per recomputed segment */
    int32_t reserved0;
    int64_t n_particles;       /* electrons, 1 .. 2^29 */
    int64_t nsteps;            /* K >= 1 */
    int64_t step0;             /* time level of the initial state (sets the RF phase) */
    double length;             /* gap [m] */
    double dt;                 /* [s] */
    double rf_freq;            /* [Hz] */
    double n0;                 /* electron density the n_particles represent [m^-3] */
    double bg_density;         /* frozen ion density [m^-3] */
} pic_adj_config;

typedef struct pic_adj pic_adj;

/* Device bytes of the adjoint arena (checkpoints, one segment of levels, the
   field tables of every level, per-particle adjoints). */
int pic_adj_required_sizes(const pic_adj_config *cfg, pic_sizes *out);
/* Caller-owned arena as for pic_init (256-byte aligned, outlives the handle). */
int pic_adj_init(const pic_adj_config *cfg, const pic_buffers *bufs, void *cuda_stream, pic_adj **out);
/* Forward run from the initial state given as DEVICE arrays of n_particles
   entries (cell in [0, n_cells), off in [0, 1), vx = v^{-1/2} [m/s]; an entry
   with another cell or offset counts as no particle).  The arrays are copied;
   the caller may reuse them on return.  Writes the time-averaged P and G to
   the HOST array power_flux[2]; synchronises the stream.  rf_volt is ignored
   in the periodic box. */
int pic_adj_forward(pic_adj *h, double rf_volt, const int32_t *cell0, const float *off0,
                    const float *vx0, double *power_flux);
/* Gradient of J = c_power <P> + c_flux <G> for the last forward run: dJ/dv^{-1/2}
   into the DEVICE array d_vx0 [n_particles] (float), dJ/dx^0 [per metre] into the
   DEVICE array d_x0 (may be NULL), dJ/d rf_volt into the HOST double d_volt (may be
   NULL; 0 in the periodic box).  PIC_EINVAL without a preceding forward run.
   Synchronises the stream. */
int pic_adj_backward(pic_adj *h, double c_power, double c_flux, float *d_vx0, float *d_x0,
                     double *d_volt);
/* State of time level K of the last forward run, HOST arrays of n_particles
   entries (absorbed particles have cell = -1). */
int pic_adj_final_state(pic_adj *h, int32_t *cell, float *off, float *vx);
void pic_adj_free(pic_adj *h);

void pic_free(pic_handle *h);

/* Message of the last failing call on h (h may be NULL for pic_init /
   pic_required_sizes failures). */
const char *pic_last_error(const pic_handle *h);

#ifdef __cplusplus
}
#endif
#endif
