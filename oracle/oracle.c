/*
 * oracle.c -- plain FP64 CPU oracle for the 1D electrostatic PIC/MCC method of
 * Wang, Sun, Jiang & Kong (energy-conserving PIC/MC benchmarked on RF
 * capacitively coupled discharges).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product library.  It is
 * written for a reader checking it against the paper: one loop per step of the
 * method, in the order the method takes them, with no blocking or fusion.
 *
 * Readings of points the paper leaves open are marked "Reading:" and collected
 * in the design notes of the repository.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 values. */
#define Q_E      1.602176634e-19
#define M_E      9.1093837015e-31
#define AMU      1.66053906660e-27
#define K_B      1.380649e-23
#define EPS_0    8.8541878128e-12
#define PI_D     3.14159265358979323846
#define EULER_N  2.71828182845904523536

/* Philox stream tags (fourth counter word = species << 24 | tag << 16 | sub). */
#define TAG_LOAD 1u
#define TAG_MCC  2u
#define TAG_WAIT 3u
#define WAIT_CAP 262144u          /* 64^3 steps: the longest count a draw gives */
#define WAIT_REDRAW 0x40000000u   /* the count ends in a fresh draw, not a selection */

#define TWO_POW_16 65536
#define TWO_POW_33 ((int64_t)1 << 33)
#define TWO_POW_12 ((int64_t)4096)
#define TWO_POW_36 ((int64_t)1 << 36)

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the  */
/* published multipliers and Weyl key increments.                             */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t k0 = key[0], k1 = key[1];
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox_stream(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t c3, int64_t n, uint32_t *out)
{
    uint32_t key[2] = {k0, k1};
    for (int64_t k = 0; k < n; ++k) {
        uint32_t ctr[4] = {c0 + (uint32_t)k, c1, c2, c3};
        orc_philox4x32_10(key, ctr, out + 4 * k);
    }
}

/* Draw the four words keyed on (seed, run) with counter (id, step, tag). */
static void draw(const orc_params *p, uint32_t id, int64_t step, uint32_t species,
                 uint32_t tag, uint32_t sub, uint32_t w[4])
{
    uint32_t key[2] = {p->seed, p->run};
    uint32_t ctr[4] = {id, (uint32_t)((uint64_t)step & 0xffffffffu),
                       (uint32_t)((uint64_t)step >> 32), (species << 24) | (tag << 16) | sub};
    orc_philox4x32_10(key, ctr, w);
}

/* Uniform on (0,1) from the top 24 bits of a word. */
static double uniform24(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Box-Muller: two uniforms on (0,1) -> two standard normals. */
static void box_muller(double u1, double u2, double *n1, double *n2)
{
    double r = sqrt(-2.0 * log(u1));
    *n1 = r * cos(2.0 * PI_D * u2);
    *n2 = r * sin(2.0 * PI_D * u2);
}

/* ------------------------------------------------------------------------- */
/* Model cross sections (analytic stand-ins for the argon set the paper takes */
/* from its MCC reference, Sec. 3).                                           */
/* ------------------------------------------------------------------------- */
static double sigma_exc(const orc_params *p, double eps)
{
    if (eps < p->exc_thr) return 0.0;
    if (eps < p->exc_ramp_end)
        return p->sig_exc_max * (eps - p->exc_thr) / (p->exc_ramp_end - p->exc_thr);
    return p->sig_exc_max;
}

static double sigma_iz(const orc_params *p, double eps)
{
    if (eps <= p->iz_thr) return 0.0;
    return p->sig_iz_peak * EULER_N * (p->iz_thr / eps) * log(eps / p->iz_thr);
}

/* Null-collision selection by waiting times (reading of the null-collision
   method, whose selection the paper does not spell out): the number of steps
   W from a particle's selection, or from its entry into the run, to its next
   selection is geometric, P(W > k) = (1 - P_null)^k -- the law of one
   Bernoulli(P_null) trial per step, drawn once per selection.  W - 1 = X is
   made of three independent base-64 digits, X = 4096 a + 64 b + c: c and b
   follow the geometric laws of ratio q = 1 - P_null and q^64 cut to 0..63,
   a the geometric law of ratio q^4096, where a = 64 stands for X >= 64^3
   (the count of WAIT_CAP steps then ends in a fresh draw, not a selection;
   the law is memoryless).  Each digit is the number of thresholds
   T_j = floor(2^32 P(digit >= j)), j = 1..63 (1..64 for a), above a 32-bit
   Philox word; the thresholds come from FP64 pow on the host. */
static void wait_tables(double p_null, uint32_t t[3][64])
{
    double q = 1.0 - p_null;
    for (int dgt = 0; dgt < 3; ++dgt) {
        double r = dgt == 0 ? q : (dgt == 1 ? pow(q, 64.0) : pow(q, 4096.0));
        double r64 = pow(r, 64.0);
        for (int j = 1; j <= 64; ++j) {
            double frac;
            if (dgt == 2) {
                frac = pow(r, (double)j);                       /* P(a >= j) */
            } else if (j == 64) {
                t[dgt][63] = 0u;                                /* unused */
                continue;
            } else {
                frac = 1.0 - r64 > 0.0 ? (pow(r, (double)j) - r64) / (1.0 - r64) : 1.0;
            }
            double v = floor(ldexp(frac, 32));
            t[dgt][j - 1] = v >= 4294967295.0 ? 0xffffffffu : (uint32_t)v;
        }
    }
}

void orc_derive(const orc_params *p, orc_derived *d)
{
    memset(d, 0, sizeof(*d));
    d->dx = p->length / p->n_cells;
    d->weight = p->n0 * p->length / p->np_init;
    d->q[0] = -Q_E;
    d->q[1] = Q_E;
    d->m[0] = M_E;
    d->m[1] = p->ion_mass_amu * AMU;
    d->vth[0] = sqrt(Q_E * p->te_ev / d->m[0]);
    d->vth[1] = sqrt(Q_E * p->ti_ev / d->m[1]);
    d->vth_gas = sqrt(K_B * p->gas_temp / d->m[1]);
    if (!p->mcc) return;
    /* Null-collision bound (Vahedi & Surendra 1995).  Reading: the bound is
       the sum over processes of each process's maximum of n_g sigma v over
       energies up to eps_cap; elastic and excitation rise monotonically, and
       sigma_iz v peaks where ln(eps/I) = 2. */
    double v_cap = sqrt(2.0 * Q_E * p->eps_cap / M_E);
    double eps_star = p->eps_cap < p->iz_thr * EULER_N * EULER_N ? p->eps_cap
                                                                   : p->iz_thr * EULER_N * EULER_N;
    double v_star = sqrt(2.0 * Q_E * eps_star / M_E);
    d->nu_max_e = p->gas_density * (p->sig_el * v_cap + sigma_exc(p, p->eps_cap) * v_cap +
                                    sigma_iz(p, eps_star) * v_star);
    d->g_max_i = sqrt(2.0 * Q_E * p->cx_vmax / d->m[1]) + 6.0 * d->vth_gas;
    d->nu_max_i = p->gas_density * p->sig_cx * d->g_max_i;
    d->p_null_e = 1.0 - exp(-d->nu_max_e * p->dt);
    d->p_null_i = 1.0 - exp(-d->nu_max_i * p->dt);
    d->thr_e = (uint32_t)floor(d->p_null_e * 16777216.0);
    d->thr_i = (uint32_t)floor(d->p_null_i * 16777216.0);
    wait_tables(d->p_null_e, d->wait_thr[0]);
    wait_tables(d->p_null_i, d->wait_thr[1]);
}

/* One digit of the waiting time: the number of thresholds above u. */
static uint32_t wait_digit(const uint32_t *t, int n, uint32_t u)
{
    uint32_t d = 0;
    for (int j = 0; j < n; ++j)
        if (u < t[j]) d += 1;
    return d;
}

uint32_t orc_wait_draw(const orc_params *p, const orc_derived *d, int species, uint32_t id,
                       int64_t step, uint32_t sub)
{
    if ((species == 0 ? d->p_null_e : d->p_null_i) <= 0.0) return WAIT_CAP | WAIT_REDRAW;
    uint32_t w[4];
    draw(p, id, step, (uint32_t)species, TAG_WAIT, sub, w);
    uint32_t a = wait_digit(d->wait_thr[species][2], 64, w[0]);
    if (a == 64u) return WAIT_CAP | WAIT_REDRAW;
    uint32_t b = wait_digit(d->wait_thr[species][1], 63, w[1]);
    uint32_t c = wait_digit(d->wait_thr[species][0], 63, w[2]);
    return 1u + 4096u * a + 64u * b + c;
}

void orc_wait_draws(const orc_params *p, int species, int64_t n, const uint32_t *id, int64_t step,
                    uint32_t sub, uint32_t *out)
{
    orc_derived d;
    orc_derive(p, &d);
    for (int64_t k = 0; k < n; ++k) out[k] = orc_wait_draw(p, &d, species, id[k], step, sub);
}

/* ------------------------------------------------------------------------- */
/* Charge assignment, Eq. (2): rho(x_g) = sum_p q_p S_m(x_g - x_p), m = 2.     */
/* ------------------------------------------------------------------------- */

/* Split a position in cell units into (cell, FP32 offset) and quantise the
   offset to 16 bits.  The quantised code is an integer decided from a float,
   so it is decided in the precision the device kernels store offsets in
   (FP32); an offset that rounds up to 1 moves to the next cell. */
static void quantise_offset(double xi, int64_t *cell, int64_t *code)
{
    double c = floor(xi);
    float off = (float)(xi - c);
    if (off >= 1.0f) {
        c += 1.0;
        off = 0.0f;
    }
    *cell = (int64_t)c;
    *code = (int64_t)floor((double)off * 65536.0);
}

/* Fold (walls) or wrap (periodic) a node index that may lie one node outside. */
static int64_t node_index(const orc_params *p, int64_t g)
{
    int64_t n = p->n_cells;
    if (p->periodic) return ((g % n) + n) % n;
    if (g < 0) return 0;   /* ghost node beyond x=0 folds onto the wall node */
    if (g > n) return n;   /* ghost node beyond x=L folds onto the wall node */
    return g;
}

/* S_2 (quadratic B-spline) weights in units of 2^-33: with the nearest node j
   and a = (1/2 + delta) 2^16, b = 2^16 - a, the nodes j-1, j, j+1 receive
   b^2, 2^33 - a^2 - b^2 and a^2, which are 2^33 times (1/2-delta)^2/2,
   3/4 - delta^2 and (1/2+delta)^2/2. */
void orc_deposit_s2_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out)
{
    memset(out, 0, sizeof(int64_t) * (size_t)(p->n_cells + 1));
    for (int64_t k = 0; k < n; ++k) {
        int64_t cell, code;
        quantise_offset(xi[k], &cell, &code);
        int64_t j, a;
        if (code < TWO_POW_16 / 2) {
            j = cell;
            a = code + TWO_POW_16 / 2;
        } else {
            j = cell + 1;
            a = code - TWO_POW_16 / 2;
        }
        int64_t b = TWO_POW_16 - a;
        out[node_index(p, j - 1)] += b * b;
        out[node_index(p, j)] += TWO_POW_33 - a * a - b * b;
        out[node_index(p, j + 1)] += a * a;
    }
}

void orc_deposit_s2_fp64(const orc_params *p, int64_t n, const double *xi, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)(p->n_cells + 1));
    for (int64_t k = 0; k < n; ++k) {
        double jd = floor(xi[k] + 0.5);
        double delta = xi[k] - jd;
        int64_t j = (int64_t)jd;
        out[node_index(p, j - 1)] += 0.5 * (0.5 - delta) * (0.5 - delta);
        out[node_index(p, j)] += 0.75 - delta * delta;
        out[node_index(p, j + 1)] += 0.5 * (0.5 + delta) * (0.5 + delta);
    }
}

/* S_1 (linear) assignment to nodes: the momentum-conserving scheme. */
void orc_deposit_s1_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out)
{
    memset(out, 0, sizeof(int64_t) * (size_t)(p->n_cells + 1));
    for (int64_t k = 0; k < n; ++k) {
        int64_t cell, code;
        quantise_offset(xi[k], &cell, &code);
        out[node_index(p, cell)] += (TWO_POW_16 - code) << 17;
        out[node_index(p, cell + 1)] += code << 17;
    }
}

/* m = 3 (Eq. (2) with the cubic B-spline S_3; Sec. 2 allows m > 2).  With
   xi = i + t, 0 <= t < 1, the nodes i-1, i, i+1, i+2 receive
       (1-t)^3 / 6,  (3t^3 - 6t^2 + 4) / 6,  (-3t^3 + 3t^2 + 3t + 1) / 6,  t^3 / 6,
   the values of S_3 at distances 1+t, t, 1-t and 2-t.  Fixed point: the
   offset is quantised to 12 bits, t = F / 2^12, and each weight is kept as
   6 * 2^36 times itself, an integer polynomial in F (exact in int64). */
static void quantise_offset12(double xi, int64_t *cell, int64_t *code)
{
    double c = floor(xi);
    float off = (float)(xi - c);
    if (off >= 1.0f) {
        c += 1.0;
        off = 0.0f;
    }
    *cell = (int64_t)c;
    *code = (int64_t)floor((double)off * 4096.0);
}

void orc_deposit_s3_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out)
{
    const int64_t T = TWO_POW_12;
    memset(out, 0, sizeof(int64_t) * (size_t)(p->n_cells + 1));
    for (int64_t k = 0; k < n; ++k) {
        int64_t i, F;
        quantise_offset12(xi[k], &i, &F);
        int64_t G = T - F;
        out[node_index(p, i - 1)] += G * G * G;
        out[node_index(p, i)] += 3 * F * F * F - 6 * T * F * F + 4 * T * T * T;
        out[node_index(p, i + 1)] += -3 * F * F * F + 3 * T * F * F + 3 * T * T * F + T * T * T;
        out[node_index(p, i + 2)] += F * F * F;
    }
}

void orc_deposit_s3_fp64(const orc_params *p, int64_t n, const double *xi, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)(p->n_cells + 1));
    for (int64_t k = 0; k < n; ++k) {
        double id = floor(xi[k]);
        double t = xi[k] - id;
        int64_t i = (int64_t)id;
        out[node_index(p, i - 1)] += (1.0 - t) * (1.0 - t) * (1.0 - t) / 6.0;
        out[node_index(p, i)] += (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
        out[node_index(p, i + 1)] += (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
        out[node_index(p, i + 2)] += t * t * t / 6.0;
    }
}

int64_t orc_charge_unit(const orc_params *p)
{
    return p->scheme == ORC_EC3_EXPLICIT ? 6 * TWO_POW_36 : TWO_POW_33;
}

/* Susceptibility weights: S_1 from the predicted position to cell centres,
   units 2^-16.  With the nearest node j and a as above, the centre of cell j
   gets a and the centre of cell j-1 gets 2^16 - a.  Reading: weight falling in
   the ghost cells beyond an electrode is dropped (conductor). */
static void deposit_chi_fixed(const orc_params *p, int64_t n, const double *xi, int64_t *out)
{
    int64_t nc = p->n_cells;
    memset(out, 0, sizeof(int64_t) * (size_t)nc);
    for (int64_t k = 0; k < n; ++k) {
        int64_t cell, code;
        quantise_offset(xi[k], &cell, &code);
        int64_t j, a;
        if (code < TWO_POW_16 / 2) {
            j = cell;
            a = code + TWO_POW_16 / 2;
        } else {
            j = cell + 1;
            a = code - TWO_POW_16 / 2;
        }
        int64_t cl = j - 1, cr = j;
        if (p->periodic) {
            cl = ((cl % nc) + nc) % nc;
            cr = ((cr % nc) + nc) % nc;
            out[cl] += TWO_POW_16 - a;
            out[cr] += a;
        } else {
            if (cl >= 0) out[cl] += TWO_POW_16 - a;
            if (cr < nc) out[cr] += a;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Field solve (Sec. 2, "field solving"): finite-difference Poisson equation  */
/* on the nodes, optionally with the implicit susceptibility on cell faces.   */
/* ------------------------------------------------------------------------- */
void orc_solve_dirichlet(int n_cells, double dx, const double *rho, const double *chi,
                         double v_left, double *phi)
{
    int n = n_cells;
    phi[0] = v_left;
    phi[n] = 0.0;
    if (n < 2) return;
    int m = n - 1; /* unknowns phi[1..n-1] */
    double *cp = (double *)malloc(sizeof(double) * (size_t)m);
    double *dp = (double *)malloc(sizeof(double) * (size_t)m);
    for (int k = 0; k < m; ++k) {
        int g = k + 1;
        double eps_l = 1.0 + (chi ? chi[g - 1] : 0.0); /* face between g-1 and g */
        double eps_r = 1.0 + (chi ? chi[g] : 0.0);     /* face between g and g+1 */
        double a = -eps_l, b = eps_l + eps_r, c = -eps_r;
        double d = rho[g] * dx * dx / EPS_0;
        if (g == 1) d -= a * v_left;
        if (k == 0) {
            cp[k] = c / b;
            dp[k] = d / b;
        } else {
            double den = b - a * cp[k - 1];
            cp[k] = c / den;
            dp[k] = (d - a * dp[k - 1]) / den;
        }
    }
    phi[m] = dp[m - 1];
    for (int k = m - 2; k >= 0; --k) phi[k + 1] = dp[k] - cp[k] * phi[k + 2];
    free(cp);
    free(dp);
}

/* Periodic box: the cyclic system is solvable when the net charge is zero, so
   the mean charge density is removed; with the gauge phi[0] = 0 the remaining
   equations g = 1..N-1 are the Dirichlet system with both ends at zero. */
void orc_solve_periodic(int n_cells, double dx, const double *rho, const double *chi,
                        double *phi)
{
    int n = n_cells;
    double mean = 0.0;
    for (int g = 0; g < n; ++g) mean += rho[g];
    mean /= n;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    for (int g = 0; g < n; ++g) r[g] = rho[g] - mean;
    r[n] = 0.0;
    orc_solve_dirichlet(n, dx, r, chi, 0.0, phi);
    free(r);
}

/* ------------------------------------------------------------------------- */
/* Force interpolation, Eq. (3): F(x_p) = sum_g q E_g S_{m-1}(x_p - x_{g+1/2}) */
/* with m = 2: linear interpolation from the cell-centred field E_{g+1/2} =   */
/* (phi_g - phi_{g+1}) / dx.  Reading: E = 0 in the ghost cells beyond an     */
/* electrode.                                                                  */
/* ------------------------------------------------------------------------- */
static double cell_field(const orc_params *p, const double *e_cc, int64_t c)
{
    int64_t n = p->n_cells;
    if (p->periodic) return e_cc[((c % n) + n) % n];
    if (c < 0 || c >= n) return 0.0;
    return e_cc[c];
}

double orc_gather_ec(const orc_params *p, const double *e_cc, double xi)
{
    double jd = floor(xi + 0.5);
    double delta = xi - jd;
    int64_t j = (int64_t)jd;
    return (0.5 - delta) * cell_field(p, e_cc, j - 1) + (0.5 + delta) * cell_field(p, e_cc, j);
}

/* m = 3: Eq. (3) with S_2 centred on the cell centres.  With xi = i + t the
   centres of cells i-1, i, i+1 lie at distances 1/2 + t, |t - 1/2| and
   3/2 - t, where S_2 is (1-t)^2 / 2, 3/4 - (t - 1/2)^2 and t^2 / 2. */
double orc_gather_ec3(const orc_params *p, const double *e_cc, double xi)
{
    double id = floor(xi);
    double t = xi - id;
    int64_t i = (int64_t)id;
    double d = t - 0.5;
    return 0.5 * (1.0 - t) * (1.0 - t) * cell_field(p, e_cc, i - 1) + (0.75 - d * d) * cell_field(p, e_cc, i) +
           0.5 * t * t * cell_field(p, e_cc, i + 1);
}

/* Momentum-conserving gather: linear interpolation from node fields. */
double orc_gather_mc(const orc_params *p, const double *e_node, double xi)
{
    int64_t n = p->n_cells;
    double id = floor(xi);
    double f = xi - id;
    int64_t i = (int64_t)id;
    int64_t i1 = i + 1;
    if (p->periodic) {
        i = ((i % n) + n) % n;
        i1 = ((i1 % n) + n) % n;
    }
    return (1.0 - f) * e_node[i] + f * e_node[i1];
}

/* ------------------------------------------------------------------------- */
/* Non-uniform grid (the multi-scale grid of Sec. 4).  The paper gives no form */
/* of Eq. (2)-(3) for unequal cells; the reading here keeps them in the cell  */
/* coordinate xi (the uniform-grid weights of xi) and takes as the force the  */
/* exact x-derivative of the particle's potential energy, so that the energy */
/* argument of the EC scheme carries over: with xi(x) linear inside each cell,*/
/* d/dx = (1/h_c) d/dxi there.  The field equation is the Gauss law between   */
/* the physical nodes, whose matrix is symmetric.                             */
/* ------------------------------------------------------------------------- */
void orc_grid_nodes(int n_cells, const double *h, double *x)
{
    x[0] = 0.0;
    for (int c = 0; c < n_cells; ++c) x[c + 1] = x[c] + h[c];
}

int orc_locate(int n_cells, const double *x_nodes, const double *h, double x, int64_t *cell,
               double *off)
{
    if (x < x_nodes[0]) return -1;
    if (x >= x_nodes[n_cells]) return 1;
    /* bisection for the last node at or below x */
    int lo = 0, hi = n_cells;  /* x_nodes[lo] <= x < x_nodes[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x_nodes[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    *cell = lo;
    *off = (x - x_nodes[lo]) / h[lo];
    if (*off >= 1.0) *off = nextafter(1.0, 0.0);  /* rounding at the right node */
    return 0;
}

void orc_solve_dirichlet_h(int n_cells, const double *h, const double *q_node, const double *chi,
                           double v_left, double *phi)
{
    int n = n_cells;
    phi[0] = v_left;
    phi[n] = 0.0;
    if (n < 2) return;
    int m = n - 1; /* unknowns phi[1..n-1] */
    double *cp = (double *)malloc(sizeof(double) * (size_t)m);
    double *dp = (double *)malloc(sizeof(double) * (size_t)m);
    for (int k = 0; k < m; ++k) {
        int g = k + 1;
        double a = -(1.0 + (chi ? chi[g - 1] : 0.0)) / h[g - 1];
        double c = -(1.0 + (chi ? chi[g] : 0.0)) / h[g];
        double b = -a - c;
        double d = q_node[g] / EPS_0;
        if (g == 1) d -= a * v_left;
        if (k == 0) {
            cp[k] = c / b;
            dp[k] = d / b;
        } else {
            double den = b - a * cp[k - 1];
            cp[k] = c / den;
            dp[k] = (d - a * dp[k - 1]) / den;
        }
    }
    phi[m] = dp[m - 1];
    for (int k = m - 2; k >= 0; --k) phi[k + 1] = dp[k] - cp[k] * phi[k + 2];
    free(cp);
    free(dp);
}

void orc_solve_periodic_h(int n_cells, const double *h, const double *q_node, const double *chi,
                          double *phi)
{
    int n = n_cells;
    double len = 0.0, tot = 0.0;
    for (int c = 0; c < n; ++c) len += h[c];
    for (int g = 0; g < n; ++g) tot += q_node[g];
    double *r = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    for (int g = 0; g < n; ++g) {
        double hl = h[(g - 1 + n) % n], hr = h[g];
        r[g] = q_node[g] - tot * 0.5 * (hl + hr) / len;
    }
    r[n] = 0.0;
    orc_solve_dirichlet_h(n, h, r, chi, 0.0, phi);
    free(r);
}

double orc_gather_ec_h(const orc_params *p, const double *u_cc, double xi)
{
    int64_t c = (int64_t)floor(xi);
    return orc_gather_ec(p, u_cc, xi) / p->cell_width[c];
}

/* m = 3: U = q sum_g phi_g S_3(xi - g) has the x-derivative
   -(q / h_c) sum_c (phi_c - phi_{c+1}) S_2(xi - c - 1/2): Eq. (3)'s S_2
   interpolation of the voltage drops over the particle's own cell width. */
double orc_gather_ec3_h(const orc_params *p, const double *u_cc, double xi)
{
    int64_t c = (int64_t)floor(xi);
    return orc_gather_ec3(p, u_cc, xi) / p->cell_width[c];
}

/* ------------------------------------------------------------------------- */
/* Scattering geometry: turn the unit vector d by polar angle chi and azimuth */
/* phi.  The azimuth is measured in the basis e1 = d(theta)/dtheta,           */
/* e2 = d(psi)/dpsi / sin(theta) of the polar angles of d about the x axis.   */
/* ------------------------------------------------------------------------- */
void orc_rotate(const double d[3], double cos_chi, double phi, double out[3])
{
    double sin_chi = sqrt(fmax(0.0, 1.0 - cos_chi * cos_chi));
    double cp = cos(phi), sp = sin(phi);
    double st = sqrt(d[1] * d[1] + d[2] * d[2]);
    if (st > 1e-6) {
        out[0] = cos_chi * d[0] - sin_chi * cp * st;
        out[1] = cos_chi * d[1] + sin_chi * (cp * d[0] * d[1] - sp * d[2]) / st;
        out[2] = cos_chi * d[2] + sin_chi * (cp * d[0] * d[2] + sp * d[1]) / st;
    } else {
        /* d along +-x: the limit of the basis above is e1 = (0, d_x, 0), e2 = (0, 0, 1). */
        out[0] = cos_chi * d[0];
        out[1] = sin_chi * cp * d[0];
        out[2] = sin_chi * sp;
    }
}

/* Vahedi & Surendra's anisotropic scattering law (their screened-Coulomb fit
   to the differential cross section sigma(eps, chi) proportional to
   eps / ((1 + eps sin^2(chi/2)) ln(1 + eps)), eps in eV), sampled by inverting
   its cumulative distribution: cos chi = (2 + eps - 2 (1 + eps)^u) / eps. */
double orc_vs_cos_chi(double eps, double u)
{
    if (eps <= 0.0) return 1.0 - 2.0 * u;  /* the isotropic limit */
    return (2.0 + eps - 2.0 * pow(1.0 + eps, u)) / eps;
}

/* Opal, Pollock & Wagner's secondary-electron spectrum, proportional to
   1 / (1 + (eps_s / B)^2) on [0, excess / 2], sampled by inverting its
   cumulative distribution arctan(eps_s / B) / arctan(excess / (2B)). */
double orc_opal_secondary(double excess, double b, double u)
{
    if (excess <= 0.0) return 0.0;
    return b * tan(u * atan(excess / (2.0 * b)));
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n, cap;
    double *xi, *vx, *vy, *vz, *abar;
    uint32_t *id;
    uint32_t *wait;   /* steps to the next null-collision selection (| WAIT_REDRAW) */
    uint8_t *dead;
    uint32_t next_id;
} species_t;

typedef struct {
    uint32_t pid;
    double xi;
    double ve[3], vi[3];
    double abar_e, abar_i;
} birth_t;

struct orc_sim {
    orc_params p;
    orc_derived d;
    species_t sp[2];
    int64_t step;
    int64_t *rho_q[2];  /* [N+1], units 2^-33 particle charge (fixed) */
    double *rho_f[2];   /* [N+1], particle units (fp64 mode) */
    int64_t *chi_q[2];  /* [N], units 2^-16 */
    double *rho, *chi, *phi, *e_cc, *e_node;
    /* non-uniform grid (NULL on the uniform grid): cell widths, node
       positions, voltage drops phi_c - phi_{c+1} of the cells */
    double *h, *xn, *u_cc;
    birth_t *births;
    int64_t n_births, cap_births;
    /* diagnostics */
    orc_diag dg;
    double *avg_ne, *avg_ni, *avg_phi, *heat[2];
    int64_t *eedf;
};

static int species_alloc(species_t *s, int64_t cap)
{
    memset(s, 0, sizeof(*s));
    s->cap = cap;
    size_t c = (size_t)(cap > 0 ? cap : 1);
    s->xi = (double *)calloc(c, sizeof(double));
    s->vx = (double *)calloc(c, sizeof(double));
    s->vy = (double *)calloc(c, sizeof(double));
    s->vz = (double *)calloc(c, sizeof(double));
    s->abar = (double *)calloc(c, sizeof(double));
    s->id = (uint32_t *)calloc(c, sizeof(uint32_t));
    s->wait = (uint32_t *)calloc(c, sizeof(uint32_t));
    s->dead = (uint8_t *)calloc(c, 1);
    return s->xi && s->vx && s->vy && s->vz && s->abar && s->id && s->wait && s->dead ? 0 : -1;
}

static void species_free(species_t *s)
{
    free(s->xi); free(s->vx); free(s->vy); free(s->vz); free(s->abar); free(s->id);
    free(s->wait); free(s->dead);
}

orc_sim *orc_sim_create(const orc_params *p, int64_t cap_e, int64_t cap_i)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    orc_derive(p, &s->d);
    int64_t nn = p->n_cells + 1;
    if (species_alloc(&s->sp[0], cap_e) || species_alloc(&s->sp[1], cap_i)) {
        orc_sim_free(s);
        return NULL;
    }
    for (int k = 0; k < 2; ++k) {
        s->rho_q[k] = (int64_t *)calloc((size_t)nn, sizeof(int64_t));
        s->rho_f[k] = (double *)calloc((size_t)nn, sizeof(double));
        s->chi_q[k] = (int64_t *)calloc((size_t)nn, sizeof(int64_t));
        s->heat[k] = (double *)calloc((size_t)nn, sizeof(double));
    }
    s->rho = (double *)calloc((size_t)nn, sizeof(double));
    s->chi = (double *)calloc((size_t)nn, sizeof(double));
    s->phi = (double *)calloc((size_t)nn, sizeof(double));
    s->e_cc = (double *)calloc((size_t)nn, sizeof(double));
    s->e_node = (double *)calloc((size_t)nn, sizeof(double));
    s->avg_ne = (double *)calloc((size_t)nn, sizeof(double));
    s->avg_ni = (double *)calloc((size_t)nn, sizeof(double));
    s->avg_phi = (double *)calloc((size_t)nn, sizeof(double));
    s->eedf = (int64_t *)calloc((size_t)(p->eedf_bins + 1), sizeof(int64_t));
    if (p->cell_width) {
        /* the EC schemes (explicit with m = 2 or 3, direct implicit) with
           mobile ions are the ones defined on it */
        if ((p->scheme != ORC_EC_EXPLICIT && p->scheme != ORC_EC_IMPLICIT && p->scheme != ORC_EC3_EXPLICIT) ||
            !p->ions_mobile) {
            orc_sim_free(s);
            return NULL;
        }
        s->h = (double *)malloc(sizeof(double) * (size_t)p->n_cells);
        s->xn = (double *)malloc(sizeof(double) * (size_t)nn);
        s->u_cc = (double *)calloc((size_t)nn, sizeof(double));
        memcpy(s->h, p->cell_width, sizeof(double) * (size_t)p->n_cells);
        orc_grid_nodes(p->n_cells, s->h, s->xn);
        s->p.cell_width = s->h;  /* the caller's array may go away */
    }
    s->cap_births = cap_e > 1024 ? cap_e : 1024;
    s->births = (birth_t *)calloc((size_t)s->cap_births, sizeof(birth_t));
    return s;
}

void orc_sim_free(orc_sim *s)
{
    if (!s) return;
    species_free(&s->sp[0]);
    species_free(&s->sp[1]);
    for (int k = 0; k < 2; ++k) {
        free(s->rho_q[k]); free(s->rho_f[k]); free(s->chi_q[k]); free(s->heat[k]);
    }
    free(s->rho); free(s->chi); free(s->phi); free(s->e_cc); free(s->e_node);
    free(s->avg_ne); free(s->avg_ni); free(s->avg_phi); free(s->eedf); free(s->births);
    free(s->h); free(s->xn); free(s->u_cc);
    free(s);
}

/* The momentum-conserving scheme always assigns in fixed point (S_1 weights
   of a 16-bit code are exact), the EC schemes when `quantized` is set. */
static int is_mc(const orc_params *p) { return p->scheme == ORC_MC_EXPLICIT || p->scheme == ORC_MC_IMPLICIT; }
static int is_implicit(const orc_params *p) { return p->scheme == ORC_EC_IMPLICIT || p->scheme == ORC_MC_IMPLICIT; }
static int uses_fixed(const orc_params *p) { return p->quantized || is_mc(p); }

/* The length a node's charge is spread over in the densities: dx on the
   uniform grid; on a non-uniform one the mean (h_{g-1} + h_g) / 2 of the two
   cells beside it, the wall nodes taking the one cell they have twice (as
   the uniform grid's wall nodes take dx), wrapped in a periodic box. */
static double node_len(const orc_sim *s, int64_t g)
{
    if (!s->h) return s->d.dx;
    int64_t n = s->p.n_cells;
    double hl, hr;
    if (s->p.periodic) {
        hl = s->h[(g - 1 + n) % n];
        hr = s->h[g % n];
    } else {
        hl = s->h[g > 0 ? g - 1 : 0];
        hr = s->h[g < n ? g : n - 1];
    }
    return 0.5 * (hl + hr);
}

/* Charge density at the nodes [C/m^3] from the per-species assignments. */
static void assemble_rho(orc_sim *s)
{
    const orc_params *p = &s->p;
    int64_t nn = p->n_cells + 1;
    for (int64_t g = 0; g < nn; ++g) {
        double scale = s->d.weight / node_len(s, g);
        double ne, ni;
        if (uses_fixed(p)) {
            ne = (double)s->rho_q[0][g] / (double)orc_charge_unit(p);
            ni = (double)s->rho_q[1][g] / (double)orc_charge_unit(p);
        } else {
            ne = s->rho_f[0][g];
            ni = s->rho_f[1][g];
        }
        s->rho[g] = Q_E * scale * (ni - ne);
        if (!p->ions_mobile) s->rho[g] += Q_E * p->bg_density;
    }
}

static void deposit_species(orc_sim *s, int k, int use_s1)
{
    species_t *sp = &s->sp[k];
    if (s->p.scheme == ORC_EC3_EXPLICIT) {
        if (s->p.quantized)
            orc_deposit_s3_fixed(&s->p, sp->n, sp->xi, s->rho_q[k]);
        else
            orc_deposit_s3_fp64(&s->p, sp->n, sp->xi, s->rho_f[k]);
    } else if (use_s1)
        orc_deposit_s1_fixed(&s->p, sp->n, sp->xi, s->rho_q[k]);
    else if (s->p.quantized)
        orc_deposit_s2_fixed(&s->p, sp->n, sp->xi, s->rho_q[k]);
    else
        orc_deposit_s2_fp64(&s->p, sp->n, sp->xi, s->rho_f[k]);
}

static double rf_voltage(const orc_params *p, int64_t n)
{
    if (p->periodic) return 0.0;
    return p->rf_volt * sin(2.0 * PI_D * p->rf_freq * (double)n * p->dt);
}

void orc_fields(const orc_params *p, const double *phi, double *e_cc, double *e_node)
{
    int n = p->n_cells;
    double dx = p->length / n;
    for (int c = 0; c < n; ++c) {
        double right = (p->periodic && c + 1 == n) ? phi[0] : phi[c + 1];
        e_cc[c] = (phi[c] - right) / dx;
    }
    for (int g = 0; g <= n; ++g) {
        if (p->periodic) {
            int gl = (g - 1 + n) % n, gr = (g + 1) % n;
            e_node[g] = (phi[gl] - phi[gr]) / (2.0 * dx);
        } else if (g == 0) {
            e_node[g] = (phi[0] - phi[1]) / dx;
        } else if (g == n) {
            e_node[g] = (phi[n - 1] - phi[n]) / dx;
        } else {
            e_node[g] = (phi[g - 1] - phi[g + 1]) / (2.0 * dx);
        }
    }
    if (p->periodic) e_node[n] = e_node[0];
}

/* Solve for phi at time level `level` and form the cell-centre and node fields. */
static void solve_field(orc_sim *s, const double *chi, int64_t level)
{
    const orc_params *p = &s->p;
    int n = p->n_cells;
    double dx = s->d.dx;
    if (s->h) {
        /* Gauss law on the physical nodes with the node charges per area */
        double *qn = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        for (int g = 0; g <= n; ++g) qn[g] = s->rho[g] * node_len(s, g);
        if (p->periodic)
            orc_solve_periodic_h(n, s->h, qn, chi, s->phi);
        else
            orc_solve_dirichlet_h(n, s->h, qn, chi, rf_voltage(p, level), s->phi);
        free(qn);
        double w = 0.0;
        for (int c = 0; c < n; ++c) {
            double right = (p->periodic && c + 1 == n) ? s->phi[0] : s->phi[c + 1];
            s->u_cc[c] = s->phi[c] - right;
            s->e_cc[c] = s->u_cc[c] / s->h[c];
            w += s->e_cc[c] * s->e_cc[c] * s->h[c];
        }
        s->dg.field_energy = 0.5 * EPS_0 * w;
        return;
    }
    if (p->periodic)
        orc_solve_periodic(n, dx, s->rho, chi, s->phi);
    else
        orc_solve_dirichlet(n, dx, s->rho, chi, rf_voltage(p, level), s->phi);
    orc_fields(p, s->phi, s->e_cc, s->e_node);
    double w = 0.0;
    for (int c = 0; c < n; ++c) w += s->e_cc[c] * s->e_cc[c];
    s->dg.field_energy = 0.5 * EPS_0 * w * dx;
}

static double gather(const orc_sim *s, double xi)
{
    if (s->h)
        return s->p.scheme == ORC_EC3_EXPLICIT ? orc_gather_ec3_h(&s->p, s->u_cc, xi)
                                               : orc_gather_ec_h(&s->p, s->u_cc, xi);
    if (is_mc(&s->p)) return orc_gather_mc(&s->p, s->e_node, xi);
    if (s->p.scheme == ORC_EC3_EXPLICIT) return orc_gather_ec3(&s->p, s->e_cc, xi);
    return orc_gather_ec(&s->p, s->e_cc, xi);
}

/* Charge assignment of the current positions, then the field at time level n. */
static void deposit_and_solve(orc_sim *s, int64_t level)
{
    int use_s1 = is_mc(&s->p);
    deposit_species(s, 0, use_s1);
    deposit_species(s, 1, use_s1);
    assemble_rho(s);
    solve_field(s, NULL, level);
}

static void accumulate_averages(orc_sim *s)
{
    const orc_params *p = &s->p;
    int64_t nn = p->n_cells + 1;
    for (int64_t g = 0; g < nn; ++g) {
        double scale = s->d.weight / node_len(s, g);
        double ne, ni;
        if (uses_fixed(p)) {
            ne = (double)s->rho_q[0][g] / (double)orc_charge_unit(p);
            ni = (double)s->rho_q[1][g] / (double)orc_charge_unit(p);
        } else {
            ne = s->rho_f[0][g];
            ni = s->rho_f[1][g];
        }
        s->avg_ne[g] += scale * ne;
        s->avg_ni[g] += scale * ni;
        s->avg_phi[g] += s->phi[g];
    }
    s->dg.n_avg += 1;
}

int orc_sim_load(orc_sim *s, int64_t n_e, int64_t n_i)
{
    const orc_params *p = &s->p;
    int64_t nload[2] = {n_e, n_i};
    for (int k = 0; k < 2; ++k) {
        species_t *sp = &s->sp[k];
        if (nload[k] > sp->cap) return -1;
        sp->n = nload[k];
        for (int64_t i = 0; i < sp->n; ++i) {
            uint32_t w[4], w2[4];
            draw(p, (uint32_t)i, 0, (uint32_t)k, TAG_LOAD, 0, w);
            draw(p, (uint32_t)i, 0, (uint32_t)k, TAG_LOAD, 1, w2);
            /* Uniform fill between the electrodes (Sec. 3): the position in
               cell units is w0 * N / 2^32, cut to 24 fractional bits. */
            uint64_t t = (uint64_t)w[0] * (uint64_t)p->n_cells;
            double cell = (double)(t >> 32);
            double off = (double)((uint32_t)t >> 8) * (1.0 / 16777216.0);
            if (s->h) {
                /* non-uniform grid: uniform in x = (w0 / 2^32) L, the offset
                   kept to FP32 (the storage precision of the particle) */
                int64_t c;
                double o;
                double x = ldexp((double)w[0], -32) * s->xn[p->n_cells];
                orc_locate(p->n_cells, s->xn, s->h, x, &c, &o);
                float of = (float)o;
                if (of >= 1.0f) {  /* rounds onto the next node */
                    if (c + 1 < p->n_cells) {
                        of = 0.0f;
                        c += 1;
                    } else {
                        of = nextafterf(1.0f, 0.0f);  /* stays below x = L */
                    }
                }
                cell = (double)c;
                off = (double)of;
            }
            sp->xi[i] = cell + off;
            double n1, n2, n3, n4;
            box_muller(uniform24(w[1]), uniform24(w[2]), &n1, &n2);
            box_muller(uniform24(w[3]), uniform24(w2[0]), &n3, &n4);
            sp->vx[i] = s->d.vth[k] * n1;
            sp->vy[i] = s->d.vth[k] * n2;
            sp->vz[i] = s->d.vth[k] * n3;
            sp->abar[i] = 0.0;
            sp->id[i] = (uint32_t)i;
            sp->wait[i] = p->mcc ? orc_wait_draw(p, &s->d, k, (uint32_t)i, 0, 1) : 0u;
            sp->dead[i] = 0;
        }
        sp->next_id = (uint32_t)sp->n;
    }
    s->step = 0;
    orc_sim_init_field(s, 1);
    return 0;
}

int orc_sim_set(orc_sim *s, int species, int64_t n, const double *xi, const double *vx,
                const double *vy, const double *vz, const uint32_t *id, const double *abar,
                uint32_t next_id, const uint32_t *wait)
{
    species_t *sp = &s->sp[species];
    if (n > sp->cap) return -1;
    sp->n = n;
    for (int64_t i = 0; i < n; ++i) {
        sp->xi[i] = xi[i];
        sp->vx[i] = vx[i];
        sp->vy[i] = vy[i];
        sp->vz[i] = vz[i];
        sp->id[i] = id[i];
        sp->abar[i] = abar ? abar[i] : 0.0;
        if (wait)
            sp->wait[i] = wait[i];
        else
            sp->wait[i] = s->p.mcc ? orc_wait_draw(&s->p, &s->d, species, id[i], s->step, 1) : 0u;
        sp->dead[i] = 0;
    }
    sp->next_id = next_id;
    return 0;
}

void orc_sim_init_field(orc_sim *s, int set_abar)
{
    deposit_and_solve(s, s->step);
    if (is_implicit(&s->p) && set_abar) {
        /* Reading: the first step of the direct-implicit push takes
           abar^{-1} = a^0, the acceleration in the t = 0 field. */
        for (int k = 0; k < 2; ++k) {
            species_t *sp = &s->sp[k];
            for (int64_t i = 0; i < sp->n; ++i)
                sp->abar[i] = s->d.q[k] / s->d.m[k] * gather(s, sp->xi[i]);
        }
    }
}

int64_t orc_sim_count(const orc_sim *s, int species) { return s->sp[species].n; }

void orc_sim_get(const orc_sim *s, int species, double *xi, double *vx, double *vy, double *vz,
                 uint32_t *id, double *abar, uint32_t *wait)
{
    const species_t *sp = &s->sp[species];
    for (int64_t i = 0; i < sp->n; ++i) {
        if (xi) xi[i] = sp->xi[i];
        if (vx) vx[i] = sp->vx[i];
        if (vy) vy[i] = sp->vy[i];
        if (vz) vz[i] = sp->vz[i];
        if (id) id[i] = sp->id[i];
        if (abar) abar[i] = sp->abar[i];
        if (wait) wait[i] = sp->wait[i];
    }
}

void orc_sim_set_step(orc_sim *s, int64_t step) { s->step = step; }

/* ------------------------------------------------------------------------- */
/* Monte Carlo collisions (Sec. 3: electron-atom and ion-atom collisions).    */
/* Null-collision selection with the bound probability P_null per step, by   */
/* waiting times (wait_tables): each step counts a particle's wait down; a    */
/* count that runs out selects it (or only draws a new wait, for a count      */
/* that stood for a wait beyond the longest one draw gives).  A selected      */
/* particle picks a process by comparing u * nu_max with the running sum of   */
/* n_g sigma_k(eps) v.                                                         */
/* ------------------------------------------------------------------------- */
/* Count down particle i of species k: 1 if it is selected in this step, else
   0; an expired count draws the next wait. */
static int selected(orc_sim *s, int k, int64_t i)
{
    species_t *sp = &s->sp[k];
    if ((k == 0 ? s->d.p_null_e : s->d.p_null_i) <= 0.0) return 0;
    uint32_t wv = sp->wait[i];
    if ((wv & ~WAIT_REDRAW) > 1u) {
        sp->wait[i] = wv - 1u;
        return 0;
    }
    sp->wait[i] = orc_wait_draw(&s->p, &s->d, k, sp->id[i], s->step, 0);
    return (wv & WAIT_REDRAW) ? 0 : 1;
}

static int collide_electron(orc_sim *s, int64_t i)
{
    const orc_params *p = &s->p;
    species_t *sp = &s->sp[0];
    if (!selected(s, 0, i)) return 0;
    uint32_t w[4];
    draw(p, sp->id[i], s->step, 0, TAG_MCC, 0, w);
    double v[3] = {sp->vx[i], sp->vy[i], sp->vz[i]};
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double g = sqrt(v2);
    double eps = 0.5 * M_E * v2 / Q_E;
    if (eps > p->eps_cap) s->dg.overflow[0] += 1;
    double r = uniform24(w[1]) * s->d.nu_max_e;
    double nu_el = p->gas_density * p->sig_el * g;
    double nu_ex = p->gas_density * sigma_exc(p, eps) * g;
    double nu_iz = p->gas_density * sigma_iz(p, eps) * g;
    const int vs = (p->coll_model & ORC_SCATTER_VS) != 0;
    double phi = 2.0 * PI_D * uniform24(w[3]);
    double d[3] = {1.0, 0.0, 0.0};
    if (g > 0.0) {
        d[0] = v[0] / g;
        d[1] = v[1] / g;
        d[2] = v[2] / g;
    }
    double g_new, cos_chi;
    if (r < nu_el) {
        /* elastic: energy loss fraction (2m/M)(1 - cos chi); the angle law is
           taken at the incident energy */
        cos_chi = vs ? orc_vs_cos_chi(eps, uniform24(w[2])) : 1.0 - 2.0 * uniform24(w[2]);
        g_new = g * sqrt(1.0 - 2.0 * M_E / s->d.m[1] * (1.0 - cos_chi));
        s->dg.coll[0] += 1;
    } else if (r < nu_el + nu_ex) {
        double e_out = eps - p->exc_thr;
        cos_chi = vs ? orc_vs_cos_chi(e_out, uniform24(w[2])) : 1.0 - 2.0 * uniform24(w[2]);
        g_new = sqrt(2.0 * Q_E * e_out / M_E);
        s->dg.coll[1] += 1;
    } else if (r < nu_el + nu_ex + nu_iz) {
        /* Reading: the excess eps - I is shared equally between the two
           electrons (or, with ORC_IZ_OPAL, the secondary takes the
           Opal-Pollock-Wagner share); each electron is scattered at the
           energy it leaves with; the new ion is drawn from the 300 K gas
           Maxwellian. */
        uint32_t w1[4], w2[4];
        draw(p, sp->id[i], s->step, 0, TAG_MCC, 1, w1);
        draw(p, sp->id[i], s->step, 0, TAG_MCC, 2, w2);
        double excess = eps - p->iz_thr;
        double e_sec = (p->coll_model & ORC_IZ_OPAL) ? orc_opal_secondary(excess, p->iz_split_b, uniform24(w2[2]))
                                                     : 0.5 * excess;
        double e_pri = (p->coll_model & ORC_IZ_OPAL) ? excess - e_sec : 0.5 * excess;
        cos_chi = vs ? orc_vs_cos_chi(e_pri, uniform24(w[2])) : 1.0 - 2.0 * uniform24(w[2]);
        g_new = sqrt(2.0 * Q_E * e_pri / M_E);
        double g_sec = sqrt(2.0 * Q_E * e_sec / M_E);
        double ps = 2.0 * PI_D * uniform24(w1[1]);
        double dc[3];
        if (vs) {
            /* the secondary turned from the incident direction by the law at its energy */
            orc_rotate(d, orc_vs_cos_chi(e_sec, uniform24(w1[0])), ps, dc);
        } else {
            /* isotropic in the laboratory frame */
            double ct = 1.0 - 2.0 * uniform24(w1[0]);
            double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            dc[0] = ct;
            dc[1] = st * cos(ps);
            dc[2] = st * sin(ps);
        }
        double n1, n2, n3, n4;
        box_muller(uniform24(w1[2]), uniform24(w1[3]), &n1, &n2);
        box_muller(uniform24(w2[0]), uniform24(w2[1]), &n3, &n4);
        if (s->n_births >= s->cap_births) return -1;
        birth_t *b = &s->births[s->n_births++];
        b->pid = sp->id[i];
        b->xi = sp->xi[i];
        b->ve[0] = g_sec * dc[0];
        b->ve[1] = g_sec * dc[1];
        b->ve[2] = g_sec * dc[2];
        b->vi[0] = s->d.vth_gas * n1;
        b->vi[1] = s->d.vth_gas * n2;
        b->vi[2] = s->d.vth_gas * n3;
        /* Reading: children of the implicit push inherit the parent's
           time-averaged field, abar for the electron and the same field times
           (q/m) of the ion for the ion (zero in the explicit schemes). */
        b->abar_e = sp->abar[i];
        b->abar_i = sp->abar[i] * (s->d.q[1] / s->d.m[1]) / (s->d.q[0] / s->d.m[0]);
        s->dg.coll[2] += 1;
    } else {
        s->dg.coll[4] += 1;
        return 0;
    }
    double dn[3];
    orc_rotate(d, cos_chi, phi, dn);
    sp->vx[i] = g_new * dn[0];
    sp->vy[i] = g_new * dn[1];
    sp->vz[i] = g_new * dn[2];
    return 1;
}

static void collide_ion(orc_sim *s, int64_t i)
{
    const orc_params *p = &s->p;
    species_t *sp = &s->sp[1];
    if (!selected(s, 1, i)) return;
    uint32_t w[4];
    draw(p, sp->id[i], s->step, 1, TAG_MCC, 0, w);
    uint32_t w1[4];
    draw(p, sp->id[i], s->step, 1, TAG_MCC, 1, w1);
    double n1, n2, n3, n4;
    box_muller(uniform24(w[2]), uniform24(w[3]), &n1, &n2);
    box_muller(uniform24(w1[0]), uniform24(w1[1]), &n3, &n4);
    double vn[3] = {s->d.vth_gas * n1, s->d.vth_gas * n2, s->d.vth_gas * n3};
    double dvx = sp->vx[i] - vn[0], dvy = sp->vy[i] - vn[1], dvz = sp->vz[i] - vn[2];
    double g = sqrt(dvx * dvx + dvy * dvy + dvz * dvz);
    if (g > s->d.g_max_i) s->dg.overflow[1] += 1;
    double r = uniform24(w[1]) * s->d.nu_max_i;
    if (r < p->gas_density * p->sig_cx * g) {
        /* charge exchange: the ion continues with the neutral's velocity */
        sp->vx[i] = vn[0];
        sp->vy[i] = vn[1];
        sp->vz[i] = vn[2];
        s->dg.coll[3] += 1;
    } else {
        s->dg.coll[4] += 1;
    }
}

static int cmp_birth(const void *a, const void *b)
{
    uint32_t x = ((const birth_t *)a)->pid, y = ((const birth_t *)b)->pid;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Remove absorbed particles (keeping order) and append this step's births:
   the children of parents taken in increasing parent id get consecutive ids. */
static int finish_population(orc_sim *s)
{
    for (int k = 0; k < 2; ++k) {
        species_t *sp = &s->sp[k];
        int64_t w = 0;
        for (int64_t i = 0; i < sp->n; ++i) {
            if (sp->dead[i]) continue;
            sp->xi[w] = sp->xi[i];
            sp->vx[w] = sp->vx[i];
            sp->vy[w] = sp->vy[i];
            sp->vz[w] = sp->vz[i];
            sp->abar[w] = sp->abar[i];
            sp->id[w] = sp->id[i];
            sp->wait[w] = sp->wait[i];
            sp->dead[w] = 0;
            ++w;
        }
        sp->n = w;
    }
    qsort(s->births, (size_t)s->n_births, sizeof(birth_t), cmp_birth);
    for (int64_t b = 0; b < s->n_births; ++b) {
        const birth_t *bb = &s->births[b];
        for (int k = 0; k < 2; ++k) {
            species_t *sp = &s->sp[k];
            if (sp->n >= sp->cap) return -1;
            int64_t i = sp->n++;
            sp->xi[i] = bb->xi;
            const double *v = k == 0 ? bb->ve : bb->vi;
            sp->vx[i] = v[0];
            sp->vy[i] = v[1];
            sp->vz[i] = v[2];
            sp->abar[i] = k == 0 ? bb->abar_e : bb->abar_i;
            sp->id[i] = sp->next_id + (uint32_t)b;
            /* a child's first wait is drawn on its birth step */
            sp->wait[i] = orc_wait_draw(&s->p, &s->d, k, sp->id[i], s->step, 1);
            sp->dead[i] = 0;
        }
    }
    s->sp[0].next_id += (uint32_t)s->n_births;
    s->sp[1].next_id += (uint32_t)s->n_births;
    s->dg.births += s->n_births;
    return 0;
}

/* Electrode absorption (Sec. 3, "plasma eliminator") or periodic wrap. */
static void boundary(orc_sim *s, int k, int64_t i)
{
    const orc_params *p = &s->p;
    species_t *sp = &s->sp[k];
    double n = (double)p->n_cells;
    if (p->periodic) {
        sp->xi[i] -= n * floor(sp->xi[i] / n);
        if (sp->xi[i] >= n) sp->xi[i] -= n;
        return;
    }
    if (sp->xi[i] < 0.0 || sp->xi[i] >= n) {
        int wall = sp->xi[i] < 0.0 ? 0 : 1;
        double v2 = sp->vx[i] * sp->vx[i] + sp->vy[i] * sp->vy[i] + sp->vz[i] * sp->vz[i];
        sp->dead[i] = 1;
        s->dg.wall_count[k][wall] += 1;
        s->dg.wall_energy_ev[k][wall] += 0.5 * s->d.m[k] * v2 / Q_E;
    }
}

static void sample_eedf(orc_sim *s)
{
    const orc_params *p = &s->p;
    if (p->eedf_bins <= 0) return;
    species_t *sp = &s->sp[0];
    double width = p->eedf_max_ev / p->eedf_bins;
    for (int64_t i = 0; i < sp->n; ++i) {
        double v2 = sp->vx[i] * sp->vx[i] + sp->vy[i] * sp->vy[i] + sp->vz[i] * sp->vz[i];
        double eps = 0.5 * M_E * v2 / Q_E;
        int64_t bin = (int64_t)floor(eps / width);
        if (bin > p->eedf_bins) bin = p->eedf_bins;
        s->eedf[bin] += 1;
    }
}

/* Collisions for all survivors, then removal and births. */
static int collisions_and_population(orc_sim *s)
{
    s->n_births = 0;
    if (s->p.mcc) {
        for (int64_t i = 0; i < s->sp[0].n; ++i) {
            if (s->sp[0].dead[i]) continue;
            if (collide_electron(s, i) < 0) return -1;
        }
        if (s->p.ions_mobile)
            for (int64_t i = 0; i < s->sp[1].n; ++i)
                if (!s->sp[1].dead[i]) collide_ion(s, i);
    }
    return finish_population(s);
}

/* The cell coordinate after a move by d metres on the non-uniform grid:
   through the physical position, wrapped in a periodic box; a position
   beyond an electrode comes back outside [0, N) for the absorption. */
static double move_on_grid(const orc_sim *s, double xi, double d)
{
    int64_t n = s->p.n_cells, c = (int64_t)floor(xi);
    double len = s->xn[n];
    double x = s->xn[c] + (xi - (double)c) * s->h[c] + d;
    if (s->p.periodic) {
        x -= len * floor(x / len);
        if (x >= len) x -= len;
    }
    int64_t cell;
    double off;
    int where = orc_locate((int)n, s->xn, s->h, x, &cell, &off);
    if (where < 0) return -0.5;
    if (where > 0) return (double)n + 0.5;
    return (double)cell + off;
}

/* One explicit step n -> n+1 (Sec. 2 schemes (1) and (2)): gather E^n at x^n,
   leapfrog v^{n-1/2} -> v^{n+1/2}, x^n -> x^{n+1}, absorb, collide, assign
   charge at x^{n+1} and solve for E^{n+1} with the electrode at V(t_{n+1}). */
static int step_explicit(orc_sim *s, int diag_step)
{
    const orc_params *p = &s->p;
    double dx = s->d.dx;
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && !p->ions_mobile) continue;
        species_t *sp = &s->sp[k];
        double qm = s->d.q[k] / s->d.m[k];
        double kx = 0.0, pw = 0.0;
        for (int64_t i = 0; i < sp->n; ++i) {
            double e = gather(s, sp->xi[i]);
            double v_old = sp->vx[i];
            double v_new = v_old + qm * e * p->dt;
            kx += 0.5 * (v_old * v_old + v_new * v_new);
            double work = s->d.q[k] * s->d.weight * e * 0.5 * (v_old + v_new);
            pw += work;
            int64_t c = (int64_t)floor(sp->xi[i]);
            if (diag_step) s->heat[k][c] += work / (s->h ? s->h[c] : dx);
            sp->vx[i] = v_new;
            if (s->h)
                sp->xi[i] = move_on_grid(s, sp->xi[i], v_new * p->dt);
            else
                sp->xi[i] += v_new * p->dt / dx;
            boundary(s, k, i);
        }
        s->dg.ke_x[k] = 0.5 * s->d.m[k] * s->d.weight * kx;
        s->dg.power[k] = pw;
    }
    s->dg.field_energy_push = s->dg.field_energy;
    if (collisions_and_population(s)) return -1;
    deposit_and_solve(s, s->step + 1);
    return 0;
}

/* One direct-implicit step (Sec. 2 schemes (4) and, with S_1 weighting and
   node fields, (3)) in the D1 form of Cohen,
   Langdon & Friedman: predictor v~ = v^{n-1/2} + dt abar^{n-1}/2, x~ = x^n +
   dt v~; charge and susceptibility assigned at x~; modified Poisson equation
   for E^{n+1}; corrector a = (q/m) E^{n+1}(x~), x^{n+1} = x~ + dt^2 a / 2,
   v^{n+1/2} = v~ + dt a / 2, abar^n = (abar^{n-1} + a) / 2.
   Reading: a predicted position beyond an electrode is assigned nowhere and
   sees no field, so the corrector leaves it outside and it is absorbed. */
static int step_implicit(orc_sim *s, int diag_step)
{
    const orc_params *p = &s->p;
    double dx = s->d.dx, dt = p->dt;
    int64_t nn = p->n_cells + 1;
    int n = p->n_cells;
    /* pass 1: predictor and assignment at x~ */
    for (int k = 0; k < 2; ++k) {
        species_t *sp = &s->sp[k];
        double *xt = (double *)malloc(sizeof(double) * (size_t)(sp->n > 0 ? sp->n : 1));
        int64_t m = 0;
        for (int64_t i = 0; i < sp->n; ++i) {
            double vt = sp->vx[i] + 0.5 * dt * sp->abar[i];
            double x;
            if (s->h) {
                x = move_on_grid(s, sp->xi[i], vt * dt);  /* wraps in the periodic box */
                if (x < 0.0 || x >= n) continue;
            } else {
                x = sp->xi[i] + vt * dt / dx;
                if (p->periodic) {
                    x -= n * floor(x / n);
                    if (x >= n) x -= n;
                } else if (x < 0.0 || x >= n) {
                    continue;
                }
            }
            xt[m++] = x;
        }
        if (is_mc(p)) {
            orc_deposit_s1_fixed(p, m, xt, s->rho_q[k]);
        } else {
            if (p->quantized)
                orc_deposit_s2_fixed(p, m, xt, s->rho_q[k]);
            else
                orc_deposit_s2_fp64(p, m, xt, s->rho_f[k]);
            deposit_chi_fixed(p, m, xt, s->chi_q[k]);
        }
        free(xt);
    }
    assemble_rho(s);
    /* EC: chi_{c+1/2} = dt^2/2 sum_s (q_s^2 w / (m_s eps0 dx)) S_1-weighted count at
       the cell centres (on a non-uniform grid the count over the cell's own
       width h_c: a density, as on the uniform grid).  MC (reading): the same
       density-like sum at the nodes with the S_1 weights of the charge
       assignment, averaged onto each face. */
    for (int c = 0; c < n; ++c) {
        double chi = 0.0;
        for (int k = 0; k < 2; ++k) {
            double coef = 0.5 * dt * dt * s->d.q[k] * s->d.q[k] * s->d.weight /
                          (s->d.m[k] * EPS_0 * (s->h ? s->h[c] : dx));
            if (is_mc(p)) {
                int64_t right = (p->periodic && c + 1 == n) ? 0 : c + 1;
                double wl = (double)s->rho_q[k][c] / (double)TWO_POW_33;
                double wr = (double)s->rho_q[k][right] / (double)TWO_POW_33;
                chi += coef * 0.5 * (wl + wr);
            } else {
                chi += coef * (double)s->chi_q[k][c] / 65536.0;
            }
        }
        s->chi[c] = chi;
    }
    (void)nn;
    solve_field(s, s->chi, s->step + 1);
    s->dg.field_energy_push = s->dg.field_energy;
    /* pass 2: corrector at x~ */
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && !p->ions_mobile) continue;
        species_t *sp = &s->sp[k];
        double qm = s->d.q[k] / s->d.m[k];
        double kx = 0.0, pw = 0.0;
        for (int64_t i = 0; i < sp->n; ++i) {
            double v_old = sp->vx[i];
            double vt = v_old + 0.5 * dt * sp->abar[i];
            double x;
            if (s->h) {
                x = move_on_grid(s, sp->xi[i], vt * dt);
            } else {
                x = sp->xi[i] + vt * dt / dx;
                if (p->periodic) {
                    x -= n * floor(x / n);
                    if (x >= n) x -= n;
                }
            }
            int inside = x >= 0.0 && x < n;
            double e = inside ? gather(s, x) : 0.0;
            double a = qm * e;
            double v_new = vt + 0.5 * dt * a;
            double abar_new = 0.5 * (sp->abar[i] + a);
            kx += 0.5 * (v_old * v_old + v_new * v_new);
            /* Reading: the step changes v by dt abar^n, so the work done on the
               particle is m w abar^n vbar (the field (m/q) abar^n, not E^{n+1}) */
            double work = s->d.m[k] * s->d.weight * abar_new * 0.5 * (v_old + v_new);
            pw += work;
            if (diag_step && inside) {
                int64_t c = (int64_t)floor(x);
                s->heat[k][c] += work / (s->h ? s->h[c] : dx);
            }
            if (s->h)
                sp->xi[i] = inside ? move_on_grid(s, x, 0.5 * dt * dt * a) : x;
            else
                sp->xi[i] = x + 0.5 * dt * dt * a / dx;
            sp->vx[i] = v_new;
            sp->abar[i] = abar_new;
            boundary(s, k, i);
        }
        s->dg.ke_x[k] = 0.5 * s->d.m[k] * s->d.weight * kx;
        s->dg.power[k] = pw;
    }
    return collisions_and_population(s);
}

int orc_sim_step(orc_sim *s, int64_t nsteps)
{
    for (int64_t t = 0; t < nsteps; ++t) {
        int diag_step = s->p.diag_period > 0 && (s->step % s->p.diag_period) == 0;
        int r = is_implicit(&s->p) ? step_implicit(s, diag_step) : step_explicit(s, diag_step);
        if (r) return r;
        accumulate_averages(s);
        if (diag_step) {
            sample_eedf(s);
            s->dg.n_diag += 1;
        }
        s->step += 1;
    }
    return 0;
}

void orc_sim_diag(const orc_sim *s, orc_diag *d)
{
    *d = s->dg;
    for (int k = 0; k < 2; ++k) {
        const species_t *sp = &s->sp[k];
        d->count[k] = sp->n;
        double perp = 0.0;
        for (int64_t i = 0; i < sp->n; ++i) perp += sp->vy[i] * sp->vy[i] + sp->vz[i] * sp->vz[i];
        d->ke_perp[k] = 0.5 * s->d.m[k] * s->d.weight * perp;
    }
    d->step = s->step;
}

void orc_sim_grids(const orc_sim *s, int64_t *rho_q_e, int64_t *rho_q_i, double *phi,
                   double *e_cc, double *chi)
{
    int64_t nn = s->p.n_cells + 1;
    for (int64_t g = 0; g < nn; ++g) {
        if (rho_q_e) rho_q_e[g] = s->rho_q[0][g];
        if (rho_q_i) rho_q_i[g] = s->rho_q[1][g];
        if (phi) phi[g] = s->phi[g];
    }
    for (int64_t c = 0; c < s->p.n_cells; ++c) {
        if (e_cc) e_cc[c] = s->e_cc[c];
        if (chi) chi[c] = s->chi[c];
    }
}

void orc_sim_averages(const orc_sim *s, double *ne, double *ni, double *phi, double *heat_e,
                      double *heat_i, int64_t *eedf)
{
    int64_t nn = s->p.n_cells + 1;
    double na = s->dg.n_avg > 0 ? (double)s->dg.n_avg : 1.0;
    double nd = s->dg.n_diag > 0 ? (double)s->dg.n_diag : 1.0;
    for (int64_t g = 0; g < nn; ++g) {
        if (ne) ne[g] = s->avg_ne[g] / na;
        if (ni) ni[g] = s->avg_ni[g] / na;
        if (phi) phi[g] = s->avg_phi[g] / na;
    }
    for (int64_t c = 0; c < s->p.n_cells; ++c) {
        if (heat_e) heat_e[c] = s->heat[0][c] / nd;
        if (heat_i) heat_i[c] = s->heat[1][c] / nd;
    }
    if (eedf)
        for (int b = 0; b <= s->p.eedf_bins; ++b) eedf[b] = s->eedf[b];
}

void orc_sim_reset_averages(orc_sim *s)
{
    int64_t nn = s->p.n_cells + 1;
    memset(s->avg_ne, 0, sizeof(double) * (size_t)nn);
    memset(s->avg_ni, 0, sizeof(double) * (size_t)nn);
    memset(s->avg_phi, 0, sizeof(double) * (size_t)nn);
    memset(s->heat[0], 0, sizeof(double) * (size_t)nn);
    memset(s->heat[1], 0, sizeof(double) * (size_t)nn);
    memset(s->eedf, 0, sizeof(int64_t) * (size_t)(s->p.eedf_bins + 1));
    s->dg.n_avg = 0;
    s->dg.n_diag = 0;
}
