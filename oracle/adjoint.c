/*
 * adjoint.c -- FP64 oracle of the collisionless energy-conserving explicit
 * step and of its discrete adjoint (reverse-mode derivative).
 *
 * TEST INFRASTRUCTURE ONLY (as the rest of oracle/): nothing in the product
 * library includes, links or calls this file.
 *
 * The forward model is the EC explicit scheme of Sec. 2 (scheme (2)): charge
 * assignment by the quadratic spline S_2 to the nodes (Eq. 2), the
 * finite-difference Poisson equation with the RF electrode (Sec. 3) or a
 * periodic box, cell-centred fields E_{c+1/2} = (phi_c - phi_{c+1})/dx and
 * force interpolation by S_1 from the cell centres (Eq. 3), leapfrog push.
 * Electrons move on a frozen uniform ion background; there are no
 * collisions.  A particle that leaves [0, L) between electrodes is absorbed
 * and takes no further part (its absorption step is an event that the
 * derivative holds fixed).
 *
 * Objectives, time averages over the K steps n = 0..K-1 (step n pushes from
 * time level n to n+1 with the field of level n, V(t_n) on the electrode):
 *   P^n     = sum_p q w E_p^n vbar_p^n               (power absorbed by the electrons)
 *   Gamma^n = sum_p w vbar_p^n S_1(xi_p^n - 1/2)/dx  (electron current density at the
 *                                                     centre of the first cell)
 * with vbar = (v^{n-1/2} + v^{n+1/2})/2, and J = c_P <P> + c_G <Gamma>.
 *
 * The adjoint follows the forward in reverse, one step at a time, with the
 * plain textbook transposes: the adjoint of the push, a scatter of the force
 * sensitivity to the cell centres (transpose of the S_1 gather), the
 * transpose of the difference E = -dphi/dx, the symmetric Poisson matrix
 * solved again by the Thomas algorithm (homogeneous boundary values), and the
 * derivative of the S_2 assignment.  The whole trajectory is kept in memory
 * (no checkpointing: the oracle is meant for small cases).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define Q_E   1.602176634e-19
#define M_E   9.1093837015e-31
#define EPS_0 8.8541878128e-12
#define PI_D  3.14159265358979323846

/* Quadratic B-spline S_2(u) and its derivative. */
static double s2(double u)
{
    double a = fabs(u);
    if (a <= 0.5) return 0.75 - u * u;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

static double s2_prime(double u)
{
    double a = fabs(u);
    if (a <= 0.5) return -2.0 * u;
    if (a < 1.5) return (u > 0.0 ? -1.0 : 1.0) * (1.5 - a);
    return 0.0;
}

/* Linear B-spline S_1(u) and its derivative (one-sided at the kinks). */
static double s1(double u)
{
    double a = fabs(u);
    return a < 1.0 ? 1.0 - a : 0.0;
}

static double s1_prime(double u)
{
    if (fabs(u) >= 1.0) return 0.0;
    return u >= 0.0 ? -1.0 : 1.0;
}

/* Node index of a stencil node: ghost nodes fold onto the wall node between
   electrodes, wrap in the periodic box. */
static int64_t fold_node(const orc_adj_problem *pb, int64_t g)
{
    int64_t n = pb->n_cells;
    if (pb->periodic) return ((g % n) + n) % n;
    if (g < 0) return 0;
    if (g > n) return n;
    return g;
}

/* Cell index of a stencil cell, or -1 for a ghost cell beyond an electrode
   (which holds E = 0). */
static int64_t wrap_cell(const orc_adj_problem *pb, int64_t c)
{
    int64_t n = pb->n_cells;
    if (pb->periodic) return ((c % n) + n) % n;
    if (c < 0 || c >= n) return -1;
    return c;
}

static double rf_level(const orc_adj_problem *pb, int64_t level, double volt)
{
    if (pb->periodic) return 0.0;
    return volt * sin(2.0 * PI_D * pb->rf_freq * (double)level * pb->dt);
}

/* S_1 weight of the first cell's centre (xi = 1/2) for the current estimator,
   with the periodic image. */
static double flux_weight(const orc_adj_problem *pb, double xi, double *deriv)
{
    double u = xi - 0.5;
    double w = s1(u), d = s1_prime(u);
    if (pb->periodic) {
        double u2 = xi - 0.5 - (double)pb->n_cells;
        w += s1(u2);
        d += s1_prime(u2);
    }
    if (deriv) *deriv = d;
    return w;
}

/* Charge density at the nodes (Eq. 2): electrons by S_2, frozen ions. */
static void charge(const orc_adj_problem *pb, int64_t np, const double *xi, const char *alive,
                   double *rho)
{
    int64_t n = pb->n_cells;
    double dx = pb->length / (double)n;
    for (int64_t g = 0; g <= n; ++g) rho[g] = Q_E * pb->bg_density;
    for (int64_t p = 0; p < np; ++p) {
        if (!alive[p]) continue;
        int64_t j = (int64_t)floor(xi[p] + 0.5);
        for (int64_t g = j - 1; g <= j + 1; ++g)
            rho[fold_node(pb, g)] -= Q_E * pb->weight / dx * s2(xi[p] - (double)g);
    }
    if (pb->periodic) rho[n] = rho[0];
}

/* Field of one time level: potential by the tridiagonal solve, cell-centred E. */
static void field(const orc_adj_problem *pb, const double *rho, double v_left, double *phi, double *e)
{
    int n = pb->n_cells;
    double dx = pb->length / (double)n;
    if (pb->periodic)
        orc_solve_periodic(n, dx, rho, NULL, phi);
    else
        orc_solve_dirichlet(n, dx, rho, NULL, v_left, phi);
    for (int c = 0; c < n; ++c) {
        double right = (pb->periodic && c + 1 == n) ? phi[0] : phi[c + 1];
        e[c] = (phi[c] - right) / dx;
    }
}

/* E at a particle (Eq. 3 with m = 2) and its derivative in xi. */
static double gather(const orc_adj_problem *pb, const double *e, double xi, double *de_dxi)
{
    int64_t j = (int64_t)floor(xi + 0.5);
    double val = 0.0, der = 0.0;
    for (int64_t c = j - 1; c <= j; ++c) {
        int64_t cc = wrap_cell(pb, c);
        double ec = cc < 0 ? 0.0 : e[cc];
        double u = xi - ((double)c + 0.5);
        val += s1(u) * ec;
        der += s1_prime(u) * ec;
    }
    if (de_dxi) *de_dxi = der;
    return val;
}

typedef struct traj {
    int64_t np, K;
    double *xi;    /* [K+1][np] positions in cell units */
    double *v;     /* [K+1][np] v^{n-1/2} at row n */
    char *alive;   /* [K+1][np] */
    double *e;     /* [K][n_cells] field of level n */
} traj;

static void traj_free(traj *t)
{
    free(t->xi);
    free(t->v);
    free(t->alive);
    free(t->e);
}

/* Forward run; fills the objectives and, when t is given, the trajectory. */
static int run_forward(const orc_adj_problem *pb, double volt, int64_t np, const double *xi0,
                       const double *vx0, double *p_avg, double *g_avg, traj *t, double *xi_end,
                       double *v_end, int64_t *absorbed_at)
{
    int64_t n = pb->n_cells, K = pb->nsteps;
    double dx = pb->length / (double)n;
    double q = -Q_E, qm = -Q_E / M_E, w = pb->weight;
    double *xi = malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    double *v = malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    char *alive = malloc((size_t)(np > 0 ? np : 1));
    double *rho = malloc(sizeof(double) * (size_t)(n + 1));
    double *phi = malloc(sizeof(double) * (size_t)(n + 1));
    double *e = malloc(sizeof(double) * (size_t)n);
    if (!xi || !v || !alive || !rho || !phi || !e) return -1;
    memcpy(xi, xi0, sizeof(double) * (size_t)np);
    memcpy(v, vx0, sizeof(double) * (size_t)np);
    for (int64_t p = 0; p < np; ++p) {
        alive[p] = 1;
        if (absorbed_at) absorbed_at[p] = -1;
    }
    double psum = 0.0, gsum = 0.0;
    for (int64_t s = 0; s < K; ++s) {
        if (t) {
            memcpy(t->xi + s * np, xi, sizeof(double) * (size_t)np);
            memcpy(t->v + s * np, v, sizeof(double) * (size_t)np);
            memcpy(t->alive + s * np, alive, (size_t)np);
        }
        charge(pb, np, xi, alive, rho);
        field(pb, rho, rf_level(pb, pb->step0 + s, volt), phi, e);
        if (t) memcpy(t->e + s * n, e, sizeof(double) * (size_t)n);
        for (int64_t p = 0; p < np; ++p) {
            if (!alive[p]) continue;
            double ep = gather(pb, e, xi[p], NULL);
            double v_new = v[p] + qm * ep * pb->dt;
            double vbar = 0.5 * (v[p] + v_new);
            psum += q * w * ep * vbar;
            gsum += w * vbar * flux_weight(pb, xi[p], NULL) / dx;
            v[p] = v_new;
            xi[p] += v_new * pb->dt / dx;
            if (pb->periodic) {
                xi[p] = fmod(xi[p], (double)n);
                if (xi[p] < 0.0) xi[p] += (double)n;
            } else if (xi[p] < 0.0 || xi[p] >= (double)n) {
                alive[p] = 0;
                if (absorbed_at) absorbed_at[p] = s;
            }
        }
    }
    if (t) {
        memcpy(t->xi + K * np, xi, sizeof(double) * (size_t)np);
        memcpy(t->v + K * np, v, sizeof(double) * (size_t)np);
        memcpy(t->alive + K * np, alive, (size_t)np);
    }
    if (p_avg) *p_avg = K > 0 ? psum / (double)K : 0.0;
    if (g_avg) *g_avg = K > 0 ? gsum / (double)K : 0.0;
    if (xi_end) memcpy(xi_end, xi, sizeof(double) * (size_t)np);
    if (v_end) memcpy(v_end, v, sizeof(double) * (size_t)np);
    free(xi);
    free(v);
    free(alive);
    free(rho);
    free(phi);
    free(e);
    return 0;
}

int orc_adj_forward(const orc_adj_problem *pb, int64_t np, const double *xi0, const double *vx0,
                    double *power_avg, double *flux_avg, double *xi_end, double *vx_end,
                    int64_t *absorbed_at)
{
    if (!pb || pb->n_cells < 2 || pb->nsteps < 0 || np < 0) return -1;
    return run_forward(pb, pb->rf_volt, np, xi0, vx0, power_avg, flux_avg, NULL, xi_end, vx_end,
                       absorbed_at);
}

int orc_adj_gradient(const orc_adj_problem *pb, int64_t np, const double *xi0, const double *vx0,
                     double *j_out, double *dj_dvx0, double *dj_dxi0, double *dj_dv0)
{
    if (!pb || pb->n_cells < 2 || pb->nsteps < 0 || np < 0) return -1;
    int64_t n = pb->n_cells, K = pb->nsteps;
    double dx = pb->length / (double)n;
    double q = -Q_E, qm = -Q_E / M_E, w = pb->weight, dt = pb->dt;
    double cp = pb->c_power / (double)(K > 0 ? K : 1), cg = pb->c_flux / (double)(K > 0 ? K : 1);
    traj t;
    t.np = np;
    t.K = K;
    size_t rows = (size_t)(K + 1) * (size_t)(np > 0 ? np : 1);
    t.xi = malloc(sizeof(double) * rows);
    t.v = malloc(sizeof(double) * rows);
    t.alive = malloc(rows);
    t.e = malloc(sizeof(double) * (size_t)(K > 0 ? K : 1) * (size_t)n);
    double pa, ga;
    if (!t.xi || !t.v || !t.alive || !t.e ||
        run_forward(pb, pb->rf_volt, np, xi0, vx0, &pa, &ga, &t, NULL, NULL, NULL)) {
        traj_free(&t);
        return -1;
    }
    if (j_out) *j_out = pb->c_power * pa + pb->c_flux * ga;

    /* lx: adjoint of x (SI metres) at level n+1; lv: adjoint of v^{n+1/2} */
    double *lx = calloc((size_t)(np > 0 ? np : 1), sizeof(double));
    double *lv = calloc((size_t)(np > 0 ? np : 1), sizeof(double));
    double *lx_new = calloc((size_t)(np > 0 ? np : 1), sizeof(double));
    double *le = malloc(sizeof(double) * (size_t)n);        /* adjoint of E_c */
    double *lphi = malloc(sizeof(double) * (size_t)(n + 1)); /* adjoint of phi_g */
    double *mu = malloc(sizeof(double) * (size_t)(n + 1));
    double *lrho = malloc(sizeof(double) * (size_t)(n + 1));
    double *tmp = malloc(sizeof(double) * (size_t)(n + 1));
    double dv0 = 0.0;
    for (int64_t s = K - 1; s >= 0; --s) {
        const double *xi = t.xi + s * np, *vm = t.v + s * np, *vp = t.v + (s + 1) * np;
        const char *al = t.alive + s * np;
        const double *e = t.e + s * n;
        memset(le, 0, sizeof(double) * (size_t)n);
        for (int64_t p = 0; p < np; ++p) {
            lx_new[p] = 0.0;
            if (!al[p]) continue;
            double de_dxi, dfl;
            double ep = gather(pb, e, xi[p], &de_dxi);
            double fl = flux_weight(pb, xi[p], &dfl);
            double vbar = 0.5 * (vm[p] + vp[p]);
            /* direct partials of this step's objective terms */
            double dj_dv = cp * q * w * ep * 0.5 + cg * w * fl / dx * 0.5;  /* d/dv^{n+1/2} = d/dv^{n-1/2} */
            double dj_dep = cp * q * w * vbar;
            double dj_dxi = cg * w * vbar * dfl / dx;
            /* x^{n+1} = x^n + dt v^{n+1/2} */
            double lvp = lv[p] + dt * lx[p] + dj_dv;
            /* v^{n+1/2} = v^{n-1/2} + dt qm E_p */
            double lep = dt * qm * lvp + dj_dep;
            lv[p] = lvp + dj_dv;
            lx_new[p] = lx[p] + lep * de_dxi / dx + dj_dxi / dx;
            /* transpose of the S_1 gather: scatter to the cell centres */
            int64_t j = (int64_t)floor(xi[p] + 0.5);
            for (int64_t c = j - 1; c <= j; ++c) {
                int64_t cc = wrap_cell(pb, c);
                if (cc >= 0) le[cc] += lep * s1(xi[p] - ((double)c + 0.5));
            }
        }
        /* transpose of E_c = (phi_c - phi_{c+1})/dx */
        for (int64_t g = 0; g <= n; ++g) lphi[g] = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            int64_t right = (pb->periodic && c + 1 == n) ? 0 : c + 1;
            lphi[c] += le[c] / dx;
            lphi[right] -= le[c] / dx;
        }
        /* transpose of the Poisson solve: the matrix is symmetric, so the same
           Thomas solve with homogeneous boundary values; rho = lphi eps0/dx^2
           makes the routine return T^-1 lphi. */
        for (int64_t g = 0; g <= n; ++g) tmp[g] = lphi[g] * EPS_0 / (dx * dx);
        if (pb->periodic) {
            tmp[n] = 0.0;
            orc_solve_periodic((int)n, dx, tmp, NULL, mu);
            double mean = 0.0;
            for (int64_t g = 0; g < n; ++g) mean += mu[g];
            mean /= (double)n;
            for (int64_t g = 0; g < n; ++g) lrho[g] = (mu[g] - mean) * dx * dx / EPS_0;
            lrho[n] = lrho[0];
        } else {
            orc_solve_dirichlet((int)n, dx, tmp, NULL, 0.0, mu);
            for (int64_t g = 1; g < n; ++g) lrho[g] = mu[g] * dx * dx / EPS_0;
            lrho[0] = lrho[n] = 0.0;  /* wall-node charge does not enter the solve */
            /* phi_0 = V(t_n): directly, and through the first interior equation */
            double dj_dphi0 = lphi[0] + mu[1];
            dv0 += dj_dphi0 * sin(2.0 * PI_D * pb->rf_freq * (double)(pb->step0 + s) * dt);
        }
        /* derivative of the S_2 assignment */
        for (int64_t p = 0; p < np; ++p) {
            if (!al[p]) {
                lx[p] = 0.0;
                lv[p] = 0.0;
                continue;
            }
            int64_t j = (int64_t)floor(xi[p] + 0.5);
            double acc = 0.0;
            for (int64_t g = j - 1; g <= j + 1; ++g)
                acc += lrho[fold_node(pb, g)] * (-Q_E * w / dx) * s2_prime(xi[p] - (double)g);
            lx[p] = lx_new[p] + acc / dx;
        }
    }
    for (int64_t p = 0; p < np; ++p) {
        if (dj_dvx0) dj_dvx0[p] = lv[p];
        if (dj_dxi0) dj_dxi0[p] = lx[p] * dx;
    }
    if (dj_dv0) *dj_dv0 = dv0;
    free(lx);
    free(lv);
    free(lx_new);
    free(le);
    free(lphi);
    free(mu);
    free(lrho);
    free(tmp);
    traj_free(&t);
    return 0;
}
