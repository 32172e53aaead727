// pic_capi.cu -- host runtime of libpic.so: configuration checks, layout of
// the caller-owned arena, derived constants, launch sequencing and CUDA-graph
// replay of whole sort cycles.  Implements include/pic.h.
#include "pic.h"
#include "pic_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pic;

namespace {

// CODATA 2018.
constexpr double kE = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kKb = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kEulerN = 2.71828182845904523536;
constexpr double kTorrPa = 101325.0 / 760.0;

thread_local std::string g_error;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(const pic_config &c) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t n1 = (size_t)c.n_cells + 1;
    L.state = take(sizeof(DevState));
    for (int p = 0; p < 2; ++p)
        for (int s = 0; s < 2; ++s) {
            const size_t cap = (size_t)c.capacity[s];
            for (int f = 0; f < 6; ++f) L.sp[p][s][f] = take(4 * cap);
            L.sp[p][s][6] = implicit_scheme(c) ? take(4 * cap) : 0;
        }
    for (int s = 0; s < 2; ++s) {
        L.acc_cnt[s] = take(8 * n1);
        L.acc_a[s] = take(8 * n1);
        L.acc_b[s] = take(8 * n1);
        L.acc_c[s] = take(8 * n1);
        L.cursor[s] = take(4 * n1);
        L.rho_q[s] = take(8 * n1);
    }
    L.e_gather = take(4 * (n1 + 1));
    L.e_hi = take(4 * n1);
    L.e_lo = take(4 * n1);
    L.e_cc = take(8 * n1);
    L.chi = take(8 * n1);
    L.avg_ne = take(8 * n1);
    L.avg_ni = take(8 * n1);
    L.avg_e = take(8 * n1);
    L.heat[0] = take(8 * n1);
    L.heat[1] = take(8 * n1);
    L.eedf = take(8 * ((size_t)c.eedf_bins + 1));
    const size_t nb = (size_t)(c.births_capacity > 0 ? c.births_capacity : 1);
    L.births = take(sizeof(Birth) * nb + 8 * nb);  // records + rank and sort scratch
    L.wait_tab = take(4 * 2 * 3 * 64);
    L.hw = L.h64 = L.xnode = L.hdw = L.wdw = 0;
    if (c.cell_width) {
        const size_t n = (size_t)c.n_cells;
        L.hw = take(8 * n);
        L.h64 = take(8 * n);
        L.xnode = take(8 * n1);
        L.hdw = take(8 * n);
        L.wdw = take(8 * n);
    }
    L.total = o;
    return L;
}

double gas_density(const pic_config &c) {
    return c.pressure_mtorr * 1e-3 * kTorrPa / (kKb * c.gas_temp);
}

double sig_exc(const pic_config &c, double eps) {
    if (eps < c.exc_thr) return 0.0;
    if (eps < c.exc_ramp_end) return c.sig_exc_max * (eps - c.exc_thr) / (c.exc_ramp_end - c.exc_thr);
    return c.sig_exc_max;
}

double sig_iz(const pic_config &c, double eps) {
    if (eps <= c.iz_thr) return 0.0;
    return c.sig_iz_peak * kEulerN * (c.iz_thr / eps) * std::log(eps / c.iz_thr);
}

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int validate(const pic_config *c) {
    if (!c) return fail(PIC_EINVAL, "config is NULL");
    if (c->scheme < 0 || c->scheme > 4) return fail(PIC_EINVAL, "unknown scheme %d", c->scheme);
    if (c->boundary != PIC_BC_ELECTRODES && c->boundary != PIC_BC_PERIODIC)
        return fail(PIC_EINVAL, "unknown boundary %d", c->boundary);
    if (c->n_cells < 2 || c->n_cells > kMaxCells)
        return fail(PIC_EINVAL, "n_cells %d outside 2..%d", c->n_cells, kMaxCells);
    if (!(c->length > 0) || !(c->dt > 0)) return fail(PIC_EINVAL, "length and dt must be positive");
    if (c->np_init < 1) return fail(PIC_EINVAL, "np_init must be >= 1 (it sets the macro weight)");
    if (!(c->n0 > 0)) return fail(PIC_EINVAL, "n0 must be positive");
    for (int s = 0; s < 2; ++s) {
        if (c->capacity[s] < 1 || c->capacity[s] >= (1ll << 29))
            return fail(PIC_EOVERFLOW, "capacity[%d] = %lld outside 1..2^29-1 (int64 charge headroom)",
                        s, (long long)c->capacity[s]);
        if (c->capacity[s] < c->np_init && (s == 0 || c->ions_mobile))
            return fail(PIC_EINVAL, "capacity[%d] below np_init", s);
        // m = 3 charges are 6 * 2^36 a particle: |prefix sums| < 2^23 * 6 * 2^36 < 2^62
        if (c->scheme == PIC_EC3_EXPLICIT && c->capacity[s] >= (1ll << 23))
            return fail(PIC_EOVERFLOW, "capacity[%d] = %lld: the m = 3 scheme takes below 2^23 (int64 charge headroom)",
                        s, (long long)c->capacity[s]);
    }
    if (c->mcc && !c->ions_mobile) return fail(PIC_EINVAL, "collisions need mobile ions");
    if (c->mcc && c->births_capacity < 1) return fail(PIC_EINVAL, "births_capacity must be >= 1");
    if (c->births_capacity < 0 || c->births_capacity > (1ll << 24))
        return fail(PIC_EINVAL, "births_capacity outside 0..2^24");
    if (c->eedf_bins < 1 || c->eedf_bins > 1024) return fail(PIC_EINVAL, "eedf_bins outside 1..1024");
    if (c->collision_model & ~(PIC_IZ_OPAL | PIC_SCATTER_VS)) return fail(PIC_EINVAL, "unknown collision_model bits");
    if ((c->collision_model & PIC_IZ_OPAL) && !(c->iz_split_b > 0.0))
        return fail(PIC_EINVAL, "iz_split_b must be positive with PIC_IZ_OPAL");
    if (!(c->eedf_max_ev > 0)) return fail(PIC_EINVAL, "eedf_max_ev must be positive");
    if (!(c->ion_mass_amu > 0) || !(c->te_ev >= 0) || !(c->ti_ev >= 0))
        return fail(PIC_EINVAL, "bad species parameters");
    if (c->mcc && (!(c->gas_temp > 0) || !(c->pressure_mtorr >= 0) || !(c->eps_cap > 0) ||
                   c->exc_ramp_end <= c->exc_thr || !(c->iz_thr > 0)))
        return fail(PIC_EINVAL, "bad collision parameters");
    if (c->sort_period < 0 || c->diag_period < 0) return fail(PIC_EINVAL, "negative period");
    if (c->cell_width) {
        if ((c->scheme != PIC_EC_EXPLICIT && c->scheme != PIC_EC_IMPLICIT && c->scheme != PIC_EC3_EXPLICIT) ||
            !c->ions_mobile)
            return fail(PIC_EINVAL, "a non-uniform grid takes the EC schemes (PIC_EC_EXPLICIT, PIC_EC_IMPLICIT, "
                                    "PIC_EC3_EXPLICIT) with mobile ions");
        double sum = 0.0;
        for (int k = 0; k < c->n_cells; ++k) {
            const double w = c->cell_width[k];
            if (!(w > 0.0) || !std::isfinite(w)) return fail(PIC_EINVAL, "cell_width[%d] = %g is not a positive width", k, w);
            sum += w;
        }
        if (!(std::fabs(sum - c->length) <= 1e-9 * c->length))
            return fail(PIC_EINVAL, "cell widths sum to %.12g m, length is %.12g m", sum, c->length);
    }
    // Eq. (1): the leapfrog push is stable only for omega_p dt < 2.
    const double wp = std::sqrt(c->n0 * kE * kE / (kEps0 * kMe));
    if (c->strict && !implicit_scheme(*c) && !(wp * c->dt < 2.0))
        return fail(PIC_EUNSTABLE, "omega_p dt = %.3f >= 2 violates the leapfrog limit of Eq. (1)",
                    wp * c->dt);
    return PIC_OK;
}

struct Snapshot {
    uint64_t magic;
    uint64_t version;
    uint64_t arena_bytes;
    int64_t host_step;
};
constexpr uint64_t kSnapMagic = 0x3150434950434547ull;

}  // namespace

void pic::set_last_error(const char *msg) { g_error = msg; }

struct pic_handle {
    pic_config cfg;
    Layout layout;
    Run run;
    unsigned char *arena;
    size_t arena_bytes;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    int grid_push;
    int grid_sort;
    long long host_step;
    std::string err;
    cudaGraphExec_t cycle_graph;
    int cycle_len;
    unsigned int check_host;  // pic_set_particles: the device check's flag, read back
    std::vector<double> widths;  // the non-uniform grid's cell widths (cfg.cell_width points here)
};

namespace {

int cuda_fail(pic_handle *h, cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_error = buf;
    if (h) h->err = buf;
    return PIC_ECUDA;
}

#define CK(h, call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// Thresholds of the waiting time between null-collision selections.  The
// steps W from a selection (or from entering the run) to the next one follow
// the geometric law P(W > k) = q^k, q = 1 - P_null (the law of one
// Bernoulli(P_null) trial per step).  W - 1 = 4096 a + 64 b + c with three
// independent digits: c and b geometric with ratios q and q^64 cut to 0..63,
// a geometric with ratio q^4096 where a = 64 stands for a wait beyond 64^3
// steps (it ends in a fresh draw).  A digit is the number of thresholds
// T_j = floor(2^32 P(digit >= j)) above a 32-bit Philox word: t[0] for c and
// t[1] for b (j = 1..63), t[2] for a (j = 1..64).
void wait_thresholds(double p_null, uint32_t t[3][64]) {
    const double q = 1.0 - p_null;
    for (int dg = 0; dg < 3; ++dg) {
        const double r = dg == 0 ? q : (dg == 1 ? std::pow(q, 64.0) : std::pow(q, 4096.0));
        const double r64 = std::pow(r, 64.0);
        for (int j = 1; j <= 64; ++j) {
            double f;
            if (dg == 2) {
                f = std::pow(r, (double)j);
            } else if (j == 64) {
                t[dg][63] = 0u;
                continue;
            } else {
                f = 1.0 - r64 > 0.0 ? (std::pow(r, (double)j) - r64) / (1.0 - r64) : 1.0;
            }
            const double v = std::floor(std::ldexp(f, 32));
            t[dg][j - 1] = v >= 4294967295.0 ? 0xffffffffu : (uint32_t)v;
        }
    }
}

void derive_impl(const pic_config &c, const Layout &L, unsigned char *A, Run &R) {
    std::memset(&R, 0, sizeof R);
    R.n_cells = c.n_cells;
    R.periodic = c.boundary == PIC_BC_PERIODIC;
    R.scheme = c.scheme;
    R.mcc = c.mcc;
    R.ions_mobile = c.ions_mobile;
    R.diag_period = c.diag_period;
    R.eedf_bins = c.eedf_bins;
    R.sort_period = c.sort_period;
    R.seed = c.seed;
    R.run = c.run;
    for (int r = 0; r < 10; ++r) {  // Philox4x32-10 key schedule (Weyl increments)
        R.rk0[r] = c.seed + (uint32_t)r * 0x9E3779B9u;
        R.rk1[r] = c.run + (uint32_t)r * 0xBB67AE85u;
    }
    R.capacity[0] = c.capacity[0];
    R.capacity[1] = c.capacity[1];
    R.births_cap = c.births_capacity > 0 ? c.births_capacity : 1;
    const double dx = c.length / c.n_cells;
    const double w = c.n0 * c.length / (double)c.np_init;
    const double q[2] = {-kE, kE};
    const double m[2] = {kMe, c.ion_mass_amu * kAmu};
    R.dx = dx;
    R.inv_dx = 1.0 / dx;
    R.dt = c.dt;
    R.rf_freq = c.rf_freq;
    R.rf_volt = R.periodic ? 0.0 : c.rf_volt;
    R.weight = w;
    // one integer charge unit of the fixed-point node charges: 2^-33 of a
    // macro-particle, 2^-36/6 for the m = 3 scheme
    const double two_m33 = c.scheme == PIC_EC3_EXPLICIT ? std::ldexp(1.0, -36) / 6.0 : std::ldexp(1.0, -33);
    R.kappa = kE * w * two_m33 / kEps0;
    R.kappa_bg = c.ions_mobile ? 0.0 : dx * kE * c.bg_density / kEps0;
    R.dens_scale = w * two_m33 / dx;
    R.eps0_dx_half = 0.5 * kEps0 * dx;
    auto split = [](double v, float (&out)[2]) {
        out[0] = (float)v;
        out[1] = (float)(v - (double)out[0]);
    };
    split(R.kappa, R.kappa_ff);
    split(R.kappa_bg, R.kbg_ff);
    split(1.0 / (double)c.n_cells, R.inv_n_ff);
    split(1.0 / ((double)c.n_cells * dx), R.inv_ndx_ff);
    for (int s = 0; s < 2; ++s) {
        R.chi_coef[s] = 0.5 * c.dt * c.dt * q[s] * q[s] * w / (m[s] * kEps0 * dx) * std::ldexp(1.0, -16);
        R.half_m_w[s] = 0.5 * m[s] * w;
        R.qm_dt[s] = (float)(q[s] / m[s] * c.dt);
        R.qm[s] = (float)(q[s] / m[s]);
        R.mq[s] = (float)(m[s] / q[s]);
        R.qw[s] = (float)(q[s] * w);
        R.half_m_over_e[s] = (float)(0.5 * m[s] / kE);
    }
    R.dt_dx = (float)(c.dt / dx);
    R.half_dt = (float)(0.5 * c.dt);
    R.half_dt2_dx = (float)(0.5 * c.dt * c.dt / dx);
    R.half_dt2 = (float)(0.5 * c.dt * c.dt);
    R.abar_ion_over_e = (float)((kE / m[1]) / (-kE / kMe));
    R.eedf_inv_width = (float)(c.eedf_bins / c.eedf_max_ev);
    // Null-collision bounds (Vahedi & Surendra): per process the maximum of
    // n_g sigma v up to the cap energy; sigma_iz v peaks where ln(eps/I) = 2.
    const double ng = gas_density(c);
    const double vth_gas = std::sqrt(kKb * c.gas_temp / m[1]);
    R.n_g = (float)ng;
    R.vth_gas = (float)vth_gas;
    if (c.mcc) {
        const double v_cap = std::sqrt(2.0 * kE * c.eps_cap / kMe);
        const double eps_star = std::fmin(c.eps_cap, c.iz_thr * kEulerN * kEulerN);
        const double v_star = std::sqrt(2.0 * kE * eps_star / kMe);
        const double nu_e = ng * (c.sig_el * v_cap + sig_exc(c, c.eps_cap) * v_cap + sig_iz(c, eps_star) * v_star);
        const double g_max = std::sqrt(2.0 * kE * c.cx_vmax / m[1]) + 6.0 * vth_gas;
        const double nu_i = ng * c.sig_cx * g_max;
        const double p_e = 1.0 - std::exp(-nu_e * c.dt);
        const double p_i = 1.0 - std::exp(-nu_i * c.dt);
        R.thr[0] = p_e > 0.0 ? 1u : 0u;
        R.thr[1] = p_i > 0.0 ? 1u : 0u;
        R.p_null[0] = p_e;
        R.p_null[1] = p_i;
        R.nu_max_e = (float)nu_e;
        R.nu_max_i = (float)nu_i;
        R.g_max_i = (float)g_max;
    }
    R.iz_opal = (c.collision_model & PIC_IZ_OPAL) ? 1 : 0;
    R.scatter_vs = (c.collision_model & PIC_SCATTER_VS) ? 1 : 0;
    R.iz_b = (float)c.iz_split_b;
    R.sig_el = (float)c.sig_el;
    R.exc_thr = (float)c.exc_thr;
    R.exc_ramp_end = (float)c.exc_ramp_end;
    R.exc_slope = (float)(c.sig_exc_max / (c.exc_ramp_end - c.exc_thr));
    R.sig_exc_max = (float)c.sig_exc_max;
    R.iz_thr = (float)c.iz_thr;
    R.sig_iz_k = (float)(c.sig_iz_peak * kEulerN);
    R.sig_cx = (float)c.sig_cx;
    R.eps_cap = (float)c.eps_cap;
    R.two_m_over_M = (float)(2.0 * kMe / m[1]);
    R.two_e_over_me = (float)(2.0 * kE / kMe);
    // pointers
    for (int p = 0; p < 2; ++p)
        for (int s = 0; s < 2; ++s) {
            Species &sp = R.buf[p][s];
            sp.cell = (int32_t *)(A + L.sp[p][s][0]);
            sp.off = (float *)(A + L.sp[p][s][1]);
            sp.vx = (float *)(A + L.sp[p][s][2]);
            sp.vy = (float *)(A + L.sp[p][s][3]);
            sp.vz = (float *)(A + L.sp[p][s][4]);
            sp.id = (uint32_t *)(A + L.sp[p][s][5]);
            sp.abar = implicit_scheme(c) ? (float *)(A + L.sp[p][s][6]) : nullptr;
        }
    for (int s = 0; s < 2; ++s) {
        R.acc_cnt[s] = (unsigned long long *)(A + L.acc_cnt[s]);
        R.acc_a[s] = (unsigned long long *)(A + L.acc_a[s]);
        R.acc_b[s] = (unsigned long long *)(A + L.acc_b[s]);
        R.acc_c[s] = (unsigned long long *)(A + L.acc_c[s]);
        R.cursor[s] = (unsigned int *)(A + L.cursor[s]);
        R.rho_q[s] = (long long *)(A + L.rho_q[s]);
        R.heat[s] = (double *)(A + L.heat[s]);
    }
    R.e_gather = (float *)(A + L.e_gather);
    R.e_hi = (float *)(A + L.e_hi);
    R.wait_tab = (const uint32_t *)(A + L.wait_tab);
    R.e_lo = (float *)(A + L.e_lo);
    R.e_cc = (double *)(A + L.e_cc);
    R.chi = (double *)(A + L.chi);
    R.avg_ne = (double *)(A + L.avg_ne);
    R.avg_ni = (double *)(A + L.avg_ni);
    R.avg_e = (double *)(A + L.avg_e);
    R.eedf = (unsigned long long *)(A + L.eedf);
    R.births = (Birth *)(A + L.births);
    R.st = (DevState *)(A + L.state);
    R.dt_f = (float)c.dt;
    R.len_f = (float)c.length;
    R.eps0_half = 0.5 * kEps0;
    split(1.0 / c.length, R.inv_len_ff);
    R.stretched = c.cell_width ? 1 : 0;
    if (R.stretched) {
        R.hw = (const float2 *)(A + L.hw);
        R.h64 = (const double *)(A + L.h64);
        R.xnode = (const double *)(A + L.xnode);
        R.hdw = (const float2 *)(A + L.hdw);
        R.wdw = (const float2 *)(A + L.wdw);
    }
}

// The non-uniform grid's tables from the cell widths: (h, 1/h) in FP32 for
// the push, node positions x_0 = 0, x_{g+1} = x_g + h_g for the load, h as
// a double-word pair for the field, and for the periodic box the share W_c
// of the net charge the nodes 0..c carry when it is spread in proportion to
// the node lengths (h_{g-1} + h_g) / 2 (double-word).
void grid_tables(const pic_config &c, std::vector<float2> &hw, std::vector<double> &xn,
                 std::vector<float2> &hdw, std::vector<float2> &wdw) {
    const int n = c.n_cells;
    auto pair = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    hw.resize(n);
    xn.assign(n + 1, 0.0);
    hdw.resize(n);
    wdw.resize(n);
    double len = 0.0;
    for (int k = 0; k < n; ++k) {
        const double h = c.cell_width[k];
        hw[k] = make_float2((float)h, (float)(1.0 / h));
        hdw[k] = pair(h);
        xn[k + 1] = xn[k] + h;
        len += h;
    }
    double acc = 0.0;
    for (int g = 0; g < n; ++g) {
        acc += 0.5 * (c.cell_width[(g - 1 + n) % n] + c.cell_width[g]) / len;
        wdw[g] = pair(acc);
    }
}

Mode push_mode(const pic_config &c) {
    if (c.cell_width && c.scheme == PIC_EC_EXPLICIT) return kExplicitNU;
    if (c.scheme == PIC_EC3_EXPLICIT) return c.cell_width ? kExplicitEC3NU : kExplicitEC3;
    return c.scheme == PIC_MC_EXPLICIT ? kExplicitMC : kExplicitEC;
}
Mode deposit_mode(const pic_config &c) {
    if (c.scheme == PIC_EC3_EXPLICIT) return kDepositEC3;
    return (c.scheme == PIC_MC_EXPLICIT || c.scheme == PIC_MC_IMPLICIT) ? kDepositMC : kDepositEC;
}
Mode pass1_mode(const pic_config &c) {
    if (c.cell_width) return kImplicit1NU;
    return c.scheme == PIC_MC_IMPLICIT ? kImplicit1MC : kImplicit1;
}
Mode pass2_mode(const pic_config &c) {
    if (c.cell_width) return kImplicit2NU;
    return c.scheme == PIC_MC_IMPLICIT ? kImplicit2MC : kImplicit2;
}

// Enqueue one step (and the sort that closes a sort cycle) on stream s.
int enqueue_step(pic_handle *h, long long step_index, cudaStream_t s) {
    const pic_config &c = h->cfg;
    if (implicit_scheme(c)) {
        CK(h, launch_particles(h->run, pass1_mode(c), h->grid_push, s));
        CK(h, launch_particles(h->run, pass2_mode(c), h->grid_push, s));
    } else {
        CK(h, launch_particles(h->run, push_mode(c), h->grid_push, s));
    }
    if (c.sort_period > 0 && (step_index + 1) % c.sort_period == 0)
        CK(h, launch_sort(h->run, h->grid_sort, s));
    return PIC_OK;
}

int sync(pic_handle *h) {
    CK(h, cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

// The device state record after everything enqueued so far (one sync).
int read_state(pic_handle *h, DevState *st) {
    CK(h, cudaMemcpyAsync(st, h->run.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    return sync(h);
}

}  // namespace

namespace pic {

Layout make_run_layout(const pic_config &c) { return make_layout(c); }
int validate_run_config(const pic_config *c) { return validate(c); }
void derive_run(const pic_config &c, const Layout &L, unsigned char *arena, Run &R) {
    derive_impl(c, L, arena, R);
}
Mode push_mode_of(const pic_config &c) { return push_mode(c); }
Mode deposit_mode_of(const pic_config &c) { return deposit_mode(c); }

#define CKE(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            char b_[512];                                                          \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));     \
            g_error = b_;                                                          \
            if (err) *err = b_;                                                    \
            return PIC_ECUDA;                                                      \
        }                                                                          \
    } while (0)

int run_diag(const Run &R, const pic_config &c, const Layout &L, unsigned char *arena, cudaStream_t s,
             pic_diag_t *out, int reset_avg, std::string *err) {
    CKE(launch_finalize(R, s));  // work the last tail left to the next launch
    CKE(cudaMemsetAsync(R.st->ke_perp, 0, sizeof(double) * 2, s));
    CKE(launch_perp_energy(R, s));
    DevState st;
    CKE(cudaMemcpyAsync(&st, R.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
    std::memset(out, 0, sizeof *out);
    out->step = st.step;
    for (int k = 0; k < 2; ++k) {
        out->count[k] = st.n_live[k];
        for (int w = 0; w < 2; ++w) {
            out->wall_count[k][w] = st.wall_count[k][w];
            out->wall_energy_ev[k][w] = st.wall_energy[k][w];
        }
        out->overflow[k] = st.overflow[k];
        out->ke_x[k] = st.ke_x[k] * R.half_m_w[k];
        out->ke_perp[k] = st.ke_perp[k];
        out->power[k] = st.power[k];
    }
    for (int k = 0; k < 5; ++k) out->coll[k] = st.coll[k];
    out->births = st.births_total;
    out->field_energy = st.field_energy;
    out->field_energy_push = st.field_energy_push;
    out->n_avg = st.n_avg;
    out->n_diag = st.n_diag;
    out->status = st.status;
    if (reset_avg) {
        const size_t n1 = (size_t)c.n_cells + 1;
        CKE(cudaMemsetAsync(arena + L.avg_ne, 0, 8 * n1, s));
        CKE(cudaMemsetAsync(arena + L.avg_ni, 0, 8 * n1, s));
        CKE(cudaMemsetAsync(arena + L.avg_e, 0, 8 * n1, s));
        CKE(cudaMemsetAsync(&R.st->v_sum, 0, sizeof(double), s));
        CKE(cudaMemsetAsync(arena + L.heat[0], 0, 8 * n1, s));
        CKE(cudaMemsetAsync(arena + L.heat[1], 0, 8 * n1, s));
        CKE(cudaMemsetAsync(arena + L.eedf, 0, 8 * ((size_t)c.eedf_bins + 1), s));
        CKE(cudaMemsetAsync(&R.st->n_avg, 0, sizeof(long long) * 2, s));
        CKE(cudaStreamSynchronize(s));
    }
    return PIC_OK;
}

int init_run_state(const pic_config &c, const Run &R, unsigned char *arena, size_t arena_bytes, int grid,
                   cudaStream_t s, std::string *err) {
    CKE(cudaMemsetAsync(arena, 0, arena_bytes, s));
    DevState st;
    std::memset(&st, 0, sizeof st);
    st.n_slots[0] = st.n_live[0] = c.np_init;
    st.n_slots[1] = st.n_live[1] = c.ions_mobile ? c.np_init : 0;
    st.next_id[0] = (unsigned int)c.np_init;
    st.next_id[1] = (unsigned int)st.n_slots[1];
    CKE(cudaMemcpyAsync(R.st, &st, sizeof st, cudaMemcpyHostToDevice, s));
    uint32_t tab[2][3][64];
    std::memset(tab, 0, sizeof tab);
    if (c.mcc) {
        wait_thresholds(R.p_null[0], tab[0]);
        wait_thresholds(R.p_null[1], tab[1]);
    }
    CKE(cudaMemcpyAsync((void *)R.wait_tab, tab, sizeof tab, cudaMemcpyHostToDevice, s));
    std::vector<float2> hw, hdw, wdw;
    std::vector<double> xn;
    if (R.stretched) {
        grid_tables(c, hw, xn, hdw, wdw);
        const size_t n = (size_t)c.n_cells;
        CKE(cudaMemcpyAsync((void *)R.hw, hw.data(), 8 * n, cudaMemcpyHostToDevice, s));
        CKE(cudaMemcpyAsync((void *)R.h64, c.cell_width, 8 * n, cudaMemcpyHostToDevice, s));
        CKE(cudaMemcpyAsync((void *)R.xnode, xn.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
        CKE(cudaMemcpyAsync((void *)R.hdw, hdw.data(), 8 * n, cudaMemcpyHostToDevice, s));
        CKE(cudaMemcpyAsync((void *)R.wdw, wdw.data(), 8 * n, cudaMemcpyHostToDevice, s));
    }
    CKE(cudaStreamSynchronize(s));
    const double vth_e = std::sqrt(kE * c.te_ev / kMe);
    const double vth_i = std::sqrt(kE * c.ti_ev / (c.ion_mass_amu * kAmu));
    CKE(launch_load(R, 0, c.np_init, (float)vth_e, s));
    if (c.ions_mobile) CKE(launch_load(R, 1, c.np_init, (float)vth_i, s));
    // t = 0 charge assignment and field, abar = a^0 for the implicit scheme
    CKE(launch_particles(R, deposit_mode(c), grid, s));
    CKE(launch_finalize(R, s));  // FP64 copy and energy of the t = 0 field
    if (implicit_scheme(c)) CKE(launch_set_abar(R, s));
    // the load is in random order: sort it once so that every block streams
    // particles of a few adjacent cells from the first step on
    CKE(launch_sort(R, grid, s));
    return PIC_OK;
}

int run_profiles(const Run &R, const pic_config &c, cudaStream_t s, double *ne, double *ni, double *phi,
                 double *heat_e, double *heat_i, uint64_t *eedf, std::string *err) {
    CKE(launch_finalize(R, s));
    CKE(cudaStreamSynchronize(s));
    DevState st;
    CKE(cudaMemcpy(&st, R.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    const size_t n1 = (size_t)c.n_cells + 1, n = (size_t)c.n_cells;
    const double na = st.n_avg > 0 ? (double)st.n_avg : 1.0;
    const double nd = st.n_diag > 0 ? (double)st.n_diag : 1.0;
    auto fetch = [&](double *dst, const double *src, size_t cnt, double scale) -> cudaError_t {
        if (!dst) return cudaSuccess;
        const cudaError_t e = cudaMemcpy(dst, src, 8 * cnt, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (size_t k = 0; k < cnt; ++k) dst[k] *= scale;
        return e;
    };
    CKE(fetch(ne, R.avg_ne, n1, R.dens_scale / na));
    CKE(fetch(ni, R.avg_ni, n1, R.dens_scale / na));
    const bool periodic = c.boundary == PIC_BC_PERIODIC;
    if (c.cell_width) {
        // a node's charge spread over its length (h_{g-1} + h_g) / 2 (the wall
        // nodes take their one cell twice, as the uniform grid's take dx)
        for (size_t g = 0; g < n1; ++g) {
            const double hl = periodic ? c.cell_width[(g + n - 1) % n] : c.cell_width[g > 0 ? g - 1 : 0];
            const double hr = periodic ? c.cell_width[g % n] : c.cell_width[g < n ? g : n - 1];
            const double f = R.dx / (0.5 * (hl + hr));
            if (ne) ne[g] *= f;
            if (ni) ni[g] *= f;
        }
    }
    CKE(fetch(heat_e, R.heat[0], n, 1.0 / nd));
    CKE(fetch(heat_i, R.heat[1], n, 1.0 / nd));
    if (phi) {
        // the averaged potential follows linearly from the averaged field and
        // electrode voltage: phi_g = <V> - sum_{c<g} h_c <E_c>
        std::vector<double> e(n);
        CKE(fetch(e.data(), R.avg_e, n, 1.0 / na));
        double acc = periodic ? 0.0 : st.v_sum / na;
        for (size_t g = 0; g < n; ++g) {
            phi[g] = acc;
            acc -= (c.cell_width ? c.cell_width[g] : R.dx) * e[g];
        }
        phi[n] = periodic ? phi[0] : 0.0;
    }
    if (eedf) CKE(cudaMemcpy(eedf, R.eedf, 8 * ((size_t)c.eedf_bins + 1), cudaMemcpyDeviceToHost));
    return PIC_OK;
}

int run_get_particles(const Run &R, cudaStream_t s, int species, pic_host_particles *out, std::string *err) {
    CKE(cudaStreamSynchronize(s));
    DevState st;
    CKE(cudaMemcpy(&st, R.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    if (out->count < st.n_live[species]) {
        char b[256];
        snprintf(b, sizeof b, "host arrays hold %lld, %lld live particles", (long long)out->count,
                 (long long)st.n_live[species]);
        g_error = b;
        if (err) *err = b;
        return PIC_EINVAL;
    }
    const long long ns = st.n_slots[species];
    const Species &sp = R.buf[st.parity][species];
    std::vector<int32_t> cell(ns);
    std::vector<float> off(ns), vx(ns), vy(ns), vz(ns), ab(ns);
    std::vector<uint32_t> id(ns);
    if (ns > 0) {
        CKE(cudaMemcpy(cell.data(), sp.cell, 4 * ns, cudaMemcpyDeviceToHost));
        CKE(cudaMemcpy(off.data(), sp.off, 4 * ns, cudaMemcpyDeviceToHost));
        CKE(cudaMemcpy(vx.data(), sp.vx, 4 * ns, cudaMemcpyDeviceToHost));
        CKE(cudaMemcpy(vy.data(), sp.vy, 4 * ns, cudaMemcpyDeviceToHost));
        CKE(cudaMemcpy(vz.data(), sp.vz, 4 * ns, cudaMemcpyDeviceToHost));
        CKE(cudaMemcpy(id.data(), sp.id, 4 * ns, cudaMemcpyDeviceToHost));
        if (sp.abar) CKE(cudaMemcpy(ab.data(), sp.abar, 4 * ns, cudaMemcpyDeviceToHost));
    }
    long long k = 0;
    for (long long i = 0; i < ns; ++i) {
        if (cell[i] < 0) continue;
        if (out->cell) out->cell[k] = cell[i] & (int32_t)kCellMask;  // without the wait bits
        if (out->off) out->off[k] = off[i];
        if (out->vx) out->vx[k] = vx[i];
        if (out->vy) out->vy[k] = vy[i];
        if (out->vz) out->vz[k] = vz[i];
        if (out->id) out->id[k] = id[i];
        if (out->abar) out->abar[k] = sp.abar ? ab[i] : 0.0f;
        ++k;
    }
    out->count = k;
    out->next_id = st.next_id[species];
    return PIC_OK;
}

}  // namespace pic

extern "C" {

int pic_version(void) { return PIC_ABI_VERSION; }

const char *pic_build_info(void) {
    return "libpic: energy-conserving 1D PIC/MCC, sm_103a, " __DATE__;
}

int pic_required_sizes(const pic_config *cfg, pic_sizes *out) {
    int r = validate(cfg);
    if (r) return r;
    if (!out) return fail(PIC_EINVAL, "out is NULL");
    const Layout L = make_layout(*cfg);
    out->arena_bytes = L.total;
    out->snapshot_bytes = L.total + sizeof(Snapshot);
    return PIC_OK;
}

int pic_init(const pic_config *cfg, const pic_buffers *bufs, void *stream, pic_handle **out) {
    int r = validate(cfg);
    if (r) return r;
    if (!bufs || !out) return fail(PIC_EINVAL, "bufs/out is NULL");
    const Layout L = make_layout(*cfg);
    if (!bufs->arena || bufs->arena_bytes < L.total)
        return fail(PIC_ENOMEM, "arena of %zu bytes, %zu needed", bufs->arena_bytes, L.total);
    if (((uintptr_t)bufs->arena & 255u) != 0) return fail(PIC_ENOMEM, "arena not 256-byte aligned");
    pic_handle *h = new pic_handle();
    h->cfg = *cfg;
    if (cfg->cell_width) {  // the caller's array may go away after this call
        h->widths.assign(cfg->cell_width, cfg->cell_width + cfg->n_cells);
        h->cfg.cell_width = h->widths.data();
    }
    h->layout = L;
    h->arena = (unsigned char *)bufs->arena;
    h->arena_bytes = L.total;
    h->stream = (cudaStream_t)stream;
    h->capture_stream = nullptr;
    h->host_step = 0;
    h->cycle_graph = nullptr;
    h->cycle_len = 0;
    derive_impl(h->cfg, h->layout, h->arena, h->run);
    auto bail = [&](int code) {
        g_error = h->err.empty() ? g_error : h->err;
        delete h;
        return code;
    };
    if (occupancy_grid(h->run, push_mode(*cfg), &h->grid_push) != cudaSuccess) {
        cuda_fail(h, cudaGetLastError(), "occupancy");
        return bail(PIC_ECUDA);
    }
    if (sort_grid(&h->grid_sort) != cudaSuccess) {
        cuda_fail(h, cudaGetLastError(), "sort occupancy");
        return bail(PIC_ECUDA);
    }
    if (implicit_scheme(*cfg)) {
        int g1 = 0, g2 = 0;
        occupancy_grid(h->run, pass1_mode(*cfg), &g1);
        occupancy_grid(h->run, pass2_mode(*cfg), &g2);
        h->grid_push = g1 < g2 ? g1 : g2;
    }
    r = init_run_state(*cfg, h->run, h->arena, L.total, h->grid_push, h->stream, &h->err);
    if (r) return bail(r);
    *out = h;
    return PIC_OK;
}

int pic_init_field(pic_handle *h, int set_abar) {
    if (!h) return fail(PIC_EINVAL, "handle is NULL");
    CK(h, launch_particles(h->run, deposit_mode(h->cfg), h->grid_push, h->stream));
    if (implicit_scheme(h->cfg) && set_abar) CK(h, launch_set_abar(h->run, h->stream));
    return PIC_OK;
}

static int capture_cycle(pic_handle *h) {
    const int len = h->cfg.sort_period > 0 ? h->cfg.sort_period : 16;
    if (!h->capture_stream) CK(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    int r = PIC_OK;
    for (int k = 0; k < len && r == PIC_OK; ++k) r = enqueue_step(h, (long long)k, h->capture_stream);
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
    if (r) return r;
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->cycle_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->cycle_len = len;
    return PIC_OK;
}

int pic_step(pic_handle *h, int64_t n) {
    if (!h) return fail(PIC_EINVAL, "handle is NULL");
    if (n < 0) return fail(PIC_EINVAL, "negative step count");
    const int K = h->cfg.sort_period > 0 ? h->cfg.sort_period : 16;
    while (n > 0) {
        const bool aligned = h->host_step % K == 0;
        if (aligned && n >= K) {
            if (!h->cycle_graph) {
                int r = capture_cycle(h);
                if (r) return r;
            }
            CK(h, cudaGraphLaunch(h->cycle_graph, h->stream));
            h->host_step += K;
            n -= K;
        } else {
            int r = enqueue_step(h, h->host_step, h->stream);
            if (r) return r;
            h->host_step += 1;
            n -= 1;
        }
    }
    return PIC_OK;
}

int pic_diag(pic_handle *h, pic_diag_t *out, int reset_avg) {
    if (!h || !out) return fail(PIC_EINVAL, "NULL argument");
    const int r = run_diag(h->run, h->cfg, h->layout, h->arena, h->stream, out, reset_avg, &h->err);
    if (r) return r;
    if (out->status & PIC_STATUS_TIMEOUT)
        return fail(PIC_ETIMEOUT, "a bounded device wait gave up (status 0x%x): a launch ended its stream early",
                    out->status);
    return PIC_OK;
}

int pic_profiles(pic_handle *h, double *ne, double *ni, double *phi, double *heat_e,
                 double *heat_i, uint64_t *eedf) {
    if (!h) return fail(PIC_EINVAL, "handle is NULL");
    return run_profiles(h->run, h->cfg, h->stream, ne, ni, phi, heat_e, heat_i, eedf, &h->err);
}

int pic_grids(pic_handle *h, int64_t *rho_q_e, int64_t *rho_q_i, double *phi, double *e_cc,
              double *chi) {
    if (!h) return fail(PIC_EINVAL, "handle is NULL");
    CK(h, launch_finalize(h->run, h->stream));
    int r = sync(h);
    if (r) return r;
    const size_t n1 = (size_t)h->cfg.n_cells + 1, n = (size_t)h->cfg.n_cells;
    if (rho_q_e) CK(h, cudaMemcpy(rho_q_e, h->run.rho_q[0], 8 * n1, cudaMemcpyDeviceToHost));
    if (rho_q_i) CK(h, cudaMemcpy(rho_q_i, h->run.rho_q[1], 8 * n1, cudaMemcpyDeviceToHost));
    if (e_cc) CK(h, cudaMemcpy(e_cc, h->run.e_cc, 8 * n, cudaMemcpyDeviceToHost));
    if (phi) {
        // node potential from the cell-centred field: phi_g = V - sum_{c<g} h_c E_c
        std::vector<double> e(n);
        DevState st;
        CK(h, cudaMemcpy(e.data(), h->run.e_cc, 8 * n, cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(&st, h->run.st, sizeof st, cudaMemcpyDeviceToHost));
        const bool periodic = h->cfg.boundary == PIC_BC_PERIODIC;
        double acc = periodic ? 0.0 : st.v_left;
        for (size_t g = 0; g < n; ++g) {
            phi[g] = acc;
            acc -= (h->cfg.cell_width ? h->cfg.cell_width[g] : h->run.dx) * e[g];
        }
        phi[n] = periodic ? phi[0] : 0.0;
    }
    if (chi) CK(h, cudaMemcpy(chi, h->run.chi, 8 * n, cudaMemcpyDeviceToHost));
    return PIC_OK;
}

int pic_count(pic_handle *h, int64_t *n_e, int64_t *n_i) {
    if (!h) return fail(PIC_EINVAL, "handle is NULL");
    DevState st;
    int r = read_state(h, &st);
    if (r) return r;
    if (n_e) *n_e = st.n_live[0];
    if (n_i) *n_i = st.n_live[1];
    return PIC_OK;
}

int pic_get_particles(pic_handle *h, int species, pic_host_particles *out) {
    if (!h || !out || species < 0 || species > 1) return fail(PIC_EINVAL, "bad argument");
    return run_get_particles(h->run, h->stream, species, out, &h->err);
}

namespace {

int check_upload_args(const pic_handle *h, int species, const pic_host_particles *in) {
    if (!in || species < 0 || species > 1) return fail(PIC_EINVAL, "bad argument");
    const long long n = in->count;
    if (n < 0 || n > h->cfg.capacity[species]) return fail(PIC_EOVERFLOW, "count %lld exceeds capacity", (long long)n);
    if (species == 1 && !h->cfg.ions_mobile && n > 0) return fail(PIC_EINVAL, "ions are frozen in this run");
    if (n > 0 && (!in->cell || !in->off || !in->vx || !in->vy || !in->vz || !in->id))
        return fail(PIC_EINVAL, "NULL particle array");
    return PIC_OK;
}

// Host arrays of one species into the idle second buffer, and their check
// (cell in [0, n_cells), offset in [0, 1)) into the state's check word.
int enqueue_upload(pic_handle *h, unsigned int parity, int species, const pic_host_particles *in) {
    const long long n = in->count;
    const Species &sp = h->run.buf[parity][species];
    const Species &up = h->run.buf[parity ^ 1u][species];
    if (n <= 0) return PIC_OK;
    const bool abar_given = sp.abar && in->abar;
    const void *src[7] = {in->cell, in->off, in->vx, in->vy, in->vz, in->id, in->abar};
    void *tmp[7] = {up.cell, up.off, up.vx, up.vy, up.vz, up.id, up.abar};
    for (int f = 0; f < (abar_given ? 7 : 6); ++f)
        CK(h, cudaMemcpyAsync(tmp[f], src[f], 4 * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_check_particles(up.cell, up.off, n, h->cfg.n_cells, &h->run.st->check, h->stream));
    return PIC_OK;
}

// The checked upload into the current buffer, with the species' counters,
// unless a check set the flag (then nothing changes).
int enqueue_apply(pic_handle *h, unsigned int parity, int species, const pic_host_particles *in) {
    const Species &sp = h->run.buf[parity][species];
    const Species &up = h->run.buf[parity ^ 1u][species];
    CK(h, launch_apply_particles(h->run, sp, up, in->count, sp.abar && in->abar, &h->run.st->check, species,
                                 in->next_id, h->stream));
    return PIC_OK;
}

// After the sync: name the first particle off the grid, if the flag is set.
int name_offender(pic_handle *h, const pic_host_particles *in) {
    for (long long i = 0; i < in->count; ++i)
        if (in->cell[i] < 0 || in->cell[i] >= h->cfg.n_cells || !(in->off[i] >= 0.0f) || !(in->off[i] < 1.0f))
            return fail(PIC_EINVAL, "particle %lld outside the grid (cell %d, offset %g)", i, in->cell[i],
                        (double)in->off[i]);
    return PIC_OK;
}

// Upload, check and apply the given species (nullptr: left as it is); if any
// particle of any of them is off the grid nothing is applied.
int set_species(pic_handle *h, const pic_host_particles *const in[2]) {
    for (int S = 0; S < 2; ++S) {
        if (!in[S]) continue;
        int r = check_upload_args(h, S, in[S]);
        if (r) return r;
    }
    DevState st;
    int r = read_state(h, &st);
    if (r) return r;
    CK(h, cudaMemsetAsync(&h->run.st->check, 0, 4, h->stream));
    for (int S = 0; S < 2; ++S)
        if (in[S] && (r = enqueue_upload(h, st.parity, S, in[S]))) return r;
    for (int S = 0; S < 2; ++S)
        if (in[S] && (r = enqueue_apply(h, st.parity, S, in[S]))) return r;
    CK(h, cudaMemcpyAsync(&h->check_host, &h->run.st->check, 4, cudaMemcpyDeviceToHost, h->stream));
    r = sync(h);
    if (r) return r;
    if (h->check_host) {
        for (int S = 0; S < 2; ++S)
            if (in[S] && (r = name_offender(h, in[S]))) return r;
        return fail(PIC_EINVAL, "a particle is outside the grid");
    }
    return PIC_OK;
}

}  // namespace

int pic_set_particles(pic_handle *h, int species, const pic_host_particles *in) {
    if (!h || !in || species < 0 || species > 1) return fail(PIC_EINVAL, "bad argument");
    const pic_host_particles *both[2] = {species == 0 ? in : nullptr, species == 1 ? in : nullptr};
    return set_species(h, both);
}

int pic_set_state(pic_handle *h, const pic_host_particles *electrons, const pic_host_particles *ions) {
    if (!h || !electrons || !ions) return fail(PIC_EINVAL, "bad argument");
    const pic_host_particles *both[2] = {electrons, ions};
    return set_species(h, both);
}

int pic_set_step(pic_handle *h, int64_t step) {
    if (!h || step < 0) return fail(PIC_EINVAL, "bad argument");
    long long s = step;
    CK(h, cudaMemcpyAsync(&h->run.st->step, &s, 8, cudaMemcpyHostToDevice, h->stream));
    h->host_step = step;
    return sync(h);
}

int pic_status(pic_handle *h, uint32_t *status) {
    if (!h || !status) return fail(PIC_EINVAL, "NULL argument");
    DevState st;
    int r = read_state(h, &st);
    if (r) return r;
    *status = st.status;
    return PIC_OK;
}

int pic_save(pic_handle *h, void *host_buf, size_t nbytes) {
    if (!h || !host_buf) return fail(PIC_EINVAL, "NULL argument");
    if (nbytes < h->arena_bytes + sizeof(Snapshot)) return fail(PIC_ENOMEM, "snapshot buffer too small");
    int r = sync(h);
    if (r) return r;
    Snapshot s = {kSnapMagic, PIC_ABI_VERSION, h->arena_bytes, h->host_step};
    std::memcpy(host_buf, &s, sizeof s);
    CK(h, cudaMemcpy((unsigned char *)host_buf + sizeof s, h->arena, h->arena_bytes, cudaMemcpyDeviceToHost));
    return PIC_OK;
}

int pic_load(pic_handle *h, const void *host_buf, size_t nbytes) {
    if (!h || !host_buf) return fail(PIC_EINVAL, "NULL argument");
    if (nbytes < sizeof(Snapshot)) return fail(PIC_EINVAL, "snapshot too small");
    Snapshot s;
    std::memcpy(&s, host_buf, sizeof s);
    if (s.magic != kSnapMagic || s.arena_bytes != h->arena_bytes || nbytes < h->arena_bytes + sizeof s)
        return fail(PIC_EINVAL, "snapshot does not match this run's layout");
    int r = sync(h);
    if (r) return r;
    CK(h, cudaMemcpy(h->arena, (const unsigned char *)host_buf + sizeof s, h->arena_bytes, cudaMemcpyHostToDevice));
    h->host_step = s.host_step;
    return PIC_OK;
}

int pic_philox_fill(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                    int64_t n, uint32_t *out_device, void *stream) {
    if (n < 0 || (n > 0 && !out_device)) return fail(PIC_EINVAL, "bad argument");
    cudaError_t e = launch_philox_fill(k0, k1, c0, c1, c2, c3, n, out_device, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox_fill");
    return PIC_OK;
}

void pic_free(pic_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->cycle_graph) cudaGraphExecDestroy(h->cycle_graph);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
}

const char *pic_last_error(const pic_handle *h) {
    if (h && !h->err.empty()) return h->err.c_str();
    return g_error.c_str();
}

}  // extern "C"
