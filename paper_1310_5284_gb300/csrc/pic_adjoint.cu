// pic_adjoint.cu -- host side of the adjoint of the collisionless EC explicit
// step (the pic_adj_* part of include/pic.h): arena layout, the checkpointed
// forward run, and the backward sweep that recomputes one segment of time
// levels from its checkpoint and runs one reverse launch per step (kernels
// k_adj_fwd / k_adj_rev in pic_kernels.cu).
#include "pic.h"
#include "pic_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pic;

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct AdjLayout {
    Layout run;                   // DevState, accumulators and field buffers of the shared step code
    size_t e_store;               // [(K+1)][n+2] float: gather table of every time level
    size_t lam[2];                // [n+2] float: adjoint field table, ping-pong
    size_t le;                    // [n+3] double: scattered sensitivities
    size_t obj;                   // [K][2] double: P^n, G^n
    size_t obj_scratch;           // [2] double: objectives of recomputed steps (discarded)
    size_t dv0;                   // double
    size_t ckpt;                  // [ncp][3][N] checkpoints (cell, off, vx)
    size_t seg;                   // [C-1][3][N] levels inside one segment
    size_t lx, lv;                // [N] float
    size_t arr;                   // bytes of one padded per-particle array
    long long ncp, C;
    size_t total;
};

pic_config run_config(const pic_adj_config &a) {
    pic_config c;
    std::memset(&c, 0, sizeof c);
    c.scheme = PIC_EC_EXPLICIT;
    c.boundary = a.boundary;
    c.n_cells = a.n_cells;
    c.mcc = 0;
    c.ions_mobile = 0;
    c.sort_period = 0;
    c.diag_period = 0;
    c.eedf_bins = 1;
    c.np_init = a.n_particles;
    c.capacity[0] = 0;
    c.capacity[1] = 0;
    c.births_capacity = 1;
    c.length = a.length;
    c.dt = a.dt;
    c.rf_freq = a.rf_freq;
    c.rf_volt = 0.0;
    c.n0 = a.n0;
    c.bg_density = a.bg_density;
    c.te_ev = 1.0;
    c.ti_ev = 0.026;
    c.ion_mass_amu = 39.948;
    c.gas_temp = 300.0;
    c.exc_thr = 11.5;
    c.exc_ramp_end = 23.0;
    c.iz_thr = 15.8;
    c.eedf_max_ev = 1.0;
    return c;
}

AdjLayout make_adj_layout(const pic_adj_config &a) {
    AdjLayout L;
    const pic_config c = run_config(a);
    L.run = make_run_layout(c);
    size_t o = a256(L.run.total);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = a256(o + bytes);
        return at;
    };
    const size_t n2 = (size_t)a.n_cells + 2;
    const long long K = a.nsteps;
    L.C = a.checkpoint_every;
    L.ncp = K / L.C + 1;
    L.arr = a256(4 * (size_t)a.n_particles);
    L.e_store = take(4 * n2 * (size_t)(K + 1));
    L.lam[0] = take(4 * n2);
    L.lam[1] = take(4 * n2);
    L.le = take(8 * (n2 + 1));
    L.obj = take(16 * (size_t)K);
    L.obj_scratch = take(16);
    L.dv0 = take(8);
    L.ckpt = take(3 * L.arr * (size_t)L.ncp);
    L.seg = take(3 * L.arr * (size_t)(L.C > 1 ? L.C - 1 : 1));
    L.lx = take(L.arr);
    L.lv = take(L.arr);
    L.total = o;
    return L;
}

int validate_adj(const pic_adj_config *a) {
    if (!a) return PIC_EINVAL;
    if (a->boundary != PIC_BC_ELECTRODES && a->boundary != PIC_BC_PERIODIC) return PIC_EINVAL;
    if (a->n_cells < 2 || a->n_cells > kMaxCells) return PIC_EINVAL;
    if (a->checkpoint_every < 1 || a->nsteps < 1 || a->step0 < 0) return PIC_EINVAL;
    if (a->n_particles < 1) return PIC_EINVAL;
    if (a->n_particles >= (1ll << 29)) return PIC_EOVERFLOW;
    if (!(a->length > 0.0) || !(a->dt > 0.0) || !(a->n0 > 0.0) || !(a->bg_density >= 0.0) ||
        !(a->rf_freq >= 0.0) || !std::isfinite(a->length) || !std::isfinite(a->dt) || !std::isfinite(a->n0))
        return PIC_EINVAL;
    return PIC_OK;
}

}  // namespace

struct pic_adj {
    pic_adj_config cfg;
    AdjLayout L;
    unsigned char *arena;
    cudaStream_t stream;
    Run R;
    int grid;
    double volt;          // rf_volt of the last forward run
    bool have_forward;
    long long seg_valid;  // segment whose inner levels the segment store holds (-1: none)
    std::vector<double> obj_host;
    std::string err;
};

namespace {

int fail_a(pic_adj *h, int code, const char *msg) {
    set_last_error(msg);
    if (h) h->err = msg;
    return code;
}

int cuda_fail_a(pic_adj *h, cudaError_t e, const char *what) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return fail_a(h, PIC_ECUDA, buf);
}

#define CKA(h, call)                                          \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail_a(h, e_, #call); \
    } while (0)

// Storage of time level k: a checkpoint at multiples of C, else a slot of the
// segment store.
AdjSlot slot_of(const pic_adj *h, long long k) {
    const AdjLayout &L = h->L;
    const long long r = k % L.C;
    unsigned char *base = r == 0 ? h->arena + L.ckpt + 3 * L.arr * (size_t)(k / L.C)
                                 : h->arena + L.seg + 3 * L.arr * (size_t)(r - 1);
    AdjSlot s;
    s.cell = (int32_t *)base;
    s.off = (float *)(base + L.arr);
    s.vx = (float *)(base + 2 * L.arr);
    return s;
}

float *e_table(const pic_adj *h, long long k) {
    return (float *)(h->arena + h->L.e_store) + (size_t)k * ((size_t)h->cfg.n_cells + 2);
}

Run run_with_volt(const pic_adj *h) {
    Run R = h->R;
    R.rf_volt = h->cfg.boundary == PIC_BC_PERIODIC ? 0.0 : h->volt;
    return R;
}

// One forward step from level k to k+1; objectives to obj (null: scratch).
int forward_step(pic_adj *h, long long k, bool keep_obj) {
    AdjFwd A;
    A.in = slot_of(h, k);
    A.out = slot_of(h, k + 1);
    A.e_in = e_table(h, k);
    A.e_out = e_table(h, k + 1);
    A.obj = keep_obj ? (double *)(h->arena + h->L.obj) + 2 * k : (double *)(h->arena + h->L.obj_scratch);
    A.np = h->cfg.n_particles;
    A.level = h->cfg.step0 + k + 1;
    CKA(h, launch_adj_fwd(run_with_volt(h), A, true, h->grid, h->stream));
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_adj_required_sizes(const pic_adj_config *cfg, pic_sizes *out) {
    const int v = validate_adj(cfg);
    if (v) return fail_a(nullptr, v, "pic_adj_required_sizes: invalid configuration");
    if (!out) return fail_a(nullptr, PIC_EINVAL, "pic_adj_required_sizes: out is NULL");
    const AdjLayout L = make_adj_layout(*cfg);
    out->arena_bytes = L.total;
    out->snapshot_bytes = 0;
    return PIC_OK;
}

int pic_adj_init(const pic_adj_config *cfg, const pic_buffers *bufs, void *cuda_stream, pic_adj **out) {
    const int v = validate_adj(cfg);
    if (v) return fail_a(nullptr, v, "pic_adj_init: invalid configuration");
    if (!bufs || !out) return fail_a(nullptr, PIC_EINVAL, "pic_adj_init: NULL argument");
    const AdjLayout L = make_adj_layout(*cfg);
    if (!bufs->arena || bufs->arena_bytes < L.total || ((uintptr_t)bufs->arena & 255u))
        return fail_a(nullptr, PIC_ENOMEM, "pic_adj_init: arena too small or not 256-byte aligned");
    pic_adj *h = new pic_adj();
    h->cfg = *cfg;
    h->L = L;
    h->arena = (unsigned char *)bufs->arena;
    h->stream = (cudaStream_t)cuda_stream;
    h->volt = 0.0;
    h->have_forward = false;
    h->seg_valid = -1;
    const pic_config c = run_config(*cfg);
    derive_run(c, L.run, h->arena, h->R);
    cudaError_t e = adj_prepare(cfg->n_cells, &h->grid);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->arena, 0, L.total, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cuda_fail_a(nullptr, e, "pic_adj_init");
        delete h;
        return PIC_ECUDA;
    }
    *out = h;
    return PIC_OK;
}

int pic_adj_forward(pic_adj *h, double rf_volt, const int32_t *cell0, const float *off0, const float *vx0,
                    double *power_flux) {
    if (!h || !cell0 || !off0 || !vx0 || !power_flux) return fail_a(h, PIC_EINVAL, "pic_adj_forward: NULL argument");
    if (!std::isfinite(rf_volt)) return fail_a(h, PIC_EINVAL, "pic_adj_forward: rf_volt not finite");
    const long long K = h->cfg.nsteps, N = h->cfg.n_particles;
    h->volt = rf_volt;
    h->have_forward = false;
    h->seg_valid = -1;
    cudaStream_t s = h->stream;
    const AdjSlot s0 = slot_of(h, 0);
    CKA(h, cudaMemcpyAsync(s0.cell, cell0, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    CKA(h, cudaMemcpyAsync(s0.off, off0, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    CKA(h, cudaMemcpyAsync(s0.vx, vx0, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    CKA(h, cudaMemsetAsync(h->arena + h->L.obj, 0, 16 * (size_t)K, s));
    // field of level 0
    AdjFwd A;
    A.in = s0;
    A.out = s0;
    A.e_in = nullptr;
    A.e_out = e_table(h, 0);
    A.obj = (double *)(h->arena + h->L.obj_scratch);
    A.np = N;
    A.level = h->cfg.step0;
    CKA(h, launch_adj_fwd(run_with_volt(h), A, false, h->grid, s));
    for (long long k = 0; k < K; ++k) {
        const int r = forward_step(h, k, true);
        if (r) return r;
    }
    h->obj_host.assign(2 * (size_t)K, 0.0);
    CKA(h, cudaMemcpyAsync(h->obj_host.data(), h->arena + h->L.obj, 16 * (size_t)K, cudaMemcpyDeviceToHost, s));
    CKA(h, cudaStreamSynchronize(s));
    double p = 0.0, g = 0.0;
    for (long long k = 0; k < K; ++k) {
        p += h->obj_host[2 * k];
        g += h->obj_host[2 * k + 1];
    }
    power_flux[0] = p / (double)K;
    power_flux[1] = g / (double)K;
    h->have_forward = true;
    h->seg_valid = (K - 1) / h->L.C;
    return PIC_OK;
}

int pic_adj_backward(pic_adj *h, double c_power, double c_flux, float *d_vx0, float *d_x0, double *d_volt) {
    if (!h || !d_vx0) return fail_a(h, PIC_EINVAL, "pic_adj_backward: NULL argument");
    if (!h->have_forward) return fail_a(h, PIC_EINVAL, "pic_adj_backward: no forward run");
    if (!std::isfinite(c_power) || !std::isfinite(c_flux))
        return fail_a(h, PIC_EINVAL, "pic_adj_backward: weights not finite");
    const AdjLayout &L = h->L;
    const long long K = h->cfg.nsteps, N = h->cfg.n_particles, C = L.C;
    cudaStream_t s = h->stream;
    CKA(h, cudaMemsetAsync(h->arena + L.lx, 0, L.arr, s));
    CKA(h, cudaMemsetAsync(h->arena + L.lv, 0, L.arr, s));
    CKA(h, cudaMemsetAsync(h->arena + L.le, 0, 8 * ((size_t)h->cfg.n_cells + 3), s));
    CKA(h, cudaMemsetAsync(h->arena + L.dv0, 0, 8, s));
    const Run R = run_with_volt(h);
    AdjRev A;
    std::memset(&A, 0, sizeof A);
    A.lx = (float *)(h->arena + L.lx);
    A.lv = (float *)(h->arena + L.lv);
    A.le = (double *)(h->arena + L.le);
    A.dv0 = (double *)(h->arena + L.dv0);
    A.np = N;
    A.c_pw = (float)(c_power / (double)K);
    A.c_fl = (float)(c_flux / (double)K);
    A.w_dx = (float)(R.weight * R.inv_dx);
    A.lam_scale = 1.602176634e-19 * R.weight / 8.8541878128e-12;
    float *lam[2] = {(float *)(h->arena + L.lam[0]), (float *)(h->arena + L.lam[1])};
    for (long long seg = (K - 1) / C; seg >= 0; --seg) {
        const long long lo = seg * C, hi = (lo + C < K) ? lo + C : K;
        if (h->seg_valid != seg) {
            // inner levels lo+1 .. hi-1, and level hi itself when it is not a checkpoint
            const long long last = hi % C == 0 ? hi - 1 : hi;
            for (long long k = lo; k < last; ++k) {
                const int r = forward_step(h, k, false);
                if (r) return r;
            }
            h->seg_valid = seg;
        }
        for (long long n = hi - 1; n >= lo; --n) {
            A.lo = slot_of(h, n);
            A.hi = slot_of(h, n + 1);
            A.e = e_table(h, n);
            A.lam_in = n + 1 < K ? lam[(n + 1) & 1] : nullptr;
            A.lam_out = lam[n & 1];
            A.level = h->cfg.step0 + n;
            A.a_part = 1;
            CKA(h, launch_adj_rev(R, A, h->grid, s));
        }
    }
    // charge assignment of level 0
    A.lo = slot_of(h, 0);
    A.hi = slot_of(h, 0);
    A.e = nullptr;
    A.lam_in = lam[0];
    A.lam_out = nullptr;
    A.level = h->cfg.step0;
    A.a_part = 0;
    CKA(h, launch_adj_rev(R, A, h->grid, s));
    CKA(h, cudaMemcpyAsync(d_vx0, A.lv, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    if (d_x0) CKA(h, cudaMemcpyAsync(d_x0, A.lx, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    double dv = 0.0;
    CKA(h, cudaMemcpyAsync(&dv, A.dv0, 8, cudaMemcpyDeviceToHost, s));
    CKA(h, cudaStreamSynchronize(s));
    if (d_volt) *d_volt = dv;
    return PIC_OK;
}

int pic_adj_final_state(pic_adj *h, int32_t *cell, float *off, float *vx) {
    if (!h || !cell || !off || !vx) return fail_a(h, PIC_EINVAL, "pic_adj_final_state: NULL argument");
    if (!h->have_forward) return fail_a(h, PIC_EINVAL, "pic_adj_final_state: no forward run");
    const long long K = h->cfg.nsteps, N = h->cfg.n_particles;
    if (K % h->L.C != 0 && h->seg_valid != (K - 1) / h->L.C)
        return fail_a(h, PIC_EINVAL, "pic_adj_final_state: the last level was overwritten by a backward run");
    const AdjSlot sl = slot_of(h, K);
    cudaStream_t s = h->stream;
    CKA(h, cudaMemcpyAsync(cell, sl.cell, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
    CKA(h, cudaMemcpyAsync(off, sl.off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
    CKA(h, cudaMemcpyAsync(vx, sl.vx, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
    CKA(h, cudaStreamSynchronize(s));
    return PIC_OK;
}

void pic_adj_free(pic_adj *h) { delete h; }

}  // extern "C"
