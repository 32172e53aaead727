// pic_kernels.cu -- sm_103a kernels of the energy-conserving PIC/MCC step.
//
// One step of the explicit schemes (Sec. 2, schemes (1) and (2)) is ONE launch
// of k_particles: every block streams a contiguous chunk of particles from HBM
// (structure of arrays, one 4-byte word per field), gathers the field from a
// shared-memory copy of the grid, pushes, tests the electrodes, draws its
// null-collision decision from Philox keyed on (id, step), collides the few
// selected particles, and assigns its charge into per-block shared-memory
// accumulators in integer fixed point.  The last block to finish (atomic
// arrival counter) runs the tail of the step: places the step's births in
// parent-id order, assembles the node charge exactly in int64, solves the
// field equation and updates the diagnostics.  The direct-implicit scheme
// (Sec. 2, scheme (4)) is two such launches (predictor + corrector).
#include "pic_internal.h"

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

namespace pic {

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies with the published multipliers, key bumped by the
// published Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                       (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same rounds with the ten round keys precomputed per run (no key
// arithmetic in the loop; the keys sit in the kernel's parameter bank).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk0)[10],
                                                  const uint32_t (&rk1)[10]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r], (uint32_t)p0);
    }
    return c;
}

constexpr uint32_t kTagLoad = 1u;
constexpr uint32_t kTagMcc = 2u;
constexpr uint32_t kTagWait = 3u;

// Counter layout: (id, step low word, step high word, species<<24 | tag<<16 | sub).
__device__ __forceinline__ uint4 draw(const Run &R, uint32_t id, long long step, int species,
                                      uint32_t tag, uint32_t sub) {
    const unsigned long long s = (unsigned long long)step;
    return philox4x32_10_rk(make_uint4(id, (uint32_t)s, (uint32_t)(s >> 32),
                                       ((uint32_t)species << 24) | (tag << 16) | sub),
                            R.rk0, R.rk1);
}

// ---------------------------------------------------------------------------
// Null-collision selection by waiting times.  One Bernoulli(P_null) trial per
// particle and step is replaced by its equivalent: the steps W between a
// particle's selections (or from its entry into the run) follow the geometric
// law P(W > k) = (1 - P_null)^k, drawn once per selection.  W - 1 =
// 4096 a + 64 b + c with three independent digits, each the number of
// thresholds of its table (computed on the host) above one 32-bit Philox word;
// a = 64 stands for a wait beyond 64^3 steps, which ends in a fresh draw.  The
// push only counts down the wait held in the cell word's upper bits.
// ---------------------------------------------------------------------------
// Number of entries of the non-increasing table t[0, n) above u.
__device__ __forceinline__ uint32_t wait_digit(const uint32_t *t, int n, uint32_t u) {
    int lo = 0, hi = n;  // t[j] > u for j < lo; t[j] <= u for j >= hi
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < t[mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    return (uint32_t)lo;
}

// The wait of particle `id` of species S drawn at `step` (sub 0: after a
// selection; 1: on entering the run), kRedrawBit set when the count ends in
// a fresh draw instead of a selection.  tab: the run's [2][3][64] thresholds
// (a shared-memory copy in the particle launches: each digit is a chain of
// dependent reads).
__device__ __forceinline__ uint32_t draw_wait(const Run &R, const uint32_t *tab, int S, uint32_t id, long long step,
                                              uint32_t sub) {
    if (!R.thr[S]) return kWaitCap | kRedrawBit;  // P_null = 0: never selected
    const uint4 w = draw(R, id, step, S, kTagWait, sub);
    const uint32_t *t = tab + S * 192;
    const uint32_t a = wait_digit(t + 128, 64, w.x);
    if (a == 64u) return kWaitCap | kRedrawBit;
    const uint32_t b = wait_digit(t + 64, 63, w.y);
    const uint32_t c = wait_digit(t, 63, w.z);
    return 1u + 4096u * a + 64u * b + c;
}

// The upper bits of a cell word that holds the wait w.
__device__ __forceinline__ uint32_t wait_bits(uint32_t w) {
    return ((w & ~kRedrawBit) << kCellBits) | (w & kRedrawBit);
}

// Uniform on (0, 1) from the top 24 bits k of a word: u = (k + 1/2) 2^-24.
__device__ __forceinline__ float u24(uint32_t w) {
    return fmaf((float)(w >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
}

// The same uniform with its complement 1 - u = (2^24 - 1 - k + 1/2) 2^-24,
// each formed from its own integer with one rounding.  u needs 25 bits once
// k >= 2^23, so 1.0f - u24(w) would carry an absolute error of 2^-25: near
// u = 1 that is a large relative error of 1 - u, which sqrt(u (1 - u)) and
// log(u) magnify (a back-scattered direction, a small Box-Muller radius).
struct U24 {
    float u, c;  // u and 1 - u
};

__device__ __forceinline__ U24 u24c(uint32_t w) {
    const uint32_t k = w >> 8;
    return {fmaf((float)k, 5.9604644775390625e-8f, 2.98023223876953125e-8f),
            fmaf((float)(0xFFFFFFu - k), 5.9604644775390625e-8f, 2.98023223876953125e-8f)};
}

// sin and cos of 2 pi u, from whichever of u, 1 - u is below one half.
__device__ __forceinline__ void sincos_2pi(const U24 &x, float &s, float &c) {
    if (x.u <= 0.5f) {
        sincospif(2.0f * x.u, &s, &c);
    } else {
        sincospif(2.0f * x.c, &s, &c);
        s = -s;
    }
}

// -log(u), through log1p(-(1 - u)) above one half.
__device__ __forceinline__ float neg_log_u(const U24 &x) {
    return x.u <= 0.5f ? -logf(x.u) : -log1pf(-x.c);
}

// Box-Muller: two uniforms -> two standard normals.
__device__ __forceinline__ void box_muller(const U24 &u1, const U24 &u2, float &n1, float &n2) {
    const float r = sqrtf(2.0f * neg_log_u(u1));
    float s, c;
    sincos_2pi(u2, s, c);
    n1 = r * c;
    n2 = r * s;
}

// Turn the unit vector d by polar angle chi and azimuth phi, the azimuth
// measured in the basis of d's polar angles about the x axis.
__device__ __forceinline__ void rotate(float dx_, float dy, float dz, float cos_chi, float sin_chi,
                                       float sp, float cp, float &ox, float &oy, float &oz) {
    const float st = sqrtf(dy * dy + dz * dz);
    if (st > 1e-6f) {
        const float inv = 1.0f / st;
        ox = cos_chi * dx_ - sin_chi * cp * st;
        oy = cos_chi * dy + sin_chi * (cp * dx_ * dy - sp * dz) * inv;
        oz = cos_chi * dz + sin_chi * (cp * dx_ * dz + sp * dy) * inv;
    } else {
        ox = cos_chi * dx_;
        oy = sin_chi * cp * dx_;
        oz = sin_chi * sp;
    }
}

__device__ __forceinline__ float sigma_exc(const Run &R, float eps) {
    if (eps < R.exc_thr) return 0.0f;
    if (eps < R.exc_ramp_end) return R.exc_slope * (eps - R.exc_thr);
    return R.sig_exc_max;
}

__device__ __forceinline__ float sigma_iz(const Run &R, float eps) {
    if (eps <= R.iz_thr) return 0.0f;
    return R.sig_iz_k * (R.iz_thr / eps) * logf(eps / R.iz_thr);
}

// Per-thread counters of one species segment.
struct Tally {
    float kx, pw;
    unsigned int el, ex, iz, cx, nul, ovf_e, ovf_i;  // collisions of both species; overflow per species
};

// 1 - cos chi and 1 + cos chi of the Vahedi-Surendra law at energy eps [eV]
// for the uniform x: cos chi = (2 + eps - 2 (1 + eps)^u) / eps, written as
// 1 - cos chi = 2 expm1(u L) / eps and 1 + cos chi = -2 (1 + eps)
// expm1(-(1 - u) L) / eps with L = log1p(eps), so neither end cancels.
__device__ __forceinline__ void vs_angle(float eps, const U24 &x, float &dm, float &dp) {
    if (!(eps > 1e-6f)) {  // the isotropic limit
        dm = 2.0f * x.u;
        dp = 2.0f * x.c;
        return;
    }
    const float L = log1pf(eps), inv = 2.0f / eps;
    dm = expm1f(x.u * L) * inv;
    dp = -(1.0f + eps) * expm1f(-x.c * L) * inv;
}

// Opal-Pollock-Wagner: the secondary electron's share of an ionisation's
// excess, B tan(u arctan(excess / 2B)).
__device__ __forceinline__ float opal_secondary(float excess, float b, float u) {
    return excess > 0.0f ? b * tanf(u * atanf(excess / (2.0f * b))) : 0.0f;
}

// Electron collision (null-collision MC): elastic, excitation or ionisation
// chosen by u * nu_max against the running sum of n_g sigma_k(eps) v.
// Kept out of line: only the few selected particles take this path.
// Returns true if the velocity changed.
__device__ __forceinline__ bool collide_electron_body(const Run &R, uint4 w, uint32_t id, long long step,
                                                     int cell, float off, float abar, float &vx, float &vy,
                                                     float &vz, Tally &t) {
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float g = sqrtf(v2);
    const float eps = R.half_m_over_e[0] * v2;
    if (eps > R.eps_cap) t.ovf_e++;
    const float r = u24(w.y) * R.nu_max_e;
    const float ngv = R.n_g * g;
    const float nu_el = R.sig_el * ngv;
    const float nu_ex = sigma_exc(R, eps) * ngv;
    const float nu_iz = sigma_iz(R, eps) * ngv;
    const U24 uc = u24c(w.z);
    float sp, cp;
    sincos_2pi(u24c(w.w), sp, cp);
    float dx_ = 1.0f, dy = 0.0f, dz = 0.0f;
    if (g > 0.0f) {
        const float inv = 1.0f / g;
        dx_ = vx * inv;
        dy = vy * inv;
        dz = vz * inv;
    }
    // the angle: isotropic, cos chi = 1 - 2u = (1 - u) - u, sin chi =
    // 2 sqrt(u (1 - u)); or the Vahedi-Surendra law at energy e_ang
    float e_ang, g_new;
    if (r < nu_el) {
        // elastic: the electron keeps 1 - (2m/M)(1 - cos chi) of its energy;
        // the law is taken at the incident energy
        e_ang = eps;
        t.el++;
    } else if (r < nu_el + nu_ex) {
        e_ang = eps - R.exc_thr;
        g_new = sqrtf(R.two_e_over_me * e_ang);
        t.ex++;
    } else if (r < nu_el + nu_ex + nu_iz) {
        // Reading: the excess eps - I is shared equally by the two electrons
        // (or the secondary takes the Opal-Pollock-Wagner share), each
        // scattered at the energy it leaves with; the ion comes from the gas.
        // The births slot is taken first: the atomic's round trip overlaps
        // the draws and the kinematics below.
        const unsigned int slot = atomicAdd(&R.st->n_births, 1u);
        const uint4 w1 = draw(R, id, step, 0, kTagMcc, 1);
        const uint4 w2 = draw(R, id, step, 0, kTagMcc, 2);
        const float excess = eps - R.iz_thr;
        const float e_sec = R.iz_opal ? opal_secondary(excess, R.iz_b, u24(w2.z)) : 0.5f * excess;
        e_ang = R.iz_opal ? excess - e_sec : 0.5f * excess;
        g_new = sqrtf(R.two_e_over_me * e_ang);
        const float g_sec = sqrtf(R.two_e_over_me * e_sec);
        const U24 u1 = u24c(w1.x);
        float sps, cps;
        sincos_2pi(u24c(w1.y), sps, cps);
        float sx, sy, sz;
        if (R.scatter_vs) {  // turned from the incident direction
            float dm, dp;
            vs_angle(e_sec, u1, dm, dp);
            rotate(dx_, dy, dz, 0.5f * (dp - dm), sqrtf(dm * dp), sps, cps, sx, sy, sz);
        } else {  // isotropic in the laboratory frame
            const float st = 2.0f * sqrtf(u1.u * u1.c);
            sx = u1.c - u1.u;
            sy = st * cps;
            sz = st * sps;
        }
        float n1, n2, n3, n4;
        box_muller(u24c(w1.z), u24c(w1.w), n1, n2);
        box_muller(u24c(w2.x), u24c(w2.y), n3, n4);
        if (slot < (unsigned int)R.births_cap) {
            Birth b;
            b.pid = id;
            b.cell = cell;
            b.off = off;
            b.abar_e = abar;
            b.ve[0] = g_sec * sx;
            b.ve[1] = g_sec * sy;
            b.ve[2] = g_sec * sz;
            b.vi[0] = R.vth_gas * n1;
            b.vi[1] = R.vth_gas * n2;
            b.vi[2] = R.vth_gas * n3;
            R.births[slot] = b;
        }
        t.iz++;
    } else {
        t.nul++;
        return false;
    }
    float cos_chi, sin_chi;
    if (R.scatter_vs) {
        float dm, dp;
        vs_angle(e_ang, uc, dm, dp);
        cos_chi = 0.5f * (dp - dm);
        sin_chi = sqrtf(dm * dp);
        if (r < nu_el) g_new = g * sqrtf(1.0f - R.two_m_over_M * dm);
    } else {
        cos_chi = uc.c - uc.u;
        sin_chi = 2.0f * sqrtf(uc.u * uc.c);
        if (r < nu_el) g_new = g * sqrtf(1.0f - R.two_m_over_M * (2.0f * uc.u));
    }
    float ox, oy, oz;
    rotate(dx_, dy, dz, cos_chi, sin_chi, sp, cp, ox, oy, oz);
    vx = g_new * ox;
    vy = g_new * oy;
    vz = g_new * oz;
    return true;
}

// Ion charge exchange against a neutral sampled from the gas Maxwellian.
__device__ __forceinline__ bool collide_ion_body(const Run &R, uint4 w, uint32_t id, long long step,
                                                float &vx, float &vy, float &vz, Tally &t) {
    const uint4 w1 = draw(R, id, step, 1, kTagMcc, 1);
    float n1, n2, n3, n4;
    box_muller(u24c(w.z), u24c(w.w), n1, n2);
    box_muller(u24c(w1.x), u24c(w1.y), n3, n4);
    const float vnx = R.vth_gas * n1, vny = R.vth_gas * n2, vnz = R.vth_gas * n3;
    const float ux = vx - vnx, uy = vy - vny, uz = vz - vnz;
    const float g = sqrtf(ux * ux + uy * uy + uz * uz);
    if (g > R.g_max_i) t.ovf_i++;
    const float r = u24(w.y) * R.nu_max_i;
    if (r < R.n_g * R.sig_cx * g) {
        vx = vnx;
        vy = vny;
        vz = vnz;
        t.cx++;
        return true;
    }
    t.nul++;
    return false;
}

// A particle crossed an electrode (Sec. 3): tally its number and energy.
__device__ __forceinline__ void absorb_body(const Run &R, int S, int wall, float vx, float vy, float vz) {
    const float en = (S ? R.half_m_over_e[1] : R.half_m_over_e[0]) * (vx * vx + vy * vy + vz * vz);
    atomicAdd(&R.st->wall_count[S][wall], 1ull);
    atomicAdd(&R.st->wall_energy[S][wall], (double)en);
    atomicAdd(&R.st->absorbed_step[S], 1ull);
}

// Out-of-line copies for the batched kernel, whose register budget the
// inlined bodies would exceed; the single-run kernel inlines the bodies
// (out of line, the run's parameters would have to be copied to the stack).
__device__ __noinline__ bool collide_electron(const Run &R, uint4 w, uint32_t id, long long step, int cell, float off,
                                              float abar, float &vx, float &vy, float &vz, Tally &t) {
    return collide_electron_body(R, w, id, step, cell, off, abar, vx, vy, vz, t);
}

__device__ __noinline__ bool collide_ion(const Run &R, uint4 w, uint32_t id, long long step, float &vx, float &vy,
                                         float &vz, Tally &t) {
    return collide_ion_body(R, w, id, step, vx, vy, vz, t);
}

__device__ __noinline__ void absorb(const Run &R, int S, int wall, float vx, float vy, float vz) {
    absorb_body(R, S, wall, vx, vy, vz);
}

template <bool INL>
__device__ __forceinline__ bool collide_e(const Run &R, uint4 w, uint32_t id, long long step, int cell, float off,
                                          float abar, float &vx, float &vy, float &vz, Tally &t) {
    if (INL) return collide_electron_body(R, w, id, step, cell, off, abar, vx, vy, vz, t);
    return collide_electron(R, w, id, step, cell, off, abar, vx, vy, vz, t);
}

template <bool INL>
__device__ __forceinline__ bool collide_i(const Run &R, uint4 w, uint32_t id, long long step, float &vx, float &vy,
                                          float &vz, Tally &t) {
    if (INL) return collide_ion_body(R, w, id, step, vx, vy, vz, t);
    return collide_ion(R, w, id, step, vx, vy, vz, t);
}

template <bool INL>
__device__ __forceinline__ void absorb_p(const Run &R, int S, int wall, float vx, float vy, float vz) {
    if (INL)
        absorb_body(R, S, wall, vx, vy, vz);
    else
        absorb(R, S, wall, vx, vy, vz);
}

// ---------------------------------------------------------------------------
// Charge assignment in fixed point.  The offset is quantised to 16 bits,
// F = floor(off * 2^16).  S_2 (Eq. 2, m = 2): nearest node j and
// a = (1/2 + delta) 2^16; the nodes j-1, j, j+1 receive b^2, 2^33 - a^2 - b^2,
// a^2 (b = 2^16 - a), i.e. 2^33 times the quadratic spline weights.  Each
// particle is accumulated under its key j as (1, a, a^2); the node charges
// are reassembled exactly from these per-key sums in the tail.  S_1 (the
// momentum-conserving scheme): key = cell, value F.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int deposit_key_s2(int cell, float off, uint32_t &a) {
    const int F = (int)(off * 65536.0f);
    if (F < 32768) {
        a = (uint32_t)(F + 32768);
        return cell;
    }
    a = (uint32_t)(F - 32768);
    return cell + 1;
}

__device__ __forceinline__ int deposit_key_s1(int cell, float off, uint32_t &a) {
    a = (uint32_t)(int)(off * 65536.0f);
    return cell;
}

// m = 3 (Eq. 2 with the cubic S_3, four nodes): key = cell, value the 12-bit
// code F = floor(off * 2^12).  With t = F / 2^12 the nodes cell-1 .. cell+2
// receive 6 * 2^36 times (1-t)^3/6, (3t^3-6t^2+4)/6, (-3t^3+3t^2+3t+1)/6 and
// t^3/6, integer polynomials in F; the per-key sums (1, F, F^2, F^3) give the
// node charges exactly (node_charge_s3_raw), in units of 2^-36/6.
__device__ __forceinline__ int deposit_key_s3(int cell, float off, uint32_t &a) {
    a = (uint32_t)(int)(off * 4096.0f);
    return cell;
}

// Per-block accumulators, four 32-bit counters per key: count, sum of a, and
// the sums of the high and low 16 bits of a^2.  Exact while a block adds at
// most 2^16 particles between two flushes (each term is below 2^16).  The
// m = 3 modes keep every sum in 32-bit counters too (native shared atomics):
// cnt, a (sum of F < 2^12), bh and bl (the sum of F^2 in 12-bit pieces of
// warp sums: sum = bh 2^12 + bl) and s3h, s3m, s3l (the sum of F^3 in the
// three 12-bit pieces of each F^3 < 2^36); each stays below 2^28 per flush.
struct Acc {
    unsigned int *cnt, *a, *bh, *bl;
    unsigned int *s3h, *s3m, *s3l;
};

constexpr long long kFlushEvery = 65536;

__device__ __forceinline__ void acc_add(const Acc &acc, int key, uint32_t c, uint32_t a, uint32_t bh,
                                        uint32_t bl, bool count_only) {
    atomicAdd(&acc.cnt[key], c);
    if (!count_only) {
        atomicAdd(&acc.a[key], a);
        atomicAdd(&acc.bh[key], bh);
        atomicAdd(&acc.bl[key], bl);
    }
}

// m = 3: per key of the warp's window (see deposit_tile below) the count
// and the sum of F packed in one word (below 2^8 and 2^20 over a warp), the
// sum of F^2 (below 2^31) and the three 12-bit pieces of each F^3 < 2^36
// summed apart (each below 2^19); the sum of F^2 is split into 12-bit pieces
// when added to the block's 32-bit counters.
__device__ __forceinline__ void acc_add3(const Acc &acc, int key, uint32_t c, uint32_t a, uint32_t s2,
                                         uint32_t s3h, uint32_t s3m, uint32_t s3l) {
    atomicAdd(&acc.cnt[key], c);
    atomicAdd(&acc.a[key], a);
    atomicAdd(&acc.bh[key], s2 >> 12);
    atomicAdd(&acc.bl[key], s2 & 0xfffu);
    atomicAdd(&acc.s3h[key], s3h);
    atomicAdd(&acc.s3m[key], s3m);
    atomicAdd(&acc.s3l[key], s3l);
}

constexpr int kDepWindow = 4;

__device__ __forceinline__ void deposit_tile3(const int (&key)[kUnroll], const uint32_t (&a)[kUnroll],
                                              const Acc &acc) {
    const int lane = threadIdx.x & 31;
    int lo = 0x7fffffff, hi = -1;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
        if (key[u] >= 0) {
            lo = min(lo, key[u]);
            hi = max(hi, key[u]);
        }
    const int K1 = __reduce_max_sync(FULL_MASK, hi);
    if (K1 < 0) return;
    const int K0 = __reduce_min_sync(FULL_MASK, lo);
    const int D = K1 - K0 + 1;
    if (D > kDepWindow) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (key[u] >= 0) {
                const uint32_t f = a[u], f2 = f * f;
                const unsigned long long f3 = (unsigned long long)f2 * f;
                acc_add3(acc, key[u], 1u, f, f2, (uint32_t)(f3 >> 24), (uint32_t)(f3 >> 12) & 0xfffu,
                         (uint32_t)f3 & 0xfffu);
            }
        return;
    }
    uint32_t m_cf = 0u, m_s2 = 0u, m_h = 0u, m_m = 0u, m_l = 0u;
#pragma unroll
    for (int d = 0; d < kDepWindow; ++d) {
        if (d >= D) break;
        uint32_t cf = 0u, s2 = 0u, h = 0u, mm = 0u, l = 0u;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (key[u] == K0 + d) {
                const uint32_t f = a[u], f2 = f * f;
                const unsigned long long f3 = (unsigned long long)f2 * f;
                cf += (f << 8) | 1u;
                s2 += f2;
                h += (uint32_t)(f3 >> 24);
                mm += (uint32_t)(f3 >> 12) & 0xfffu;
                l += (uint32_t)f3 & 0xfffu;
            }
        cf = __reduce_add_sync(FULL_MASK, cf);
        s2 = __reduce_add_sync(FULL_MASK, s2);
        h = __reduce_add_sync(FULL_MASK, h);
        mm = __reduce_add_sync(FULL_MASK, mm);
        l = __reduce_add_sync(FULL_MASK, l);
        if (lane == d) {
            m_cf = cf;
            m_s2 = s2;
            m_h = h;
            m_m = mm;
            m_l = l;
        }
    }
    if (lane < D && (m_cf & 0xffu)) acc_add3(acc, K0 + lane, m_cf & 0xffu, m_cf >> 8, m_s2, m_h, m_m, m_l);
}

// Deposit of a warp's tile share (32 x kUnroll particles).  Kept sorted by
// key between sorts, a warp's particles span a narrow window of keys: the
// ions one or two, the electrons (which cross about a tenth of a cell a
// step) a few more.  The warp finds its window [K0, K1] with two
// reductions, sums each key of the window across the warp (count and sum of
// a packed in one word, the halves of a^2 in two), and lane d adds key
// K0 + d: one set of shared atomics per warp, on consecutive words.  A
// warp spread wider than kDepWindow keys adds particle by particle.

__device__ __forceinline__ void deposit_tile(const int (&key)[kUnroll], const uint32_t (&a)[kUnroll],
                                             const Acc &acc, bool count_only) {
    const int lane = threadIdx.x & 31;
    int lo = 0x7fffffff, hi = -1;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
        if (key[u] >= 0) {
            lo = min(lo, key[u]);
            hi = max(hi, key[u]);
        }
    const int K1 = __reduce_max_sync(FULL_MASK, hi);
    if (K1 < 0) return;  // no particle in the warp
    const int K0 = __reduce_min_sync(FULL_MASK, lo);
    const int D = K1 - K0 + 1;
    if (D > kDepWindow) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (key[u] >= 0) {
                const uint32_t q = a[u] * a[u];
                acc_add(acc, key[u], 1u, a[u], q >> 16, q & 0xffffu, count_only);
            }
        return;
    }
    // per lane: count <= kUnroll and a < 2^16, so over the warp the count
    // stays below 2^8 and the sum of a below 2^23: (sum a) << 8 | count is
    // exact in 32 bits; each half of a^2 sums below 2^23
    uint32_t m_ca = 0u, m_h = 0u, m_l = 0u;
#pragma unroll
    for (int d = 0; d < kDepWindow; ++d) {
        if (d >= D) break;  // the same in every lane
        uint32_t ca = 0u, h = 0u, l = 0u;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (key[u] == K0 + d) {
                ca += (a[u] << 8) | 1u;
                if (!count_only) {
                    const uint32_t q = a[u] * a[u];
                    h += q >> 16;
                    l += q & 0xffffu;
                }
            }
        ca = __reduce_add_sync(FULL_MASK, ca);
        if (!count_only) {
            h = __reduce_add_sync(FULL_MASK, h);
            l = __reduce_add_sync(FULL_MASK, l);
        }
        if (lane == d) {
            m_ca = ca;
            m_h = h;
            m_l = l;
        }
    }
    if (lane < D && (m_ca & 0xffu)) acc_add(acc, K0 + lane, m_ca & 0xffu, m_ca >> 8, m_h, m_l, count_only);
}

// ---------------------------------------------------------------------------
// Block-wide scans and sums (kThreads threads).
// ---------------------------------------------------------------------------
template <typename T>
__device__ T block_exclusive_scan(T v, T *scratch /*[33]*/, T &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int nw = kThreads / 32;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(FULL_MASK, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) scratch[lane] = s;
    }
    __syncthreads();
    const T before = wid > 0 ? scratch[wid - 1] : T(0);
    total = scratch[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Exclusive prefix of x over the block; y is replaced by its block total.
__device__ double block_exclusive_scan2(double x, double &y, double *scratch /*[2*kThreads/32]*/) {
    constexpr int nw = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += t;
    }
    const double ys = warp_sum(y);
    if (lane == 31) scratch[wid] = inc;
    if (lane == 0) scratch[nw + wid] = ys;
    __syncthreads();
    double before = 0.0, ytot = 0.0;
    for (int k = 0; k < nw; ++k) {
        if (k < wid) before += scratch[k];
        ytot += scratch[nw + k];
    }
    __syncthreads();
    y = ytot;
    return before + inc - x;
}

// Sum of two doubles over the block (one barrier pair).
__device__ void block_sum2(double &x, double &y, double *scratch /*[2*kThreads/32]*/) {
    constexpr int nw = kThreads / 32;
    x = warp_sum(x);
    y = warp_sum(y);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        scratch[wid] = x;
        scratch[nw + wid] = y;
    }
    __syncthreads();
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < nw; ++k) {
        sx += scratch[k];
        sy += scratch[nw + k];
    }
    __syncthreads();
    x = sx;
    y = sy;
}

// ---------------------------------------------------------------------------
// Shared-memory layout of the particle kernels.
// ---------------------------------------------------------------------------
// Deferred collisions: particles whose wait ran out in the push wait here
// (their slot and species; kQueueRedraw marks a count that only ends in a
// fresh draw of the wait) and are collided later by full warps, which read
// their ids and draw their Philox words and next waits.  The queue is
// drained before a tile whenever fewer than a tile's worth of entries are
// free, so it cannot overflow, and at the end of the block's stream; a
// block's switch from electrons to ions leaves it as it is.  Slots are below
// 2^29.
#ifndef PIC_QDRAIN
#define PIC_QDRAIN 128
#endif
constexpr unsigned int kQueueDrainAbove = PIC_QDRAIN;
constexpr int kQueue = (int)kQueueDrainAbove + kThreads * kUnroll;  // + one tile
constexpr uint32_t kQueueRedraw = 0x80000000u;  // in a queue entry: no collision, only a new wait
constexpr uint32_t kQueueIon = 0x40000000u;     // in a queue entry: an ion
struct CollQueue {
    uint32_t *slot;            // [cap] slot | kQueueIon | kQueueRedraw
    unsigned int *n;           // entries queued
    unsigned int cap;          // entries the queue holds
};

struct SmemMain {
    float *e;                  // [n+2] gather table
    Acc acc;                   // 4 x [n+1] (m = 3: and a 64-bit [n+1])
    float *heat;               // [n]
    unsigned int *eedf;        // [bins+1]
    CollQueue q;
    const uint32_t *wtab;      // [2][3][64] waiting-time thresholds (static shared memory)
    float2 *hw;                // non-uniform grid: [n] (h_c, 1/h_c)
};

constexpr int kWaitTab = 2 * 3 * 64;

// The run's waiting-time thresholds into shared memory (every thread calls
// this before a barrier).
__device__ __forceinline__ void load_wait_tab(const Run &R, uint32_t *dst) {
    if (!R.mcc) return;
    for (int k = threadIdx.x; k < kWaitTab; k += kThreads) dst[k] = R.wait_tab[k];
}

__host__ __device__ inline size_t align8(size_t x) { return (x + 7) & ~size_t(7); }

__host__ __device__ inline size_t main_smem_bytes(int n, int bins, bool ec3, bool nu = false) {
    return align8(4 * (size_t)(n + 2)) + (ec3 ? 7 : 4) * align8(4 * (size_t)(n + 1)) +
           align8(4 * (size_t)n) + align8(4 * (size_t)(bins + 1)) + 4 * (size_t)kQueue + 16 +
           (nu ? 8 + 8 * (size_t)n : 0);
}

// The tail's scratch: the field solve's arrays (32 bytes a node), or, before
// them, the births ranking's 2048-bucket histogram.
__host__ __device__ inline size_t tail_smem_bytes(int n) {
    const size_t field = 32 * (size_t)(n + 1), births = 4 * 2048;
    return field > births ? field : births;
}

// The last block's tail reuses the whole dynamic shared memory (ring and grid
// are idle by then): the staged per-key sums (6 x 8 bytes a key, 8 x 8 for
// m = 3) first, the tail's scratch after them.
__host__ __device__ inline size_t tail_stage_bytes(int n, bool ec3 = false) {
    return ((size_t)(ec3 ? 64 : 48) * (n + 1) + 255) & ~size_t(255);
}

__device__ SmemMain carve_main(unsigned char *base, int n, int bins, bool ec3, const uint32_t *wtab,
                               bool nu = false) {
    SmemMain s;
    s.wtab = wtab;
    s.hw = nullptr;
    size_t o = 0;
    s.e = (float *)(base + o);
    o += align8(4 * (size_t)(n + 2));
    unsigned int **slots[4] = {&s.acc.cnt, &s.acc.a, &s.acc.bh, &s.acc.bl};
    for (int k = 0; k < 4; ++k) {
        *slots[k] = (unsigned int *)(base + o);
        o += align8(4 * (size_t)(n + 1));
    }
    s.acc.s3h = s.acc.s3m = s.acc.s3l = nullptr;
    if (ec3) {
        unsigned int **s3[3] = {&s.acc.s3h, &s.acc.s3m, &s.acc.s3l};
        for (int k = 0; k < 3; ++k) {
            *s3[k] = (unsigned int *)(base + o);
            o += align8(4 * (size_t)(n + 1));
        }
    }
    s.heat = (float *)(base + o);
    o += align8(4 * (size_t)n);
    s.eedf = (unsigned int *)(base + o);
    o += align8(4 * (size_t)(bins + 1));
    s.q.slot = (uint32_t *)(base + o);
    o += 4 * (size_t)kQueue;
    s.q.n = (unsigned int *)(base + o);
    s.q.cap = (unsigned int)kQueue;
    if (nu) s.hw = (float2 *)(base + align8(o + 16));
    return s;
}

template <int MODE>
struct ModeInfo {
    static constexpr bool pass1 = (MODE == kImplicit1 || MODE == kImplicit1MC || MODE == kImplicit1NU);
    static constexpr bool pass2 = (MODE == kImplicit2 || MODE == kImplicit2MC || MODE == kImplicit2NU);
    static constexpr bool ec3 = (MODE == kExplicitEC3 || MODE == kDepositEC3 || MODE == kExplicitEC3NU);
    // non-uniform grid
    static constexpr bool nu = (MODE == kExplicitNU || MODE == kImplicit1NU || MODE == kImplicit2NU ||
                                MODE == kExplicitEC3NU);
    static constexpr bool deposit = (MODE == kDepositEC || MODE == kDepositMC || MODE == kDepositEC3);
    static constexpr bool push = !(deposit || pass1);
    static constexpr bool needs_field = (MODE == kExplicitEC || MODE == kExplicitMC || MODE == kExplicitEC3 ||
                                         MODE == kExplicitNU || MODE == kExplicitEC3NU || pass2);
    static constexpr bool implicit = pass1 || pass2;
    static constexpr bool count_only = pass2;
    static constexpr bool mc = (MODE == kExplicitMC || MODE == kDepositMC || MODE == kImplicit1MC ||
                                MODE == kImplicit2MC);
    static constexpr bool loads_v = !deposit;
    static constexpr bool explicit_push = (MODE == kExplicitEC || MODE == kExplicitMC || MODE == kExplicitEC3 ||
                                           MODE == kExplicitNU || MODE == kExplicitEC3NU);
};

// Renormalise an offset that left [0, 1) into the cell index.
__device__ __forceinline__ void renormalise(int &c, float &s) {
    if (!(s >= 0.0f && s < 1.0f)) {
        const float fl = floorf(s);
        c += (int)fl;
        s -= fl;
        if (s >= 1.0f) {
            s = 0.0f;
            c += 1;
        }
    }
}

// A move by d metres on the non-uniform grid that leaves the particle's cell
// (c, s): walk cell by cell with the distance left, from the cell's left
// node (d >= 0) or right node (d < 0).  Returns 0 <= s < 1 inside the grid,
// or c = -1 / c = N past an electrode; wraps in the periodic box.  At most
// N + 2 cells are visited (|d| < L after the wrap or the electrode test).
// Inlined: as a call it took 1.6 % longer on the stretched benchmark grid,
// whose sheath electrons cross several cells a step.
__device__ __forceinline__ void walk_nu(const float2 *hw, int N, bool periodic, float len, int &c, float &s,
                                     float d) {
    constexpr float kBelowOne = 0.99999994f;  // the largest FP32 below 1
    if (periodic) {
        d = fmodf(d, len);
    } else if (!(fabsf(d) < len)) {  // beyond the gap (or not a number)
        c = d > 0.0f ? N : -1;
        s = 0.0f;
        return;
    }
    int k = c;
    if (d >= 0.0f) {
        float r = fmaf(s, hw[k].x, d);  // from the left node of cell k
        for (int it = 0; it < N + 2; ++it) {
            const float2 h = hw[k];
            if (r < h.x) {
                c = k;
                s = fminf(fmaxf(r * h.y, 0.0f), kBelowOne);
                return;
            }
            r -= h.x;
            if (++k == N) {
                if (!periodic) break;
                k = 0;
            }
        }
        c = N;  // past the right electrode
    } else {
        float l = fmaf(1.0f - s, hw[k].x, -d);  // back from the right node of cell k
        for (int it = 0; it < N + 2; ++it) {
            const float2 h = hw[k];
            if (l <= h.x) {
                c = k;
                s = fminf(fmaxf(1.0f - l * h.y, 0.0f), kBelowOne);
                return;
            }
            l -= h.x;
            if (--k < 0) {
                if (!periodic) break;
                k = N - 1;
            }
        }
        c = -1;  // past the left electrode
    }
    s = 0.0f;
}

// A move by d metres on the non-uniform grid from (c, s), hc = (h_c, 1/h_c):
// d / h_c of the cell while it stays inside; into the next cell over (the
// common crossing) from the two widths; further by the walk.
__device__ __forceinline__ void move_nu(const float2 *hw, int N, bool periodic, float len, int &c, float &s,
                                        float d, float2 hc) {
    const float off = s;
    s = fmaf(d, hc.y, off);
    if (s >= 0.0f && s < 1.0f) return;
    const bool right = s >= 1.0f;
    const int cn = right ? c + 1 : c - 1;
    if (cn >= 0 && cn < N) {
        const float hn_inv = hw[cn].y;
        const float t = right ? (s - 1.0f) * hc.x * hn_inv : fmaf(s * hc.x, hn_inv, 1.0f);
        if (t >= 0.0f && t < 1.0f) {
            c = cn;
            s = t;
            return;
        }
    }
    s = off;  // further: walk
    walk_nu(hw, N, periodic, len, c, s, d);
}

// EC force interpolation, Eq. (3) with m = 2: S_1 from the cell-centred field
// table e[] (e[k] = E of cell k-1; ghost cells beyond the walls hold zero).
__device__ __forceinline__ float gather_ec(const float *e, int cell, float off) {
    const int j = cell + (off >= 0.5f ? 1 : 0);
    const float w1 = off >= 0.5f ? off - 0.5f : off + 0.5f;  // 1/2 + delta
    return (1.0f - w1) * e[j] + w1 * e[j + 1];
}

// m = 3: S_2 from the centres of cells cell-1, cell, cell+1 (table entries
// cell .. cell+2), at distances 1/2 + t, |t - 1/2| and 3/2 - t.
__device__ __forceinline__ float gather_ec3(const float *e, int cell, float t) {
    const float u = 1.0f - t, d = t - 0.5f;
    return 0.5f * u * u * e[cell] + (0.75f - d * d) * e[cell + 1] + 0.5f * t * t * e[cell + 2];
}

__device__ __forceinline__ void eedf_sample(const Run &R, const SmemMain &sm, float vx, float vy, float vz) {
    const float en = R.half_m_over_e[0] * (vx * vx + vy * vy + vz * vz);
    int bin = (int)floorf(en * R.eedf_inv_width);
    bin = bin > R.eedf_bins ? R.eedf_bins : (bin < 0 ? 0 : bin);
    atomicAdd(&sm.eedf[bin], 1u);
}

// Collide the queued particles, one per thread, and draw their next waits.
// Their post-push cell word (count zero), position and velocity were stored
// before the barrier that precedes this call.  se, si: the arrays the
// queued slots of electrons and ions index.
template <bool INL>
__device__ __forceinline__ void drain_body(const Run &R, const SmemMain &sm, const Species &se, const Species &si,
                                           long long step, bool diag, Tally &t) {
    __syncthreads();
    const unsigned int nq = min(*sm.q.n, (unsigned int)kQueue);
    for (unsigned int q = threadIdx.x; q < nq; q += kThreads) {
        const uint32_t entry = sm.q.slot[q];
        const int S = (entry & kQueueIon) ? 1 : 0;
        const Species &sp = S ? si : se;
        const int idx = (int)(entry & ~(kQueueRedraw | kQueueIon));
        // every load first, so their latencies overlap
        const uint32_t id = sp.id[idx];
        const int c = sp.cell[idx] & (int)kCellMask;
        float vx = sp.vx[idx], vy = sp.vy[idx], vz = sp.vz[idx];
        const float off = sp.off[idx];
        const float abar = (S == 0 && sp.abar) ? sp.abar[idx] : 0.0f;
        if (!(entry & kQueueRedraw)) {  // selected: the collision's words
            const uint4 w = draw(R, id, step, S, kTagMcc, 0);
            bool changed;
            if (S == 0) {
                changed = collide_e<INL>(R, w, id, step, c, off, abar, vx, vy, vz, t);
            } else {
                changed = collide_i<INL>(R, w, id, step, vx, vy, vz, t);
            }
            if (changed) {
                sp.vx[idx] = vx;
                sp.vy[idx] = vy;
                sp.vz[idx] = vz;
            }
        }
        sp.cell[idx] = c | (int)wait_bits(draw_wait(R, sm.wtab, S, id, step, 0));
        if (S == 0 && diag && R.eedf_bins > 0) eedf_sample(R, sm, vx, vy, vz);
    }
    __syncthreads();
    if (threadIdx.x == 0) *sm.q.n = 0u;
    __syncthreads();
}

__device__ __noinline__ void drain_collisions(const Run &R, const SmemMain &sm, Species se, Species si,
                                              long long step, bool diag, Tally &t) {
    drain_body<false>(R, sm, se, si, step, diag, t);
}

template <bool INL>
__device__ __forceinline__ void drain_q(const Run &R, const SmemMain &sm, const Species &se, const Species &si,
                                        long long step, bool diag, Tally &t) {
    if (INL)
        drain_body<true>(R, sm, se, si, step, diag, t);
    else
        drain_collisions(R, sm, se, si, step, diag, t);
}

// The per-species constants of the push, selected once per tile: the
// particle code exists once for both species (two copies would double the
// hot loop's instruction footprint).
struct SpK {
    float qm, qw, qm_dt, mq;  // q/m, q w, (q/m) dt, m/q
    uint32_t collides;        // the species' P_null > 0
    int S;
};

__device__ __forceinline__ SpK species_k(const Run &R, int S) {
    return S ? SpK{R.qm[1], R.qw[1], R.qm_dt[1], R.mq[1], R.thr[1], 1}
             : SpK{R.qm[0], R.qw[0], R.qm_dt[0], R.mq[0], R.thr[0], 0};
}

// ---------------------------------------------------------------------------
// One particle of each mode.  `cell` is the particle's cell word (cell and,
// with collisions, its wait).  Returns its deposit key (-1: none) and value a.
// On return cell < 0 marks an absorbed particle.
// ---------------------------------------------------------------------------
template <int MODE, bool INL>
__device__ __forceinline__ int step_particle(const Run &R, const SmemMain &sm, const Species &sp, const SpK &k,
                                             long long idx, int &cell, float &off, float &vx,
                                             float &abar, bool diag, long long step,
                                             Tally &t, float &kx, float &pw, uint32_t &a_out) {
    using MI = ModeInfo<MODE>;
    const int N = R.n_cells;
    const int c0 = cell & (int)kCellMask;
    if (MODE == kDepositEC) return deposit_key_s2(c0, off, a_out);
    if (MODE == kDepositMC) return deposit_key_s1(c0, off, a_out);
    if (MODE == kDepositEC3) return deposit_key_s3(c0, off, a_out);
    const float v_old = vx;
    float e_field, v_new, s;
    int c = c0;
    if (MI::implicit) {
        // predictor: v~ = v + dt abar / 2, x~ = x + dt v~
        const float vt = fmaf(R.half_dt, abar, vx);
        bool inside = true;
        if (MI::nu) {
            // non-uniform grid: through the physical position (wraps in the
            // periodic box; c = -1 / N past an electrode)
            s = off;
            move_nu(sm.hw, N, R.periodic != 0, R.len_f, c, s, vt * R.dt_f, sm.hw[c0]);
            inside = c >= 0 && c < N;
        } else {
            s = fmaf(vt, R.dt_dx, off);
            if (!(fabsf(s) < 1.0e6f)) s = (float)(2 * N + 2);  // runaway: lands outside
            renormalise(c, s);
            if (R.periodic) {
                if (c < 0 || c >= N) c = ((c % N) + N) % N;
            } else if (c < 0 || c >= N) {
                inside = false;
            }
        }
        if (MI::pass1) {
            if (!inside) return -1;  // Reading: nothing assigned beyond an electrode
            return MI::mc ? deposit_key_s1(c, s, a_out) : deposit_key_s2(c, s, a_out);
        }
        // corrector with E^{n+1} at x~ (S_1 from the cell-centred field, or
        // linear from the node field of the momentum-conserving scheme; on a
        // non-uniform grid the voltage drops over x~'s own cell width)
        if (MI::nu) {
            e_field = !inside ? 0.0f : gather_ec(sm.e, c, s) * sm.hw[c].y;
        } else {
            e_field = !inside ? 0.0f
                              : (MI::mc ? (1.0f - s) * sm.e[c] + s * sm.e[c + 1] : gather_ec(sm.e, c, s));
        }
        const float acc = k.qm * e_field;
        v_new = fmaf(R.half_dt, acc, vt);
        if (!MI::nu) s = fmaf(acc, R.half_dt2_dx, s);
        abar = 0.5f * (abar + acc);
        // Reading: the step changes v by dt abar^n, so the work done on the
        // particle is that of the field (m/q) abar^n, not of E^{n+1}
        e_field = abar * k.mq;
        if (diag && inside) atomicAdd(&sm.heat[c], k.qw * e_field * 0.5f * (v_old + v_new));  // x~'s cell
        if (MI::nu && inside) move_nu(sm.hw, N, R.periodic != 0, R.len_f, c, s, acc * R.half_dt2, sm.hw[c]);
    } else if (MI::nu) {
        // non-uniform grid: the table holds the cells' voltage drops; the
        // force is their S_1 interpolation over the particle's own cell
        // width (the x-derivative of its potential energy), and the move of
        // v dt goes through the physical position
        const float2 hc = sm.hw[c0];
        e_field = (MI::ec3 ? gather_ec3(sm.e, c0, off) : gather_ec(sm.e, c0, off)) * hc.y;
        v_new = fmaf(k.qm_dt, e_field, vx);
        if (diag) atomicAdd(&sm.heat[c0], k.qw * e_field * 0.5f * (v_old + v_new));
        s = off;
        move_nu(sm.hw, N, R.periodic != 0, R.len_f, c, s, v_new * R.dt_f, hc);
    } else {
        // explicit leapfrog with E^n at x^n (Sec. 2 schemes (1), (2))
        e_field = MI::mc ? (1.0f - off) * sm.e[c0] + off * sm.e[c0 + 1]
                         : (MI::ec3 ? gather_ec3(sm.e, c0, off) : gather_ec(sm.e, c0, off));
        v_new = fmaf(k.qm_dt, e_field, vx);
        if (diag) atomicAdd(&sm.heat[c0], k.qw * e_field * 0.5f * (v_old + v_new));
        s = fmaf(v_new, R.dt_dx, off);
    }
    kx += 0.5f * (v_old * v_old + v_new * v_new);  // kept in registers: t lives in memory
    pw += k.qw * e_field * 0.5f * (v_old + v_new);
    if (!MI::nu) {
        if (!(fabsf(s) < 1.0e6f)) s = (float)(2 * N + 2);
        renormalise(c, s);
    }
    vx = v_new;
    off = s;
    // electrodes (Sec. 3) or periodic wrap
    if (R.periodic) {
        if (c < 0 || c >= N) c = ((c % N) + N) % N;
    } else if (c < 0 || c >= N) {
        absorb_p<INL>(R, k.S, c < 0 ? 0 : 1, v_new, sp.vy[idx], sp.vz[idx]);
        cell = -1;
        return -1;
    }
    // null-collision Monte Carlo: count the wait down; a wait that runs out
    // queues the particle, which full warps collide later and give its next
    // wait (a collision leaves the position, hence the charge assignment, as
    // it is)
    uint32_t hi = (uint32_t)cell & ~kCellMask;
    bool queued = false;
    if (R.mcc && k.collides) {
        if (((hi & ~kRedrawBit) >> kCellBits) > 1u) {
            hi -= kWaitOne;
        } else {
            const unsigned int pos = atomicAdd(sm.q.n, 1u);
            if (pos < sm.q.cap) {  // always: drains keep a tile's room
                sm.q.slot[pos] = (uint32_t)idx | (k.S ? kQueueIon : 0u) | (hi & kRedrawBit ? kQueueRedraw : 0u);
                queued = true;
            } else {
                atomicOr(&R.st->status, 0x8u);
            }
            hi = 0u;  // the drain stores the next wait
        }
    }
    cell = c | (int)hi;
    if (k.S == 0 && diag && R.eedf_bins > 0 && !queued) eedf_sample(R, sm, vx, sp.vy[idx], sp.vz[idx]);
    if (MI::mc) return deposit_key_s1(c, s, a_out);
    if (MI::ec3) return deposit_key_s3(c, s, a_out);
    return deposit_key_s2(c, s, a_out);
}

// Vector load / store of U consecutive 4-byte values (U = 1, 2, 4); the
// address is U*4-byte aligned.
template <typename T> struct Vec2;
template <> struct Vec2<int> { using type = int2; };
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<uint32_t> { using type = uint2; };
template <typename T> struct Vec4;
template <> struct Vec4<int> { using type = int4; };
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<uint32_t> { using type = uint4; };

template <int U, typename T>
__device__ __forceinline__ void ldv(const T *p, T (&o)[kUnroll]) {
    if constexpr (U == 4) {
        const auto v = *reinterpret_cast<const typename Vec4<T>::type *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (U == 2) {
        const auto v = *reinterpret_cast<const typename Vec2<T>::type *>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = p[0];
    }
}

template <int U, typename T>
__device__ __forceinline__ void stv(T *p, const T (&o)[kUnroll]) {
    if constexpr (U == 4) {
        typename Vec4<T>::type v;
        v.x = o[0]; v.y = o[1]; v.z = o[2]; v.w = o[3];
        *reinterpret_cast<typename Vec4<T>::type *>(p) = v;
    } else if constexpr (U == 2) {
        typename Vec2<T>::type v;
        v.x = o[0]; v.y = o[1];
        *reinterpret_cast<typename Vec2<T>::type *>(p) = v;
    } else {
        p[0] = o[0];
    }
}

// ---------------------------------------------------------------------------
// Asynchronous staging of the particle stream.  One thread streams tiles of
// kTile particles of every field the mode reads from HBM into a ring of
// kStages shared-memory buffers with cp.async.bulk, completion signalled on
// one mbarrier per buffer, while all warps work on the current tile.  Every
// wait is bounded: a wait that runs out sets PIC_STATUS_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr int kTile = kThreads * kUnroll;
static_assert(kQueueDrainAbove + kTile <= kQueue, "a tile must fit the undrained queue");
#ifndef PIC_STAGES
#define PIC_STAGES 2
#endif
constexpr int kStages = PIC_STAGES;
constexpr int kMaxFields = 4;  // cell, off, vx, abar
// A wait gives up after about a second (or 2^30 polls, whichever comes first).
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr long long kWaitPolls = 1ll << 30;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned int bytes,
                                         unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned int parity) {
    unsigned int done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for one phase of a barrier for at most limit_ns; false if it never
// completed.  The clock is read only once the first poll has failed.
__device__ __forceinline__ bool mbar_wait_for(unsigned long long *bar, unsigned int parity,
                                              unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (long long i = 0; i < kWaitPolls; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) break;
    }
    return false;
}

// Bounded wait for one phase of a stage barrier; false (status bit set) if it
// never completed.
__device__ __forceinline__ bool mbar_wait(const Run &R, unsigned long long *bar, unsigned int parity) {
    if (mbar_wait_for(bar, parity, kWaitNs)) return true;
    atomicOr(&R.st->status, 0x4u);
    return false;
}

// The wait of the particle launches on a barrier that nothing completes: one
// arrival with 16 bytes expected and no copy issued, so the phase never ends,
// no memory is ever written to it and the wait can only run out.
__global__ void k_wait_selftest(unsigned long long limit_ns, unsigned int *status, unsigned long long *waited_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, 16u);
    const unsigned long long t0 = globaltimer_ns();
    const bool done = mbar_wait_for(&bar, 0u, limit_ns);
    *waited_ns = globaltimer_ns() - t0;
    *status = done ? 0u : 0x4u;
}

// The ring: kStages x nf arrays of kTile words, one barrier per stage.  The
// implicit passes stage cell, off, vx and abar; the other modes cell, off and
// vx (the id of a particle is read only when its wait runs out).
struct Ring {
    uint32_t *buf;               // [kStages][nf][kTile]
    unsigned long long *bar;     // [kStages] (static shared)
    unsigned int *uses;          // tiles issued so far by this block (static shared)
    int nf;                      // 3 or kMaxFields
};

__host__ __device__ constexpr size_t ring_bytes(bool implicit) {
    return (size_t)kStages * (implicit ? kMaxFields : kMaxFields - 1) * kTile * 4;
}
// The idle ring holds the tail's copy of the per-key sums (6 x 8 bytes a key).

__device__ __forceinline__ uint32_t *ring_field(const Ring &g, int stage, int f) {
    return g.buf + ((size_t)stage * g.nf + f) * kTile;
}

// A thread's kUnroll consecutive words of a staged field, from place s0 of the
// tile (a multiple of kUnroll): one 16-byte shared load for kUnroll = 4, which
// keeps the warp's access free of bank conflicts.  Words beyond the tile's
// particles are stale; the caller masks them.
__device__ __forceinline__ void ring_words(const Ring &g, int stage, int f, int s0, uint32_t (&o)[kUnroll]) {
    const uint32_t *p = ring_field(g, stage, f) + s0;
    if constexpr (kUnroll == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (kUnroll == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = p[0];
    }
}

// Load a thread's particles of a staged tile: n_ok of them are real (cell -1
// marks the rest); fields a mode does not use read as zero.
template <int MODE>
__device__ __forceinline__ void ring_particles(const Ring &g, int stage, int s0, int n_ok, int (&cell)[kUnroll],
                                               float (&off)[kUnroll], float (&vx)[kUnroll],
                                               float (&abar)[kUnroll]) {
    using MI = ModeInfo<MODE>;
    uint32_t w[kUnroll];
#pragma unroll
    for (int q = 0; q < kUnroll; ++q) vx[q] = abar[q] = 0.0f;
    ring_words(g, stage, 0, s0, w);
#pragma unroll
    for (int q = 0; q < kUnroll; ++q) cell[q] = (int)w[q];
    ring_words(g, stage, 1, s0, w);
#pragma unroll
    for (int q = 0; q < kUnroll; ++q) off[q] = __uint_as_float(w[q]);
    if (MI::loads_v) {
        ring_words(g, stage, 2, s0, w);
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) vx[q] = __uint_as_float(w[q]);
    }
    if (MI::implicit) {
        ring_words(g, stage, 3, s0, w);
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) abar[q] = __uint_as_float(w[q]);
    }
    if (n_ok < kUnroll) {  // the tile's ragged end: the words beyond it are stale
#pragma unroll
        for (int q = 0; q < kUnroll; ++q)
            if (q >= n_ok) {
                cell[q] = -1;
                off[q] = vx[q] = abar[q] = 0.0f;
            }
    }
}

// Issue the copies of tile t (block-relative tile counter u) of segment
// [b, b + len): fields in the order cell, off, vx, abar.
template <int MODE>
__device__ __forceinline__ void ring_issue(const Ring &g, const Species &sp0, long long b, int len, int t,
                                           unsigned int u) {
    using MI = ModeInfo<MODE>;
    const int stage = (int)(u % kStages);
    const int first = t * kTile;
    const int n = min(kTile, len - first);
    const unsigned int bytes = (unsigned int)(((n * 4) + 15) & ~15);  // arrays are padded to 16 bytes
    const int nf = 2 + (MI::loads_v ? 1 : 0) + (MI::implicit ? 1 : 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&g.bar[stage], bytes * nf);
    const long long o = b + first;
    bulk_g2s(ring_field(g, stage, 0), sp0.cell + o, bytes, &g.bar[stage]);
    bulk_g2s(ring_field(g, stage, 1), sp0.off + o, bytes, &g.bar[stage]);
    if (MI::loads_v) bulk_g2s(ring_field(g, stage, 2), sp0.vx + o, bytes, &g.bar[stage]);
    if (MI::implicit) bulk_g2s(ring_field(g, stage, 3), sp0.abar + o, bytes, &g.bar[stage]);
}

// Stream one species segment [b, e) through the block in staged tiles; each
// thread takes kUnroll consecutive particles of a tile, steps them
// independently, stores them back with vector stores and deposits the tile.
template <int MODE, int S>
__device__ void process_segment(const Run &R, const SmemMain &sm, const Ring &g, const Species &sp0,
                                long long b, long long e, bool diag, long long step, Tally &t) {
    constexpr int U = kUnroll;
    static_assert(U == 1 || U == 2 || U == 4, "vector width");
    using MI = ModeInfo<MODE>;
    Species sp;
    sp.cell = sp0.cell + b;
    sp.off = sp0.off + b;
    sp.vx = sp0.vx + b;
    sp.vy = sp0.vy + b;
    sp.vz = sp0.vz + b;
    sp.id = sp0.id + b;
    sp.abar = MI::implicit ? sp0.abar + b : nullptr;
    const int len = (int)(e - b);
    const int ntiles = (len + kTile - 1) / kTile;
    const unsigned int u0 = *g.uses;  // tiles this block issued before this segment
    float kx = 0.0f, pw = 0.0f;
    if (threadIdx.x == 0)
        for (int tt = 0; tt < kStages - 1 && tt < ntiles; ++tt) ring_issue<MODE>(g, sp0, b, len, tt, u0 + tt);
    for (int tl = 0; tl < ntiles; ++tl) {
        const unsigned int u = u0 + tl;
        const int stage = (int)(u % kStages);
        if (threadIdx.x == 0 && tl + kStages - 1 < ntiles)
            ring_issue<MODE>(g, sp0, b, len, tl + kStages - 1, u + kStages - 1);
        if (!mbar_wait(R, &g.bar[stage], (u / kStages) & 1u)) {
            // give up on this segment, but not before the copies already
            // issued into the ring have landed (bounded as well)
            for (int tw = tl + 1; tw < ntiles && tw < tl + kStages; ++tw)
                mbar_wait(R, &g.bar[(u0 + tw) % kStages], ((u0 + tw) / kStages) & 1u);
            __syncthreads();
            if (threadIdx.x == 0) *g.uses = u0 + (unsigned int)min(ntiles, tl + kStages);
            __syncthreads();
            t.kx += kx;
            t.pw += pw;
            return;
        }
        const int base = tl * kTile;
        const int i0 = base + U * (int)threadIdx.x;   // segment-relative index of the first particle
        const int s0 = U * (int)threadIdx.x;          // its place in the tile
        const bool full = i0 + U - 1 < len;
        int cell[U];
        float off[U], vx[U], abar[U];
        ring_particles<MODE>(g, stage, s0, len - i0, cell, off, vx, abar);
        const SpK k = species_k(R, S);
        int key[U];
        uint32_t a[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            a[q] = 0u;
            key[q] = -1;
            if (cell[q] < 0) continue;  // beyond the segment, or a hole left by absorption
            key[q] = step_particle<MODE, false>(R, sm, sp, k, (long long)(i0 + q), cell[q], off[q], vx[q],
                                            abar[q], diag, step, t, kx, pw, a[q]);
        }
        if (MI::push) {
            if (full) {
                stv<U>(sp.cell + i0, cell);
                stv<U>(sp.off + i0, off);
                stv<U>(sp.vx + i0, vx);
                if (MI::implicit) stv<U>(sp.abar + i0, abar);
            } else {
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int i = i0 + q;
                    if (i < len) {
                        sp.cell[i] = cell[q];
                        sp.off[i] = off[q];
                        sp.vx[i] = vx[q];
                        if (MI::implicit) sp.abar[i] = abar[q];
                    }
                }
            }
        }
        deposit_tile(key, a, sm.acc, MI::count_only);
        // The stage is free again.  The drain is the block's decision, taken
        // by the barrier: the thread that queued the tile's last particle
        // reads the count after doing so (a count read after the barrier could
        // already include the next tile's particles in some threads only).
        const bool drain = __syncthreads_or((MI::push && R.mcc && *sm.q.n > kQueueDrainAbove) ? 1 : 0) != 0;
        if (drain) drain_collisions(R, sm, sp, sp, step, diag, t);
    }
    if (MI::push && R.mcc) {
        __syncthreads();
        if (*sm.q.n > 0u) drain_collisions(R, sm, sp, sp, step, diag, t);
    }
    t.kx += kx;
    t.pw += pw;
    __syncthreads();
    if (threadIdx.x == 0) *g.uses = u0 + (unsigned int)ntiles;
    __syncthreads();
}

// Add the block's shared accumulators of one species to the run's global ones.
__device__ void flush_species(const Run &R, const SmemMain &sm, int S, bool count_only, bool ec3 = false) {
    __syncthreads();
    const int n1 = R.n_cells + 1;
    for (int k = threadIdx.x; k < n1; k += kThreads) {
        const unsigned int c = sm.acc.cnt[k];
        if (c && ec3) {
            atomicAdd(&R.acc_cnt[S][k], (unsigned long long)c);
            atomicAdd(&R.acc_a[S][k], (unsigned long long)sm.acc.a[k]);
            atomicAdd(&R.acc_b[S][k], ((unsigned long long)sm.acc.bh[k] << 12) + sm.acc.bl[k]);
            atomicAdd(&R.acc_c[S][k], ((unsigned long long)sm.acc.s3h[k] << 24) +
                                          ((unsigned long long)sm.acc.s3m[k] << 12) + sm.acc.s3l[k]);
            sm.acc.cnt[k] = 0u;
            sm.acc.a[k] = 0u;
            sm.acc.bh[k] = 0u;
            sm.acc.bl[k] = 0u;
            sm.acc.s3h[k] = 0u;
            sm.acc.s3m[k] = 0u;
            sm.acc.s3l[k] = 0u;
        } else if (c) {
            atomicAdd(&R.acc_cnt[S][k], (unsigned long long)c);
            if (!count_only) {
                atomicAdd(&R.acc_a[S][k], (unsigned long long)sm.acc.a[k]);
                atomicAdd(&R.acc_b[S][k], ((unsigned long long)sm.acc.bh[k] << 16) + sm.acc.bl[k]);
            }
            sm.acc.cnt[k] = 0u;
            sm.acc.a[k] = 0u;
            sm.acc.bh[k] = 0u;
            sm.acc.bl[k] = 0u;
        }
    }
    __syncthreads();
}

// Block totals of the per-thread tallies, one barrier pair.
__device__ void flush_tally(const Run &R, int S, const Tally &t) {
    constexpr int nw = kThreads / 32;
    __shared__ float s_f[2][nw];
    __shared__ unsigned int s_u[7][nw];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float kx = warp_sum(t.kx), pw = warp_sum(t.pw);
    const unsigned int u[7] = {warp_sum(t.el), warp_sum(t.ex), warp_sum(t.iz), warp_sum(t.cx),
                               warp_sum(t.nul), warp_sum(t.ovf_e), warp_sum(t.ovf_i)};
    if (lane == 0) {
        s_f[0][wid] = kx;
        s_f[1][wid] = pw;
        for (int k = 0; k < 7; ++k) s_u[k][wid] = u[k];
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        const int k = threadIdx.x;
        if (k < 2) {
            double acc = 0.0;
            for (int w = 0; w < nw; ++w) acc += (double)s_f[k][w];
            if (acc != 0.0) atomicAdd(k == 0 ? &R.st->ke_x_acc[S] : &R.st->power_acc[S], acc);
        } else {
            unsigned long long acc = 0;
            for (int w = 0; w < nw; ++w) acc += s_u[k - 2][w];
            if (acc) atomicAdd(k - 2 < 5 ? &R.st->coll[k - 2] : &R.st->overflow[k - 7], acc);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tail pieces (run by the last block of a particle launch).
// ---------------------------------------------------------------------------

// Per-key sums of species S with the periodic fold (key n is key 0).
struct KeySums {
    unsigned long long c, a, b;
};

// Where the tail reads the per-key sums (count, sum a, sum a^2) of both
// species: the run's global accumulators or the tail's shared-memory copy.
struct Keys {
    unsigned long long *c[2], *a[2], *b[2];
    unsigned long long *d[2];  // m = 3: sum F^3 (b holds sum F^2)
};

__device__ __forceinline__ Keys global_keys(const Run &R) {
    Keys K;
    for (int S = 0; S < 2; ++S) {
        K.c[S] = R.acc_cnt[S];
        K.a[S] = R.acc_a[S];
        K.b[S] = R.acc_b[S];
        K.d[S] = R.acc_c[S];
    }
    return K;
}

__device__ __forceinline__ KeySums key_sums(const Run &R, const Keys &K, int S, int k) {
    const int n = R.n_cells;
    KeySums r = {0ull, 0ull, 0ull};
    if (R.periodic) {
        k = ((k % n) + n) % n;
        r.c = K.c[S][k];
        r.a = K.a[S][k];
        r.b = K.b[S][k];
        if (k == 0) {
            r.c += K.c[S][n];
            r.a += K.a[S][n];
            r.b += K.b[S][n];
        }
    } else if (k >= 0 && k <= n) {
        r.c = K.c[S][k];
        r.a = K.a[S][k];
        r.b = K.b[S][k];
    }
    return r;
}

// Node charge of species S in units of 2^-33 macro-particle charges,
// reassembled from the per-key sums (count c, sum a = A, sum a^2 = B):
// node g gets 2^32 c_g + 2^17 A_g - 2 B_g from key g, B_{g-1} from key g-1 and
// 2^32 c_{g+1} - 2^17 A_{g+1} + B_{g+1} from key g+1.  Electrodes fold the
// ghost nodes onto the wall nodes; the periodic box wraps.  Unsigned
// arithmetic: the result is exact modulo 2^64 and lies in range.
__device__ __forceinline__ unsigned long long node_charge_s2(const Run &R, const Keys &K, int S, int g) {
    const int n = R.n_cells;
    if (R.periodic && g == n) return 0ull;
    const KeySums m = key_sums(R, K, S, g - 1), z = key_sums(R, K, S, g), p = key_sums(R, K, S, g + 1);
    unsigned long long q = (z.c << 32) + (z.a << 17) - 2ull * z.b + m.b + (p.c << 32) - (p.a << 17) + p.b;
    if (!R.periodic) {
        if (g == 0) q += (z.c << 32) - (z.a << 17) + z.b;  // ghost node -1
        if (g == n) q += z.b;                               // ghost node n+1
    }
    return q;
}

// The same from raw pointers and scalars (the tail's loops: nothing they
// store can alias these inputs).
__device__ __forceinline__ unsigned long long ksum_c(const unsigned long long *__restrict__ p, int n, bool periodic,
                                                     int k) {
    if (periodic) {
        k = k < 0 ? k + n : (k >= n ? k - n : k);
        return k == 0 ? p[0] + p[n] : p[k];
    }
    return (k >= 0 && k <= n) ? p[k] : 0ull;
}

__device__ __forceinline__ unsigned long long node_charge_s2_raw(const unsigned long long *__restrict__ C,
                                                                 const unsigned long long *__restrict__ A,
                                                                 const unsigned long long *__restrict__ B, int n,
                                                                 bool periodic, int g) {
    if (periodic && g == n) return 0ull;
    const unsigned long long mb = ksum_c(B, n, periodic, g - 1);
    const unsigned long long zc = ksum_c(C, n, periodic, g), za = ksum_c(A, n, periodic, g),
                             zb = ksum_c(B, n, periodic, g);
    const unsigned long long pc = ksum_c(C, n, periodic, g + 1), pa = ksum_c(A, n, periodic, g + 1),
                             pb = ksum_c(B, n, periodic, g + 1);
    unsigned long long q = (zc << 32) + (za << 17) - 2ull * zb + mb + (pc << 32) - (pa << 17) + pb;
    if (!periodic) {
        if (g == 0) q += (zc << 32) - (za << 17) + zb;  // ghost node -1
        if (g == n) q += zb;                             // ghost node n+1
    }
    return q;
}

// m = 3 node charge in units of 2^-36/6 macro-particle charges from the
// per-cell sums (count c, sum F = A, sum F^2 = B, sum F^3 = D), T = 2^12:
// cell g+1 gives its left node T^3 c - 3 T^2 A + 3 T B - D, cell g gives
// 4 T^3 c - 6 T B + 3 D, cell g-1 gives T^3 c + 3 T^2 A + 3 T B - 3 D and
// cell g-2 gives D (the spline weights of deposit_key_s3 summed over the
// cell's particles).  Electrodes fold the ghost nodes -1 and n+1 onto the
// wall nodes; the periodic box wraps (node n is node 0).  Unsigned
// arithmetic: exact modulo 2^64, and the result lies in range.
__device__ __forceinline__ unsigned long long cell_sum(const unsigned long long *__restrict__ p, int n,
                                                       bool periodic, int k) {
    if (periodic) return p[k < 0 ? k + n : (k >= n ? k - n : k)];
    return (k >= 0 && k < n) ? p[k] : 0ull;
}

__device__ __forceinline__ unsigned long long node_charge_s3_raw(const unsigned long long *__restrict__ C,
                                                                 const unsigned long long *__restrict__ A,
                                                                 const unsigned long long *__restrict__ B,
                                                                 const unsigned long long *__restrict__ D, int n,
                                                                 bool periodic, int g) {
    if (periodic && g == n) return 0ull;
    // left node of cell k (k = g+1; with the fold, also cell 0 for node 0)
    auto left = [&](int k) {
        return (cell_sum(C, n, periodic, k) << 36) - 3ull * (cell_sum(A, n, periodic, k) << 24) +
               3ull * (cell_sum(B, n, periodic, k) << 12) - cell_sum(D, n, periodic, k);
    };
    auto own = [&](int k) {
        return (cell_sum(C, n, periodic, k) << 38) - 6ull * (cell_sum(B, n, periodic, k) << 12) +
               3ull * cell_sum(D, n, periodic, k);
    };
    auto right = [&](int k) {
        return (cell_sum(C, n, periodic, k) << 36) + 3ull * (cell_sum(A, n, periodic, k) << 24) +
               3ull * (cell_sum(B, n, periodic, k) << 12) - 3ull * cell_sum(D, n, periodic, k);
    };
    unsigned long long q = left(g + 1) + own(g) + right(g - 1) + cell_sum(D, n, periodic, g - 2);
    if (!periodic) {
        if (g == 0) q += left(0);                         // ghost node -1
        if (g == n) q += cell_sum(D, n, periodic, n - 1);  // ghost node n+1
    }
    return q;
}

// S_1 node charge (momentum-conserving scheme), key = cell, value F:
// node g gets (2^16 c_g - A_g) from cell g and A_{g-1} from cell g-1, times 2^17.
__device__ __forceinline__ unsigned long long node_charge_s1(const Run &R, const Keys &K, int S, int g) {
    const int n = R.n_cells;
    const unsigned long long *C = K.c[S], *A = K.a[S];
    if (R.periodic && g == n) return 0ull;
    unsigned long long q = 0;
    if (g < n) q += (C[g] << 16) - A[g];
    const int gl = R.periodic ? (g - 1 + n) % n : g - 1;
    if (gl >= 0 && gl < n) q += A[gl];
    return q << 17;
}

// Susceptibility weight of cell c (units 2^-16): a from key c, 2^16 - a from key c+1.
__device__ __forceinline__ unsigned long long chi_count(const Run &R, const Keys &K, int S, int c) {
    const KeySums z = key_sums(R, K, S, c), p = key_sums(R, K, S, c + 1);
    return z.a + (p.c << 16) - p.a;
}

// What the tail reads of the run state, loaded by thread 0 together with the
// staged sums (one round trip) and kept in shared memory.
struct TailHead {
    unsigned int B, ok;          // births of the step (capped at the buffer) and those placed
    unsigned int id_e, id_i;     // next ids
    long long ne, ni;            // slots before the births
    int parity;
    // read for the counters thread 0 rewrites at the end
    unsigned int nb;
    long long live[2], n_avg, n_diag;
    unsigned long long absorbed[2], births_total;
    double ke_acc[2], pw_acc[2], fe_acc;
    double vl_v;                 // electrode voltage stored at launch start
    float vl_hi, vl_lo;
};

// Place the step's births: rank by parent id, append children at the end of
// both species' slots with consecutive ids, assign their charge (explicit) or
// count their keys (implicit pass 2, for the sort).  Up to kThreads births
// each thread holds one record, loaded with the staged sums (`my`); more go
// through a bucketed ranking in global memory.  The counters are advanced by
// the caller.
// A store, or an add, to global memory that takes effect only if `p`: a
// warming pass executes the instruction (so its code is fetched) with p false.
__device__ __forceinline__ void st_g32_if(bool p, const void *addr, uint32_t v) {
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.global.b32 [%1], %2;\n}" ::"r"((unsigned)p),
                 "l"(__cvta_generic_to_global(addr)), "r"(v)
                 : "memory");
}
__device__ __forceinline__ void red_g64_if(bool p, const void *addr, unsigned long long v) {
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q red.global.add.u64 [%1], %2;\n}" ::"r"((unsigned)p),
                 "l"(__cvta_generic_to_global(addr)), "l"(v)
                 : "memory");
}

template <int MODE>
__device__ void tail_births(const Run &R, Keys K, unsigned char *smem, bool diag, const TailHead &hd,
                            const Birth &my_rec, bool dry, long long step, const uint32_t *wtab) {
    // A warming pass takes one made-up birth (cell 0, no global write)
    // through the code of the few-births path, whatever the step's count.
    const unsigned int B = dry ? 1u : hd.B, ok = dry ? 1u : hd.ok;
    if (B == 0) return;
    Birth my = my_rec;
    if (dry) {
        my = Birth{};
        my.off = 0.25f;
    }
    const Species se = R.buf[hd.parity][0], si = R.buf[hd.parity][1];
    const unsigned int id_e = hd.id_e, id_i = hd.id_i;
    const long long s_ne = hd.ne, s_ni = hd.ni;
    // One child of birth bb (rank r): species S's key sums, its first wait
    // (drawn on its birth step) and its slot; a warming pass runs the stores
    // with their predicate off.
    auto place_child = [&](int cell, float off, float vx, float vy, float vz, float abar, unsigned int r, int S) {
        const long long j = (S ? s_ni : s_ne) + r;
        const Species &sp = S ? si : se;
        const uint32_t id = (S ? id_i : id_e) + r;
        uint32_t a;
        const int key = ModeInfo<MODE>::mc    ? deposit_key_s1(cell, off, a)
                        : ModeInfo<MODE>::ec3 ? deposit_key_s3(cell, off, a)
                                              : deposit_key_s2(cell, off, a);
        atomicAdd(&K.c[S][key], 1ull);
        if (!ModeInfo<MODE>::count_only) {
            atomicAdd(&K.a[S][key], (unsigned long long)a);
            atomicAdd(&K.b[S][key], (unsigned long long)a * a);
            if (ModeInfo<MODE>::ec3) atomicAdd(&K.d[S][key], (unsigned long long)a * a * a);
        }
        const bool w = !dry;
        const uint32_t cw = (uint32_t)cell | (R.mcc ? wait_bits(draw_wait(R, wtab, S, id, step, 1)) : 0u);
        st_g32_if(w, sp.cell + j, cw);
        st_g32_if(w, sp.off + j, __float_as_uint(off));
        st_g32_if(w, sp.vx + j, __float_as_uint(vx));
        st_g32_if(w, sp.vy + j, __float_as_uint(vy));
        st_g32_if(w, sp.vz + j, __float_as_uint(vz));
        st_g32_if(w, sp.id + j, id);
        if (ModeInfo<MODE>::implicit) st_g32_if(w, sp.abar + j, __float_as_uint(abar));
        if (S == 0 && diag && R.eedf_bins > 0) {
            const float en = R.half_m_over_e[0] * (vx * vx + vy * vy + vz * vz);
            int bin = (int)floorf(en * R.eedf_inv_width);
            bin = bin > R.eedf_bins ? R.eedf_bins : (bin < 0 ? 0 : bin);
            red_g64_if(w, R.eedf + bin, 1ull);
        }
    };
    auto place = [&](const Birth &bb, unsigned int r) {
        place_child(bb.cell, bb.off, bb.ve[0], bb.ve[1], bb.ve[2], bb.abar_e, r, 0);
        place_child(bb.cell, bb.off, bb.vi[0], bb.vi[1], bb.vi[2], bb.abar_e * R.abar_ion_over_e, r, 1);
    };
    auto rank_of = [&](const uint32_t *spid, uint32_t p) {
        // rank = number of births with a smaller parent id (ids are unique),
        // against all parent ids staged in shared memory (padded to a
        // multiple of 4 with the largest id)
        const uint4 *sp4 = (const uint4 *)spid;
        const unsigned int nq = (B + 3u) / 4u;
        unsigned int r = 0;
        for (unsigned int k = 0; k < nq; ++k) {
            const uint4 v = sp4[k];
            r += (v.x < p ? 1u : 0u) + (v.y < p ? 1u : 0u) + (v.z < p ? 1u : 0u) + (v.w < p ? 1u : 0u);
        }
        return r;
    };
    if (B <= (unsigned int)kThreads / 2) {
        // thread t places the electron child of birth t and thread
        // kThreads/2 + t its ion child, side by side
        uint32_t *spid = (uint32_t *)smem;  // [kThreads]
        spid[threadIdx.x] = threadIdx.x < B ? my.pid : 0xffffffffu;
        __syncthreads();
        const unsigned int t = threadIdx.x % (kThreads / 2);
        const int S = (int)(threadIdx.x / (kThreads / 2));
        if (t < B) {
            // the ion side reads birth t's record (the electron side holds it)
            const Birth *g = (S == 1 && !dry) ? R.births + t : nullptr;
            const uint32_t pid = g ? g->pid : my.pid;
            const unsigned int r = rank_of(spid, pid);
            if (r < ok) {
                if (S == 0)
                    place_child(my.cell, my.off, my.ve[0], my.ve[1], my.ve[2], my.abar_e, r, 0);
                else if (g)
                    place_child(g->cell, g->off, g->vi[0], g->vi[1], g->vi[2], g->abar_e * R.abar_ion_over_e, r, 1);
                else
                    place_child(my.cell, my.off, my.vi[0], my.vi[1], my.vi[2], my.abar_e * R.abar_ion_over_e, r, 1);
            }
        }
        __syncthreads();
        return;
    }
    if (B <= (unsigned int)kThreads) {
        // rank = number of births with a smaller parent id (ids are unique),
        // by comparison against all parent ids staged in shared memory (padded
        // to a multiple of 4 with the largest id)
        uint32_t *spid = (uint32_t *)smem;  // [kThreads]
        spid[threadIdx.x] = threadIdx.x < B ? my.pid : 0xffffffffu;
        __syncthreads();
        if (threadIdx.x < B) {
            const unsigned int r = rank_of(spid, my.pid);
            if (r < ok) place(my, r);
        }
        __syncthreads();
        return;
    }
    // many births: counting pass over 2048 buckets of the parent id's top
    // bits, then a comparison within the bucket
    unsigned int *hist = (unsigned int *)smem;                       // [2048]
    unsigned int *rank = (unsigned int *)(R.births + R.births_cap);  // [births_cap]
    uint32_t *sorted = (uint32_t *)(rank + R.births_cap);            // [births_cap]
    const int bits = 32 - __clz(id_e | 1u);  // parent ids are below the next electron id
    const int shift = bits > 11 ? bits - 11 : 0;
    for (int k = threadIdx.x; k < 2048; k += kThreads) hist[k] = 0u;
    __syncthreads();
    for (unsigned int b = threadIdx.x; b < B; b += kThreads) {
        const unsigned int pos = atomicAdd(&hist[R.births[b].pid >> shift], 1u);
        if (!dry) rank[b] = pos;
    }
    __syncthreads();
    {
        __shared__ unsigned int sc_h[33];
        constexpr int per = 2048 / kThreads;
        unsigned int loc[per];
        unsigned int run = 0;
        for (int k = 0; k < per; ++k) {
            loc[k] = hist[threadIdx.x * per + k];
            run += loc[k];
        }
        unsigned int tot;
        unsigned int ex = block_exclusive_scan<unsigned int>(run, sc_h, tot);
        for (int k = 0; k < per; ++k) {
            hist[threadIdx.x * per + k] = ex;  // bucket start
            ex += loc[k];
        }
    }
    __syncthreads();
    for (unsigned int b = threadIdx.x; b < B && !dry; b += kThreads) {
        const uint32_t p = R.births[b].pid;
        sorted[hist[p >> shift] + rank[b]] = p;
    }
    __syncthreads();
    for (unsigned int b = threadIdx.x; b < B; b += kThreads) {
        const Birth bb = R.births[b];
        const unsigned int bk = bb.pid >> shift;
        const unsigned int lo = hist[bk], hi = bk + 1 < 2048u ? hist[bk + 1] : B;
        unsigned int r = lo;
        for (unsigned int k = lo; k < hi; ++k) r += sorted[k] < bb.pid ? 1u : 0u;
        if (r < ok) place(bb, r);
    }
    __syncthreads();
}

// Sum of a double over the block: warp shuffles, then one warp (few FP64
// operations: the FP64 pipe is narrow on this part).  All threads get it.
__device__ double block_sum_lean(double x, double *scratch /*[kThreads/32 + 1]*/) {
    constexpr int nw = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    x = warp_sum(x);
    if (lane == 0) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double y = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(FULL_MASK, y, o);
        if (lane == 0) scratch[nw] = y;
    }
    __syncthreads();
    const double r = scratch[nw];
    __syncthreads();
    return r;
}

// Exclusive block scan of two 64-bit integers at once.
__device__ void block_exclusive_scan_pair(long long &x, unsigned long long &y, long long &tx,
                                          unsigned long long &ty, long long *sx, unsigned long long *sy) {
    constexpr int nw = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long ix = x;
    unsigned long long iy = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(FULL_MASK, ix, o);
        const unsigned long long b = __shfl_up_sync(FULL_MASK, iy, o);
        if (lane >= o) {
            ix += a;
            iy += b;
        }
    }
    if (lane == 31) {
        sx[wid] = ix;
        sy[wid] = iy;
    }
    __syncthreads();
    long long bx = 0;
    unsigned long long by = 0;
    tx = 0;
    ty = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < wid) {
            bx += sx[w];
            by += sy[w];
        }
        tx += sx[w];
        ty += sy[w];
    }
    __syncthreads();
    x = bx + ix - x;
    y = by + iy - y;
}

// The same scan of (x, y), and the block totals (th, tl) of (h, l) with it:
// one pass of barriers for both.
__device__ void block_scan_pair_sum_pair(long long &x, unsigned long long &y, long long &tx, unsigned long long &ty,
                                         long long h, unsigned long long l, long long &th, unsigned long long &tl,
                                         long long *sx, unsigned long long *sy, long long *sh,
                                         unsigned long long *sl) {
    constexpr int nw = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long ix = x;
    unsigned long long iy = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(FULL_MASK, ix, o);
        const unsigned long long b = __shfl_up_sync(FULL_MASK, iy, o);
        if (lane >= o) {
            ix += a;
            iy += b;
        }
        h += __shfl_xor_sync(FULL_MASK, h, o);
        l += __shfl_xor_sync(FULL_MASK, l, o);
    }
    if (lane == 31) {
        sx[wid] = ix;
        sy[wid] = iy;
        sh[wid] = h;
        sl[wid] = l;
    }
    __syncthreads();
    long long bx = 0;
    unsigned long long by = 0;
    tx = 0;
    ty = 0;
    th = 0;
    tl = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < wid) {
            bx += sx[w];
            by += sy[w];
        }
        tx += sx[w];
        ty += sy[w];
        th += sh[w];
        tl += sl[w];
    }
    __syncthreads();
    x = bx + ix - x;
    y = by + iy - y;
}

// Field solve by the discrete Gauss law.  The finite-difference Poisson
// equation -(phi_{g-1} - 2 phi_g + phi_{g+1})/dx^2 = rho_g/eps0 (with (1+chi)
// on the cell faces in the implicit scheme) is D_{c} - D_{c-1} = dx rho_c / eps0
// for the face quantity D_c = (1 + chi_c) E_c, E_c = (phi_c - phi_{c+1})/dx.
// So D_c = D_0 + kappa P_c with the exact int64 prefix sum P_c of the node
// charge; the electrode condition sum_c E_c dx = V(t) (or zero mean field in
// the periodic box) fixes D_0.  O(n) work, O(log n) depth; the same linear
// system the oracle solves with the Thomas algorithm.  The node potential is
// a diagnostic only (the gather uses E): it follows from E and V on the host,
// and so does its time average from the averages of E and V.
// With `cursors` the same integer scan also yields the sort cursors (the
// exclusive prefix of the per-key counts of both species).
// ---------------------------------------------------------------------------
// Double-word ("float-float") arithmetic, after Joldes, Muller & Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017): a value is an unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The field
// solve of the explicit schemes runs in it because FP64 latency on this part
// dominated the serial tail; FP64 only converts the result afterwards.
// ---------------------------------------------------------------------------
struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_two_sum(float a, float b) {  // Knuth: a + b exactly
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {  // Dekker, |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dw dw_add(dw x, dw y) {  // accurate DW + DW (their Algorithm 6)
    const dw s = dw_two_sum(x.hi, y.hi);
    const dw t = dw_two_sum(x.lo, y.lo);
    const dw v = dw_fast_two_sum(s.hi, s.lo + t.hi);
    return dw_fast_two_sum(v.hi, t.lo + v.lo);
}

__device__ __forceinline__ dw dw_mul(dw x, dw y) {  // DW x DW (their Algorithm 12)
    const float ch = x.hi * y.hi;
    const float cl = fmaf(x.hi, y.hi, -ch);
    const float tl = fmaf(x.lo, y.hi, x.hi * y.lo);
    return dw_fast_two_sum(ch, cl + tl);
}

__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }

// An int64 as a double-word: three pieces of at most 22 bits are exact in
// FP32; their sum is rounded once to the double-word precision.
__device__ __forceinline__ dw dw_from_i64(long long v) {
    // each piece goes through a 32-bit integer: the 64-bit conversion is slow here
    const float a = (float)(int)(v >> 44) * 17592186044416.0f;        // * 2^44
    const float b = (float)(int)((v >> 22) & 0x3fffffll) * 4194304.0f; // * 2^22
    const float c = (float)(int)(v & 0x3fffffll);
    return dw_add(dw_two_sum(a, b), dw{c, 0.0f});
}

__device__ __forceinline__ dw dw_of(const float (&p)[2]) { return {p[0], p[1]}; }

// Sum of a double-word value over the block (all threads get it).
__device__ dw block_sum_dw(dw x, float2 *scratch /*[kThreads/32 + 1]*/) {
    constexpr int nw = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        x = dw_add(x, dw{__shfl_xor_sync(FULL_MASK, x.hi, o), __shfl_xor_sync(FULL_MASK, x.lo, o)});
    if (lane == 0) scratch[wid] = make_float2(x.hi, x.lo);
    __syncthreads();
    if (wid == 0) {
        dw y = lane < nw ? dw{scratch[lane].x, scratch[lane].y} : dw{0.0f, 0.0f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            y = dw_add(y, dw{__shfl_xor_sync(FULL_MASK, y.hi, o), __shfl_xor_sync(FULL_MASK, y.lo, o)});
        if (lane == 0) scratch[nw] = make_float2(y.hi, y.lo);
    }
    __syncthreads();
    const float2 r = scratch[nw];
    __syncthreads();
    return dw{r.x, r.y};
}

// Electrode voltage V(t) = rf_volt sin(2 pi f t) at time level `level` (0 in
// the periodic box), with its double-word split.
struct Volt {
    double v;
    float hi, lo;
};

__device__ __forceinline__ Volt electrode_volt(const Run &R, long long level) {
    Volt r;
    r.v = R.periodic ? 0.0 : R.rf_volt * sin(2.0 * 3.14159265358979323846 * R.rf_freq * ((double)level * R.dt));
    r.hi = (float)r.v;
    r.lo = (float)(r.v - (double)r.hi);
    return r;
}

// Field of the new time level from the node charges (discrete Gauss law, see
// the notes above the particle kernel).  defer: leave the FP64 conversion of
// the field, the running averages and the field energy to the next launch
// (st->pending); otherwise do them here.  vl: the electrode voltage if the
// caller computed it already (vl_ok), else it is computed here.  fe_acc: the
// run's sum of E_c^2 of the field this launch pushed with (read by the caller
// with the rest of the run state; a deferring explicit tail reports it).
template <int MODE>
__device__ void tail_field(const Run &R, Keys K, unsigned char *smem, long long level, bool accumulate,
                           bool cursors, bool defer, Volt vl, bool vl_ok, double fe_acc, bool dry) {
    DevState *st = R.st;
    const int n = R.n_cells, n1 = n + 1;
    __shared__ long long sc_x[kThreads / 32], sc_h[kThreads / 32];
    __shared__ unsigned long long sc_y[kThreads / 32], sc_l[kThreads / 32];
    __shared__ double sc_d[kThreads / 32 + 1];
    __shared__ Volt s_vl;
    long long *q = (long long *)smem;               // [n+1] net node charge, then P_c
    double *rinv = (double *)(smem + 8 * (n + 1));   // [n] 1/(1+chi)
    double *pp = rinv + n;                           // [n] kappa P_c (+ background), then E_c
    float2 *ew = (float2 *)pp;                       // [n] explicit: E_c as a double-word pair
    constexpr bool mc = ModeInfo<MODE>::mc;
    constexpr bool ec3 = ModeInfo<MODE>::ec3;
    constexpr bool implicit = ModeInfo<MODE>::implicit;
    if (threadIdx.x == 0) s_vl = vl_ok ? vl : electrode_volt(R, level);
    // the modes that run on a non-uniform grid (the others never see one, and
    // their tails carry none of its code)
    constexpr bool nu_capable = MODE == kExplicitNU || MODE == kDepositEC || MODE == kExplicitEC3NU || MODE == kDepositEC3;
    const bool acc_now = accumulate && (implicit || !defer);
    // node charges, densities, susceptibility (pointers and scalars held in
    // registers: the stores below cannot alias them)
    {
        const bool periodic = R.periodic;
        const unsigned long long *__restrict__ c0 = K.c[0], *__restrict__ a0 = K.a[0], *__restrict__ b0 = K.b[0];
        const unsigned long long *__restrict__ c1 = K.c[1], *__restrict__ a1 = K.a[1], *__restrict__ b1 = K.b[1];
        const unsigned long long *__restrict__ d0 = K.d[0], *__restrict__ d1 = K.d[1];
        long long *__restrict__ qs = q;
        long long *__restrict__ rq0 = R.rho_q[0];
        long long *__restrict__ rq1 = R.rho_q[1];
        double *__restrict__ ane = R.avg_ne;
        double *__restrict__ ani = R.avg_ni;
        for (int g = threadIdx.x; g <= n; g += kThreads) {
            const unsigned long long ne = mc    ? node_charge_s1(R, K, 0, g)
                                          : ec3 ? node_charge_s3_raw(c0, a0, b0, d0, n, periodic, g)
                                                : node_charge_s2_raw(c0, a0, b0, n, periodic, g);
            const unsigned long long ni = mc    ? node_charge_s1(R, K, 1, g)
                                          : ec3 ? node_charge_s3_raw(c1, a1, b1, d1, n, periodic, g)
                                                : node_charge_s2_raw(c1, a1, b1, n, periodic, g);
            qs[g] = (long long)(ni - ne);
            if (dry) continue;
            rq0[g] = (long long)ne;
            rq1[g] = (long long)ni;
            if (acc_now) {
                atomicAdd(&ane[g], (double)(long long)ne);  // one writer per node: a plain sum
                atomicAdd(&ani[g], (double)(long long)ni);
            }
        }
    }
    // the direct-implicit passes on a non-uniform grid
    constexpr bool nu_implicit = MODE == kImplicit1NU || MODE == kImplicit2NU;
    if (implicit) {
        for (int c = threadIdx.x; c < n; c += kThreads) {
            double chi;
            if (mc) {
                // Reading: the node sums of the S_1 weights (the node charges,
                // 2^-33 units) averaged onto the face between them
                const int r = (R.periodic && c + 1 == n) ? 0 : c + 1;
                chi = ldexp(R.chi_coef[0], -18) * (double)(node_charge_s1(R, K, 0, c) + node_charge_s1(R, K, 0, r)) +
                      ldexp(R.chi_coef[1], -18) * (double)(node_charge_s1(R, K, 1, c) + node_charge_s1(R, K, 1, r));
            } else {
                chi = R.chi_coef[0] * (double)chi_count(R, K, 0, c) + R.chi_coef[1] * (double)chi_count(R, K, 1, c);
                // non-uniform grid: the count over the cell's own width
                if constexpr (nu_implicit) chi *= R.dx / R.h64[c];
            }
            if (!dry) R.chi[c] = chi;
            rinv[c] = 1.0 / (1.0 + chi);
        }
    }
    __syncthreads();
    // one integer scan: P_c over the cells, sort cursors over the keys; with
    // it the exact sum over the cells of P_c = sum_g q_g (n - g), in 32-bit
    // halves of q_g (high part signed)
    const int span = n1 > n ? n1 : n;
    const int per = (span + kThreads - 1) / kThreads;
    const int c_begin = threadIdx.x * per;
    long long runP = 0, wh = 0;
    unsigned long long runC = 0, wl = 0;
    for (int k = 0; k < per; ++k) {
        const int c = c_begin + k;
        if (c < n) {
            const long long qc = (R.periodic || c >= 1) ? q[c] : 0ll;
            runP += qc;
            wh += (qc >> 32) * (long long)(n - c);
            wl += ((unsigned long long)qc & 0xffffffffull) * (unsigned long long)(n - c);
        }
        if (cursors && c < n1) runC += K.c[0][c] | (K.c[1][c] << 32);
    }
    long long totP, tot_hi;
    unsigned long long totC, tot_lo;
    long long P = runP;
    unsigned long long Cx = runC;
    block_scan_pair_sum_pair(P, Cx, totP, totC, wh, wl, tot_hi, tot_lo, sc_x, sc_y, sc_h, sc_l);
    if (implicit) {
        // modified Poisson (direct implicit): FP64 with the susceptibility weights
        double s1 = 0.0, s0 = 0.0;
        for (int k = 0; k < per; ++k) {
            const int c = c_begin + k;
            if (cursors && !dry && c < n1) {
                R.cursor[0][c] = (unsigned int)(Cx & 0xffffffffull);
                R.cursor[1][c] = (unsigned int)(Cx >> 32);
                Cx += K.c[0][c] | (K.c[1][c] << 32);
            }
            if (c < n) {
                P += (R.periodic || c >= 1) ? q[c] : 0ll;
                double v;
                if constexpr (nu_implicit) {
                    // non-uniform grid: the periodic box's net charge spread by
                    // node lengths, and sum_c h_c E_c = V weighting each cell
                    const float2 w = R.wdw[c];
                    v = R.periodic ? R.kappa * ((double)P - (double)totP * ((double)w.x + (double)w.y))
                                   : R.kappa * (double)P;
                    pp[c] = v;
                    s1 += R.h64[c] * rinv[c] * v;
                    s0 += R.h64[c] * rinv[c];
                } else {
                    const double qbar = R.periodic ? (double)totP / (double)n : 0.0;
                    v = R.periodic ? R.kappa * ((double)P - (double)(c + 1) * qbar)
                                   : R.kappa * (double)P + R.kappa_bg * (double)c;
                    pp[c] = v;
                    s1 += rinv[c] * v;
                    s0 += rinv[c];
                }
            }
        }
        s1 = block_sum_lean(s1, sc_d);
        s0 = block_sum_lean(s0, sc_d);
        const double v_left = s_vl.v;
        const double d0 = R.periodic ? -s1 / s0 : ((nu_implicit ? v_left : v_left / R.dx) - s1) / s0;
        double wsum = 0.0;
        for (int k = 0; k < per; ++k) {
            const int c = c_begin + k;
            if (c < n) {
                const double e = rinv[c] * (d0 + pp[c]);
                // now the face field (a non-uniform grid's gather table: the
                // cell's voltage drop)
                pp[c] = nu_implicit ? e * R.h64[c] : e;
                wsum += nu_implicit ? e * e * R.h64[c] : e * e;
                if (dry) continue;
                R.e_cc[c] = e;
                if (accumulate) atomicAdd(&R.avg_e[c], e);
                if (!mc) R.e_gather[c + 1] = (float)pp[c];
            }
        }
        wsum = block_sum_lean(wsum, sc_d);  // includes the barrier that publishes pp[]
        if (threadIdx.x == 0 && !dry) {
            st->field_energy = (nu_implicit ? R.eps0_half : R.eps0_dx_half) * wsum;
            if (ModeInfo<MODE>::pass1) st->field_energy_push = st->field_energy;
            st->v_left = v_left;
            if (accumulate) st->v_sum += v_left;
            st->pending = 0u;  // everything of this field is done
            if (!mc) {
                R.e_gather[0] = R.periodic ? (float)pp[n - 1] : 0.0f;
                R.e_gather[n + 1] = R.periodic ? (float)pp[0] : 0.0f;
            }
        }
        if (mc) {
            // node field (E_{g-1/2} + E_{g+1/2})/2, one-sided at the electrodes
            for (int g = threadIdx.x; g <= n; g += kThreads) {
                double e;
                if (R.periodic)
                    e = 0.5 * (pp[(g - 1 + n) % n] + pp[g % n]);
                else
                    e = g == 0 ? pp[0] : (g == n ? pp[n - 1] : 0.5 * (pp[g - 1] + pp[g]));
                if (!dry) R.e_gather[g] = (float)e;
            }
        }
        __syncthreads();
        return;
    }
    // Explicit schemes: E_c = base + kappa (P_c - mean P) + K2 (c - (n-1)/2), with
    // base = V/(n dx), K2 = kappa_bg between electrodes (the constant d0 of the
    // Gauss law fixed by sum_c E_c dx = V), base = 0, K2 = -kappa Q/n in the
    // periodic box (zero-mean field, Q the total charge).  The sum of P_c is
    // exact in two 64-bit halves; everything else is double-word FP32.
    for (int k = 0; k < per; ++k) {
        const int c = c_begin + k;
        if (cursors && !dry && c < n1) {
            R.cursor[0][c] = (unsigned int)(Cx & 0xffffffffull);
            R.cursor[1][c] = (unsigned int)(Cx >> 32);
            Cx += K.c[0][c] | (K.c[1][c] << 32);
        }
        if (c < n) {
            P += (R.periodic || c >= 1) ? q[c] : 0ll;
            q[c] = P;  // this thread's own cells only
        }
    }
    if constexpr (nu_capable) if (R.stretched) {
        // Non-uniform grid, double-word FP32 like the uniform grid's solve:
        // E_c = D_0 + kappa P'_c, P'_c = P_c - Q W_c, where the periodic box
        // spreads the net charge Q over the nodes in proportion to their
        // lengths (W_c: the share of nodes 0..c; none between electrodes),
        // and D_0 = (V - kappa sum_c h_c P'_c) / L makes sum_c h_c E_c = V
        // (zero in the box).  The gather table takes the cells' voltage drops
        // h_c E_c; FP64 conversion, averages and energy are left to the next
        // launch as on the uniform grid.
        __shared__ float2 s_dw[kThreads / 32 + 1];
        const dw qnet = R.periodic ? dw_from_i64(totP) : dw{0.0f, 0.0f};
        const dw kap = dw_of(R.kappa_ff);
        dw sh = {0.0f, 0.0f};
        for (int k = 0; k < per; ++k) {
            const int c = c_begin + k;
            if (c < n) {
                const float2 w = R.wdw[c];
                const float2 h = R.hdw[c];
                const dw pc = dw_add(dw_from_i64(q[c]), dw_neg(dw_mul(qnet, dw{w.x, w.y})));
                ew[c] = make_float2(pc.hi, pc.lo);
                sh = dw_add(sh, dw_mul(dw{h.x, h.y}, pc));
            }
        }
        sh = block_sum_dw(sh, s_dw);
        const dw v = R.periodic ? dw{0.0f, 0.0f} : dw{s_vl.hi, s_vl.lo};
        const dw d0 = dw_mul(dw_add(v, dw_neg(dw_mul(kap, sh))), dw_of(R.inv_len_ff));
        double wsum = 0.0;
        for (int k = 0; k < per; ++k) {
            const int c = c_begin + k;
            if (c < n) {
                const float2 p2 = ew[c];
                const float2 h = R.hdw[c];
                const dw e = dw_add(d0, dw_mul(kap, dw{p2.x, p2.y}));
                const dw u = dw_mul(e, dw{h.x, h.y});  // the cell's voltage drop
                ew[c] = make_float2(u.hi, u.lo);
                if (dry) continue;
                R.e_gather[c + 1] = u.hi;
                if (defer) {
                    R.e_hi[c] = e.hi;
                    R.e_lo[c] = e.lo;
                } else {
                    const double ed = (double)e.hi + (double)e.lo;
                    R.e_cc[c] = ed;
                    if (accumulate) atomicAdd(&R.avg_e[c], ed);
                    wsum += ed * ed * R.h64[c];
                }
            }
        }
        __syncthreads();  // publishes ew[]
        if (threadIdx.x == 0 && !dry) {
            R.e_gather[0] = R.periodic ? ew[n - 1].x : 0.0f;
            R.e_gather[n + 1] = R.periodic ? ew[0].x : 0.0f;
            st->v_left = s_vl.v;
        }
        if (defer) {
            if (threadIdx.x == 0 && !dry) {
                if (ModeInfo<MODE>::explicit_push) st->field_energy_push = R.eps0_half * fe_acc;
                st->fe_acc = 0.0;
                st->pending = (accumulate ? 1u : 0u) | 2u;
            }
        } else {
            wsum = block_sum_lean(wsum, sc_d);
            if (threadIdx.x == 0 && !dry) {
                if (ModeInfo<MODE>::explicit_push) st->field_energy_push = st->field_energy;
                st->field_energy = R.eps0_half * wsum;
                if (accumulate) st->v_sum += s_vl.v;
                st->pending = 0u;
            }
        }
        __syncthreads();
        return;
    }
    const dw sum_p = dw_add(dw_mul(dw_from_i64(tot_hi), dw{4294967296.0f, 0.0f}), dw_from_i64((long long)tot_lo));
    const dw mean_p = dw_mul(sum_p, dw_of(R.inv_n_ff));
    const dw kap = dw_of(R.kappa_ff);
    dw base, k2;
    if (R.periodic) {
        base = dw{0.0f, 0.0f};
        k2 = dw_neg(dw_mul(dw_mul(kap, dw_from_i64(totP)), dw_of(R.inv_n_ff)));
    } else {
        base = dw_mul(dw{s_vl.hi, s_vl.lo}, dw_of(R.inv_ndx_ff));
        k2 = dw_of(R.kbg_ff);
    }
    const float mid = 0.5f * (float)(n - 1);
    double wsum = 0.0;
    for (int k = 0; k < per; ++k) {
        const int c = c_begin + k;
        if (c < n) {
            const dw d = dw_add(dw_from_i64(q[c]), dw_neg(mean_p));
            const dw e = dw_add(dw_add(base, dw_mul(kap, d)), dw_mul(k2, dw{(float)c - mid, 0.0f}));
            ew[c] = make_float2(e.hi, e.lo);
            if (dry) continue;
            if (!mc) R.e_gather[c + 1] = e.hi;
            if (defer) {
                R.e_hi[c] = e.hi;
                R.e_lo[c] = e.lo;
            } else {
                const double ed = (double)e.hi + (double)e.lo;
                R.e_cc[c] = ed;
                if (accumulate) atomicAdd(&R.avg_e[c], ed);
                wsum += ed * ed;
            }
        }
    }
    __syncthreads();  // publishes ew[]
    if (threadIdx.x == 0 && !dry) {
        if (!mc) {
            R.e_gather[0] = R.periodic ? ew[n - 1].x : 0.0f;
            R.e_gather[n + 1] = R.periodic ? ew[0].x : 0.0f;
        }
        st->v_left = s_vl.v;
    }
    if (mc) {
        // node field of the momentum-conserving scheme, (phi_{g-1} - phi_{g+1})/(2dx)
        // = (E_{g-1/2} + E_{g+1/2})/2, one-sided at the electrodes
        for (int g = threadIdx.x; g <= n; g += kThreads) {
            float e;
            if (R.periodic) {
                const float2 a = ew[(g - 1 + n) % n], b = ew[g % n];
                const dw h = dw_add(dw{a.x, a.y}, dw{b.x, b.y});
                e = 0.5f * h.hi;
            } else if (g == 0) {
                e = ew[0].x;
            } else if (g == n) {
                e = ew[n - 1].x;
            } else {
                const float2 a = ew[g - 1], b = ew[g];
                const dw h = dw_add(dw{a.x, a.y}, dw{b.x, b.y});
                e = 0.5f * h.hi;
            }
            if (!dry) R.e_gather[g] = e;
        }
    }
    if (defer) {
        if (threadIdx.x == 0 && !dry) {
            // the energy of the field this launch pushed with was summed by the
            // launch's deferred-work blocks into fe_acc
            if (ModeInfo<MODE>::explicit_push) st->field_energy_push = R.eps0_dx_half * fe_acc;
            st->fe_acc = 0.0;
            st->pending = (accumulate ? 1u : 0u) | 2u;
        }
    } else {
        wsum = block_sum_lean(wsum, sc_d);
        if (threadIdx.x == 0 && !dry) {
            if (ModeInfo<MODE>::explicit_push) st->field_energy_push = st->field_energy;
            st->field_energy = R.eps0_dx_half * wsum;
            if (accumulate) st->v_sum += s_vl.v;
            st->pending = 0u;  // everything of this field is done
        }
    }
    __syncthreads();
}

// The FP64 work a deferring tail left for nodes and cells of part `part` of
// `parts`: the newest field to FP64, the running averages, the field energy
// summed into st->fe_acc (NU: the caller may run on a non-uniform grid, where
// the energy weights each cell by its width).  Every thread of the block
// calls this.
template <bool NU>
__device__ void deferred_work(const Run &R, unsigned int pend, int part, int parts) {
    __shared__ double sc_d[kThreads / 32 + 1];
    const int n = R.n_cells;
    const int chunk = (n + 1 + parts - 1) / parts;
    const int lo = part * chunk, hi = min(lo + chunk, n + 1);
    double fe = 0.0;
    for (int k = lo + (int)threadIdx.x; k < hi; k += kThreads) {
        if (k < n) {
            const double e = (double)R.e_hi[k] + (double)R.e_lo[k];
            R.e_cc[k] = e;
            fe += (NU && R.stretched) ? e * e * R.h64[k] : e * e;  // sum_c h_c E_c^2 on a non-uniform grid
            if (pend & 1u) atomicAdd(&R.avg_e[k], e);
        }
        if (pend & 1u) {
            atomicAdd(&R.avg_ne[k], (double)R.rho_q[0][k]);
            atomicAdd(&R.avg_ni[k], (double)R.rho_q[1][k]);
        }
    }
    fe = block_sum_lean(fe, sc_d);
    if (threadIdx.x == 0) {
        if (fe != 0.0) atomicAdd(&R.st->fe_acc, fe);
        if (part == 0 && (pend & 1u)) R.st->v_sum += R.st->v_left;
    }
}

// Reset of the per-step accumulators.
__device__ void tail_reset(const Run &R) {
    const int n1 = R.n_cells + 1;
    for (int S = 0; S < 2; ++S)
        for (int k = threadIdx.x; k < n1; k += kThreads) {
            R.acc_cnt[S][k] = 0ull;
            R.acc_a[S][k] = 0ull;
            R.acc_b[S][k] = 0ull;
        }
}

// Sort cursors alone (implicit pass 2, which solves no field).
__device__ void tail_cursors(const Run &R, Keys K) {
    __shared__ long long sc_x[kThreads / 32];
    __shared__ unsigned long long sc_y[kThreads / 32];
    const int n1 = R.n_cells + 1;
    const int per = (n1 + kThreads - 1) / kThreads;
    const int b0 = threadIdx.x * per;
    unsigned long long run = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < n1) run += K.c[0][b0 + k] | (K.c[1][b0 + k] << 32);
    long long dummy = 0, tdummy;
    unsigned long long tot;
    block_exclusive_scan_pair(dummy, run, tdummy, tot, sc_x, sc_y);
    for (int k = 0; k < per; ++k) {
        const int j = b0 + k;
        if (j < n1) {
            R.cursor[0][j] = (unsigned int)(run & 0xffffffffull);
            R.cursor[1][j] = (unsigned int)(run >> 32);
            run += K.c[0][j] | (K.c[1][j] << 32);
        }
    }
    __syncthreads();
}

template <int MODE>
// dry: a warming pass by a block that is not the last (no global writes;
// phases [ph_lo, ph_hi) of 0 stage, 1 births, 2 field, 3 cursors and counters),
// so that the last block finds this code in L2 instead of fetching it cold.
// vl_state: the electrode voltage was stored in the run state at launch start
// (else the field phase computes it).
__device__ __forceinline__ void tail_body(const Run &R, unsigned char *smem, unsigned char *stage, bool diag,
                                          bool defer, bool vl_state, const uint32_t *wtab, bool dry = false,
                                          int ph_lo = 0, int ph_hi = 4) {
    using MI = ModeInfo<MODE>;
    constexpr bool births = MI::explicit_push || MI::pass2;
    DevState *st = R.st;
    __shared__ TailHead s_hd;
    const long long step = st->step;
    // One batch of independent loads: the per-key sums of both species (into
    // shared memory; everything after reads, and the births add to, this copy
    // through Ks; the global sums are cleared right behind the loads), one
    // birth record per thread, and the run-state words thread 0 updates at
    // the end.
    const int n1 = R.n_cells + 1;
    Keys Ks;
    TailHead &hd = s_hd;
    if (threadIdx.x == 0) {
        hd.nb = st->n_births;
        hd.ne = st->n_slots[0];
        hd.ni = st->n_slots[1];
        hd.id_e = st->next_id[0];
        hd.id_i = st->next_id[1];
        hd.parity = (int)st->parity;
        hd.births_total = st->births_total;
        hd.n_avg = st->n_avg;
        hd.n_diag = st->n_diag;
        hd.fe_acc = st->fe_acc;
        if (vl_state) {
            hd.vl_v = st->volt_v;
            hd.vl_hi = st->volt_hi;
            hd.vl_lo = st->volt_lo;
        }
        for (int S = 0; S < 2; ++S) {
            hd.live[S] = st->n_live[S];
            hd.absorbed[S] = st->absorbed_step[S];
            hd.ke_acc[S] = st->ke_x_acc[S];
            hd.pw_acc[S] = st->power_acc[S];
        }
    }
    Birth my = {};
    if (births && threadIdx.x < R.births_cap) my = R.births[threadIdx.x];  // beyond the step's count: unused
    {
        unsigned long long *base = (unsigned long long *)stage;
        constexpr int nk = MI::ec3 ? 4 : 3;  // sums per key
        for (int S = 0; S < 2; ++S) {
            Ks.c[S] = base + (size_t)(nk * S + 0) * n1;
            Ks.a[S] = base + (size_t)(nk * S + 1) * n1;
            Ks.b[S] = base + (size_t)(nk * S + 2) * n1;
            Ks.d[S] = MI::ec3 ? base + (size_t)(nk * S + 3) * n1 : nullptr;
        }
        constexpr int kPer = (kMaxCells + 1 + kThreads - 1) / kThreads;
        for (int S = 0; S < 2 && ph_lo <= 0; ++S) {  // per species: all loads first, then the stores
            unsigned long long v[kPer][nk];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int k = threadIdx.x + j * kThreads;
                if (k < n1) {
                    v[j][0] = R.acc_cnt[S][k];
                    v[j][1] = R.acc_a[S][k];
                    v[j][2] = R.acc_b[S][k];
                    if constexpr (MI::ec3) v[j][3] = R.acc_c[S][k];
                }
            }
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int k = threadIdx.x + j * kThreads;
                if (k < n1) {
                    Ks.c[S][k] = v[j][0];
                    Ks.a[S][k] = v[j][1];
                    Ks.b[S][k] = v[j][2];
                    if constexpr (MI::ec3) Ks.d[S][k] = v[j][3];
                    if (dry) continue;
                    R.acc_cnt[S][k] = 0ull;
                    R.acc_a[S][k] = 0ull;
                    R.acc_b[S][k] = 0ull;
                    if constexpr (MI::ec3) R.acc_c[S][k] = 0ull;
                }
            }
        }
    }
    unsigned int status_bits = 0u;
    if (threadIdx.x == 0) {
        // births recorded beyond the buffer are lost; those beyond the slots' room too
        unsigned int B = births ? hd.nb : 0u;
        if (B > (unsigned int)R.births_cap) {
            B = (unsigned int)R.births_cap;
            status_bits |= 0x2u;
        }
        long long room = R.capacity[0] - hd.ne;
        if (R.capacity[1] - hd.ni < room) room = R.capacity[1] - hd.ni;
        unsigned int ok = B;
        if ((long long)ok > room) {
            ok = room > 0 ? (unsigned int)room : 0u;
            status_bits |= 0x1u;
        }
        hd.B = B;
        hd.ok = ok;
    }
    __syncthreads();
    if (births && ph_lo <= 1 && 1 < ph_hi) tail_births<MODE>(R, Ks, smem, diag, hd, my, dry, step, wtab);
    if (ph_lo <= 2 && 2 < ph_hi) {
        const Volt vl = {hd.vl_v, hd.vl_hi, hd.vl_lo};  // read only if vl_state
        if (MI::explicit_push)
            tail_field<MODE>(R, Ks, smem, step + 1, true, true, defer, vl, vl_state, hd.fe_acc, dry);
        if (MI::pass1) tail_field<MODE>(R, Ks, smem, step + 1, true, false, defer, vl, vl_state, hd.fe_acc, dry);
        if (MI::deposit)
            tail_field<MODE>(R, Ks, smem, step, false, true, defer, vl, vl_state, hd.fe_acc, dry);
    }
    if (ph_hi <= 3) return;  // a warming pass ends here
    if (MI::pass2) tail_cursors(R, Ks);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ok = hd.ok;
        if (births) {
            st->n_slots[0] = hd.ne + ok;
            st->n_slots[1] = hd.ni + ok;
            st->next_id[0] = hd.id_e + ok;
            st->next_id[1] = hd.id_i + ok;
            st->births_total = hd.births_total + ok;
        }
        if (MI::push) {
            for (int S = 0; S < 2; ++S) {
                st->ke_x[S] = hd.ke_acc[S];
                st->power[S] = hd.pw_acc[S];
                st->ke_x_acc[S] = 0.0;
                st->power_acc[S] = 0.0;
                st->n_live[S] = hd.live[S] + (long long)ok - (long long)hd.absorbed[S];
                st->absorbed_step[S] = 0ull;
            }
            st->step = step + 1;
            st->n_avg = hd.n_avg + 1;
            if (diag) st->n_diag = hd.n_diag + 1;
        }
        if (status_bits) atomicOr(&st->status, status_bits);
        st->n_births = 0u;
        st->next_item = 0u;
        st->blocks_done = 0u;
    }
}

// Out of line for the batched kernel (register budget); the single-run
// kernel inlines the body.
template <int MODE>
__device__ __noinline__ void tail(const Run &R, unsigned char *smem, unsigned char *stage, bool diag, bool defer,
                                  bool vl_state, const uint32_t *wtab) {
    tail_body<MODE>(R, smem, stage, diag, defer, vl_state, wtab);
}

// The block's share of the particles: blocks are split between the species in
// proportion to their slots; each takes a contiguous chunk of one species,
// a multiple of 32 long (so every chunk starts 16-byte aligned).
__device__ __forceinline__ void block_segment(long long ne, long long ni, int &S, long long &b,
                                              long long &e) {
    const int G = gridDim.x;
    int ge = G;
    if (ni > 0) {
        ge = (int)(((double)G * (double)ne) / (double)(ne + ni) + 0.5);
        if (ne > 0 && ge < 1) ge = 1;
        if (ge > G - 1) ge = G - 1;
    }
    const int k = blockIdx.x < ge ? (int)blockIdx.x : (int)blockIdx.x - ge;
    const int gs = blockIdx.x < ge ? ge : G - ge;
    const long long ns = blockIdx.x < ge ? ne : ni;
    S = blockIdx.x < ge ? 0 : 1;
    long long ch = (ns + gs - 1) / gs;
    ch = (ch + 31) & ~31ll;
    b = (long long)k * ch;
    e = b + ch < ns ? b + ch : ns;
    if (b > e) b = e;
}

// ---------------------------------------------------------------------------
// Dynamic work distribution of the particle launch.  The slots of both
// species are cut into items of one tile each (electrons first, then
// ions); blocks claim items from an atomic counter until none are left, so
// blocks that met cheap particles take more of them.  Thread 0 of a block is the producer of its copy ring: it claims
// one item ahead and issues the tiles of consecutive items back to back,
// writing each tile's species, first slot and length next to the ring stage;
// the other warps consume the stages in order.  Claims only increase, so a
// block switches species at most once: its shared accumulators, tallies and
// collision queue are flushed at that switch.
// ---------------------------------------------------------------------------
constexpr int kDeferParts = 4;  // blocks that take the deferred FP64 work of the previous tail
constexpr int kWarmBlocks = 3;  // first finishers that warm the tail's code (stage, births, field)

struct Stream {
    int *S;            // [kStages] species of the staged tile
    long long *o;      // [kStages] first slot
    int *n;            // [kStages] particles (0: the stream has ended)
};

// Producer state (shared memory, used by thread 0 only).  Items are whole
// tiles: electrons first, then ions.  (Cutting the last half wave into
// quarter tiles, so that blocks finish closer together, measured 7 % slower:
// a quarter tile leaves three quarters of the block idle.)
struct Producer {
    long long pos, end, total, ne, ni;
    long long e_items;     // items of species 0
    int S;
    int k;                 // items started so far
    bool inflight;         // a claim on the counter is held in the caller's register
    bool done;
};

// Set up the item table of a launch over ne electron and ni ion slots.
__device__ __forceinline__ void producer_items(Producer &p, long long ne, long long ni) {
    p.ne = ne;
    p.ni = ni;
    p.e_items = (ne + kTile - 1) / kTile;
    p.total = p.e_items + (ni + kTile - 1) / kTile;
}

// Items: a block's first two are blockIdx.x and blockIdx.x + gridDim.x; the
// counter hands out the rest.  The claim for the item after the one being
// started is taken here into `claim`, a register of the calling thread, and
// read at the next item start, a tile later: the atomic's latency is never
// waited on (a claim kept in shared memory would stall the issuing warp on
// the store of its result).  can_claim: `claim` outlives this call.
__device__ __forceinline__ void producer_issue(const Run &R, const Ring &g, const Stream &ms, Producer &p,
                                               int par, unsigned int u, int mode_fields, bool implicit,
                                               unsigned int &claim, bool can_claim) {
    const int stage = (int)(u % kStages);
    if (p.pos >= p.end) {
        long long it = p.total;
        if (!p.done) {
            if (p.k < 2)
                it = (long long)blockIdx.x + (long long)p.k * gridDim.x;
            else
                it = (long long)(p.inflight ? claim : atomicAdd(&R.st->next_item, 1u)) + 2ll * gridDim.x;
            ++p.k;
            p.inflight = false;
            p.done = it >= p.total;
        }
        if (p.done) {
            ms.n[stage] = 0;
            return;
        }
        if (it < p.e_items) {
            p.S = 0;
            p.pos = it * kTile;
            p.end = min(p.pos + kTile, p.ne);
        } else {
            p.S = 1;
            p.pos = (it - p.e_items) * kTile;
            p.end = min(p.pos + kTile, p.ni);
        }
        if (p.k >= 2 && can_claim) {
            claim = atomicAdd(&R.st->next_item, 1u);
            p.inflight = true;
        }
    }
    const int n = (int)min((long long)kTile, p.end - p.pos);
    ms.S[stage] = p.S;
    ms.o[stage] = p.pos;
    ms.n[stage] = n;
    const unsigned int bytes = (unsigned int)(((n * 4) + 15) & ~15);  // arrays are padded to 16 bytes
    const int nf = mode_fields + (implicit ? 1 : 0);
    const Species &s = R.buf[par][p.S];
    const long long o = p.pos;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&g.bar[stage], bytes * nf);
    bulk_g2s(ring_field(g, stage, 0), s.cell + o, bytes, &g.bar[stage]);
    bulk_g2s(ring_field(g, stage, 1), s.off + o, bytes, &g.bar[stage]);
    if (mode_fields >= 3) bulk_g2s(ring_field(g, stage, 2), s.vx + o, bytes, &g.bar[stage]);
    if (implicit) bulk_g2s(ring_field(g, stage, 3), s.abar + o, bytes, &g.bar[stage]);
    p.pos += n;
}

// One staged tile of species S: n particles from slot o.  Indices handed to
// step_particle and the collision queue are absolute slots of sp.
template <int MODE>
__device__ __forceinline__ void stream_tile(const Run &R, const SmemMain &sm, const Ring &g, int stage, int S,
                                            const Species &sp, long long o, int len, bool diag,
                                            long long step, Tally &t, float &kx, float &pw) {
    constexpr int U = kUnroll;
    using MI = ModeInfo<MODE>;
    const int i0 = U * (int)threadIdx.x;  // place of the first particle in the tile
    const bool full = i0 + U - 1 < len;
    int cell[U];
    float off[U], vx[U], abar[U];
    ring_particles<MODE>(g, stage, i0, len - i0, cell, off, vx, abar);
    const SpK k = species_k(R, S);
    int key[U];
    uint32_t a[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
        a[q] = 0u;
        key[q] = -1;
        if (cell[q] < 0) continue;  // beyond the tile, or a hole left by absorption
        key[q] = step_particle<MODE, true>(R, sm, sp, k, o + i0 + q, cell[q], off[q], vx[q], abar[q], diag, step,
                                        t, kx, pw, a[q]);
    }
    if (MI::push) {
        const long long b = o + i0;
        if (full) {
            stv<U>(sp.cell + b, cell);
            stv<U>(sp.off + b, off);
            stv<U>(sp.vx + b, vx);
            if (MI::implicit) stv<U>(sp.abar + b, abar);
        } else {
#pragma unroll
            for (int q = 0; q < U; ++q) {
                if (i0 + q < len) {
                    sp.cell[b + q] = cell[q];
                    sp.off[b + q] = off[q];
                    sp.vx[b + q] = vx[q];
                    if (MI::implicit) sp.abar[b + q] = abar[q];
                }
            }
        }
    }
    if constexpr (MI::ec3)
        deposit_tile3(key, a, sm.acc);
    else
        deposit_tile(key, a, sm.acc, MI::count_only);
}

// Everything a block adds to the run for species S before it moves on: the
// deposit accumulators, the tallies and the heating profile.
template <int MODE>
__device__ void stream_flush(const Run &R, const SmemMain &sm, int S, bool diag, Tally &t) {
    using MI = ModeInfo<MODE>;
    flush_species(R, sm, S, MI::count_only, MI::ec3);
    if (MI::push) flush_tally(R, S, t);
    t = Tally{0.0f, 0.0f, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (diag) {
        __syncthreads();
        for (int k = threadIdx.x; k < R.n_cells; k += kThreads) {
            const float h = sm.heat[k];
            if (h != 0.0f) atomicAdd(&R.heat[S][k], (double)h / (MI::nu ? R.h64[k] : R.dx));
            sm.heat[k] = 0.0f;
        }
        __syncthreads();
    }
}

// Thread 0, first thing in the launch: set up the block's work items and
// issue the copies of its first tiles (static items: no wait on the counter),
// so they travel while the block reads the grid and clears its accumulators.
template <int MODE>
__device__ __forceinline__ void stream_prime(const Run &R, const Ring &g, const Stream &ms, Producer &p) {
    using MI = ModeInfo<MODE>;
    const DevState *st = R.st;
    const int par = st->parity;
    p.pos = p.end = 0;
    producer_items(p, st->n_slots[0], R.ions_mobile ? st->n_slots[1] : 0);
    p.S = 0;
    p.k = 0;
    p.inflight = p.done = false;
    unsigned int unused = 0u;
    for (int k = 0; k < kStages - 1; ++k)
        producer_issue(R, g, ms, p, par, (unsigned int)k, MI::loads_v ? 3 : 2, MI::implicit, unused, false);
}

// The block's stream of tiles (primed by stream_prime; the caller's barrier
// separates the two).
template <int MODE>
__device__ void stream_block(const Run &R, const SmemMain &sm, const Ring &g, const Stream &ms, Producer &p,
                             bool diag, long long step) {
    using MI = ModeInfo<MODE>;
    DevState *st = R.st;
    const int par = st->parity;
    const Species sp[2] = {R.buf[par][0], R.buf[par][1]};
    const int mode_fields = MI::loads_v ? 3 : 2;
    Tally t = {0.0f, 0.0f, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    float kx = 0.0f, pw = 0.0f;  // the per-particle sums stay in registers
    int cur = -1;
    long long added = 0;
    bool gave_up = false;
    unsigned int claim = 0u;  // thread 0: the counter claim in flight
    // Set by the barrier that ends a tile, the same in every thread: the tile
    // left the queue above its drain mark, or some thread's wait gave up.
    bool flag = false;
    for (unsigned int u = 0;; ++u) {
        if (flag) gave_up = __syncthreads_or(gave_up ? 1 : 0) != 0;  // which of the two (rare)
        const int stage = (int)(u % kStages);
        const int n = gave_up ? 0 : ms.n[stage];
        const int S = n ? ms.S[stage] : cur;
        const bool closing = cur >= 0 && (n == 0 || S != cur || added + n > kFlushEvery);
        // the one place the queue is drained (keeps a single inlined copy of
        // the collision code in the loop): above the drain mark, or at the end
        // of the block's stream.  The queue holds both species, so the switch
        // from electrons to ions does not drain it (a drain is a few
        // microseconds of latency for the whole block).  Every thread must take
        // the same branch: the count decides only where the barrier that ended
        // the last tile had already seen it above the mark (`flag`), or at the
        // end of the stream, after which nothing is queued; a thread that read
        // it after another had started the next tile would enter the drain's
        // barriers alone.
        if (MI::push && R.mcc && cur >= 0) {
            const unsigned int qn = *sm.q.n;
            if (n == 0 ? qn > 0u : (flag && qn > kQueueDrainAbove)) drain_q<true>(R, sm, sp[0], sp[1], step, diag, t);
        }
        if (closing) {
            t.kx += kx;
            t.pw += pw;
            kx = pw = 0.0f;
            stream_flush<MODE>(R, sm, cur, diag, t);
            added = 0;
        }
        if (n == 0) break;
        cur = S;
        const long long o = ms.o[stage];
        if (threadIdx.x == 0)
            producer_issue(R, g, ms, p, par, u + kStages - 1, mode_fields, MI::implicit, claim, true);
        if (!mbar_wait(R, &g.bar[stage], (u / kStages) & 1u)) {
            // give up, but not before the copies already issued have landed (bounded)
            for (unsigned int w = u + 1; w < u + kStages; ++w)
                if (ms.n[w % kStages] > 0) mbar_wait(R, &g.bar[w % kStages], (w / kStages) & 1u);
            gave_up = true;
        } else {
            stream_tile<MODE>(R, sm, g, stage, S, S ? sp[1] : sp[0], o, n, diag, step, t, kx, pw);
        }
        added += n;
        // The stage is free again.  The thread that queued the tile's last
        // particle reads the queue count after doing so, so the OR over the
        // block sees the final count; a thread whose wait gave up ends the
        // stream for the whole block at the next pass.
        flag = __syncthreads_or((gave_up || (MI::push && R.mcc && *sm.q.n > kQueueDrainAbove)) ? 1 : 0) != 0;
    }
}

// ---------------------------------------------------------------------------
// The particle kernel: one launch per explicit step / implicit pass / deposit.
// ---------------------------------------------------------------------------
// The m = 3 modes hold three blocks per SM (their shared memory), so they
// may use the registers of three.
template <int MODE>
__global__ void __launch_bounds__(kThreads,
                                  (MODE == kExplicitEC3 || MODE == kDepositEC3 || MODE == kExplicitEC3NU) ? 3 : kMinBlocks)
    k_particles(Run R) {
    extern __shared__ __align__(128) unsigned char smem_all[];
    __shared__ bool s_last;
    __shared__ int s_warm;
    __shared__ __align__(8) unsigned long long s_bar[kStages];
    __shared__ unsigned int s_uses;
    __shared__ int s_ms_S[kStages], s_ms_n[kStages];
    __shared__ long long s_ms_o[kStages];
    __shared__ Producer s_prod;
    using MI = ModeInfo<MODE>;
    DevState *st = R.st;
    const int n = R.n_cells;
    Ring g;
    g.buf = (uint32_t *)smem_all;
    g.bar = s_bar;
    g.uses = &s_uses;
    g.nf = MI::implicit ? kMaxFields : kMaxFields - 1;
    const Stream ms = {s_ms_S, s_ms_o, s_ms_n};
    unsigned char *smem = smem_all + ring_bytes(MI::implicit);  // grid, accumulators, queue; the tail's space
    __shared__ uint32_t s_wtab[kWaitTab];
    const SmemMain sm = carve_main(smem, n, R.eedf_bins, MI::ec3, s_wtab, MI::nu);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[s], 1u);
        s_uses = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stream_prime<MODE>(R, g, ms, s_prod);
    }
    const long long step = st->step;
    const bool diag = MI::push && R.diag_period > 0 && (step % R.diag_period) == 0;
    // shared-memory grid
    if (MI::needs_field)
        for (int k = threadIdx.x; k < n + 2; k += kThreads) sm.e[k] = R.e_gather[k];
    if (MI::nu)
        for (int k = threadIdx.x; k < n; k += kThreads) sm.hw[k] = R.hw[k];
    if (MI::push) load_wait_tab(R, s_wtab);
    for (int k = threadIdx.x; k <= n; k += kThreads) {
        sm.acc.cnt[k] = 0u;
        sm.acc.a[k] = 0u;
        sm.acc.bh[k] = 0u;
        sm.acc.bl[k] = 0u;
        if (MI::ec3) {
            sm.acc.s3h[k] = 0u;
            sm.acc.s3m[k] = 0u;
            sm.acc.s3l[k] = 0u;
        }
    }
    if (diag) {
        for (int k = threadIdx.x; k < n; k += kThreads) sm.heat[k] = 0.0f;
        for (int k = threadIdx.x; k <= R.eedf_bins; k += kThreads) sm.eedf[k] = 0u;
    }
    if (threadIdx.x == 0) *sm.q.n = 0u;
    __syncthreads();
    // the FP64 work the previous tail left (a few blocks; the others start streaming)
    {
        const unsigned int pend = st->pending;
        if (pend && blockIdx.x < kDeferParts)
            deferred_work<MI::nu || MODE == kDepositEC || MODE == kDepositEC3>(R, pend, (int)blockIdx.x, kDeferParts);
    }
    // The electrode voltage of the field the tail solves: FP64 is slow here,
    // so one thread of one block (past the deferring ones) computes it while
    // the rest stream, and stores it for the tail.  Its block's arrival
    // fence below orders the store before the last block's reads.
    if (blockIdx.x == (gridDim.x > (unsigned int)kDeferParts ? (unsigned int)kDeferParts : 0u) && threadIdx.x == 0) {
        const Volt v = electrode_volt(R, MI::deposit ? step : step + 1);
        st->volt_v = v.v;
        st->volt_hi = v.hi;
        st->volt_lo = v.lo;
    }
    stream_block<MODE>(R, sm, g, ms, s_prod, diag, step);
    if (diag) {
        for (int k = threadIdx.x; k <= R.eedf_bins; k += kThreads)
            if (sm.eedf[k]) atomicAdd(&R.eedf[k], (unsigned long long)sm.eedf[k]);
    }
    // The last block runs the tail.  The first kWarmBlocks to finish each run
    // one phase of it as a dry pass (no global writes): the tail's code is
    // otherwise fetched cold by the last block, from DRAM after an L2 flush.
    // One call site, so the warming passes run the very same code.
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int k = atomicAdd(&st->blocks_done, 1u);
        s_last = k == gridDim.x - 1;
        s_warm = (!s_last && k < (unsigned int)kWarmBlocks) ? (int)k : -1;
    }
    __syncthreads();
    if (!s_last && s_warm < 0) return;
    if (s_last) __threadfence();
    tail_body<MODE>(R, smem_all + tail_stage_bytes(n, MI::ec3), smem_all, diag, true, true, s_wtab, !s_last,
                    s_last ? 0 : s_warm, s_last ? 4 : s_warm + 1);
}

// The work the last tail left, before the host reads diagnostics (one block).
__global__ void __launch_bounds__(kThreads) k_finalize(Run R) {
    const unsigned int pend = R.st->pending;
    if (!pend) return;
    deferred_work<true>(R, pend, 0, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        R.st->field_energy = (R.stretched ? R.eps0_half : R.eps0_dx_half) * R.st->fe_acc;
        R.st->pending = 0u;
    }
}

// ---------------------------------------------------------------------------
// Counting sort by deposit key (nearest node for S_2, cell for S_1): the
// cursors were prepared by the previous tail; live particles are scattered
// into the other buffer, holes are dropped.
// ---------------------------------------------------------------------------
// Scatter the live particles of [b, e) of species S into the other buffer at
// the cursor of their key (warp-aggregated: lanes sharing a key take
// consecutive positions from one atomic).
__device__ void sort_chunk(const Run &R, int par, int S, long long b, long long e) {
#ifndef PIC_SORT_V
#define PIC_SORT_V 4
#endif
    constexpr int V = PIC_SORT_V;  // particles per thread in flight: all their loads are issued first
    // the key of the deposit: the cell for S_1 and for the m = 3 scheme, the
    // nearest node for S_2
    const bool mc = R.scheme == 1 || R.scheme == 3 || R.scheme == 4;
    const bool implicit = R.scheme == 2 || R.scheme == 3;
    const int lane = threadIdx.x & 31;
    const Species src = R.buf[par][S], dst = R.buf[par ^ 1][S];
    for (long long base = b; base < e; base += (long long)kThreads * V) {
        int cell[V];
        float off[V], vx[V], vy[V], vz[V], ab[V];
        uint32_t id[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const long long i = base + (long long)q * kThreads + threadIdx.x;
            const bool ok = i < e;
            cell[q] = ok ? src.cell[i] : -1;
            off[q] = ok ? src.off[i] : 0.0f;
            vx[q] = ok ? src.vx[i] : 0.0f;
            vy[q] = ok ? src.vy[i] : 0.0f;
            vz[q] = ok ? src.vz[i] : 0.0f;
            id[q] = ok ? src.id[i] : 0u;
            ab[q] = (ok && implicit) ? src.abar[i] : 0.0f;
        }
        // the cursor claims of all V groups are issued before any result is
        // used: one round trip to L2 per batch, not V
        int key[V];
        unsigned int peers[V], claim[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            uint32_t a;
            const int c = cell[q] & (int)kCellMask;
            key[q] = cell[q] < 0 ? -1 : (mc ? deposit_key_s1(c, off[q], a) : deposit_key_s2(c, off[q], a));
            peers[q] = __match_any_sync(FULL_MASK, key[q]);
            claim[q] = 0u;
            if (key[q] >= 0 && lane == __ffs(peers[q]) - 1)
                claim[q] = atomicAdd(&R.cursor[S][key[q]], (unsigned int)__popc(peers[q]));
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const unsigned int base_pos = __shfl_sync(FULL_MASK, claim[q], __ffs(peers[q]) - 1);
            if (key[q] >= 0) {
                const unsigned int pos = base_pos + __popc(peers[q] & ((1u << lane) - 1u));
                dst.cell[pos] = cell[q];
                dst.off[pos] = off[q];
                dst.vx[pos] = vx[q];
                dst.vy[pos] = vy[q];
                dst.vz[pos] = vz[q];
                dst.id[pos] = id[q];
                if (implicit) dst.abar[pos] = ab[q];
            }
        }
    }
}

// After the last scatter of a run: switch buffers; holes are gone.
__device__ void sort_finish(const Run &R) {
    DevState *st = R.st;
    st->parity ^= 1u;
    st->n_slots[0] = st->n_live[0];
    st->n_slots[1] = st->n_live[1];
    st->sort_blocks_done = 0u;
}

#ifndef PIC_SORT_MIN_BLOCKS
#define PIC_SORT_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(kThreads, PIC_SORT_MIN_BLOCKS) k_sort(Run R) {
    __shared__ bool s_last;
    DevState *st = R.st;
    const int par = st->parity;
    long long b, e;
    int S;
    block_segment(st->n_slots[0], R.ions_mobile ? st->n_slots[1] : 0, S, b, e);
    if (b < e) sort_chunk(R, par, S, b, e);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->sort_blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) sort_finish(R);
}

// ---------------------------------------------------------------------------
// Uniform Maxwellian load (Sec. 3: the gap is filled uniformly at t = 0).
// Position in cell units = w0 * n / 2^32, cut to 24 fractional bits (exact in
// the FP32 offset); velocities from two Box-Muller pairs.
// ---------------------------------------------------------------------------
__global__ void k_load(Run R, int S, long long count, float vth) {
    const Species sp = R.buf[0][S];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 w = draw(R, (uint32_t)i, 0, S, kTagLoad, 0);
        const uint4 w2 = draw(R, (uint32_t)i, 0, S, kTagLoad, 1);
        const unsigned long long t = (unsigned long long)w.x * (unsigned long long)R.n_cells;
        int cell = (int)(t >> 32);
        float off = (float)((uint32_t)t >> 8) * 5.9604644775390625e-8f;
        if (R.stretched) {
            // non-uniform grid: uniform in x = (w / 2^32) L; the cell by
            // bisection over the node positions, the offset rounded to FP32
            const double x = ldexp((double)w.x, -32) * R.xnode[R.n_cells];
            int lo = 0, hi = R.n_cells;  // xnode[lo] <= x < xnode[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (R.xnode[mid] <= x)
                    lo = mid;
                else
                    hi = mid;
            }
            double o = (x - R.xnode[lo]) / R.h64[lo];
            if (o >= 1.0) o = 0.99999999999999989;  // rounding at the right node
            cell = lo;
            off = (float)o;
            if (off >= 1.0f) {  // rounds onto the next node
                if (cell + 1 < R.n_cells) {
                    off = 0.0f;
                    cell += 1;
                } else {
                    off = 0.99999994f;  // stays below x = L
                }
            }
        }
        // the first wait to a null-collision selection is drawn at the load
        sp.cell[i] = cell | (R.mcc ? (int32_t)wait_bits(draw_wait(R, R.wait_tab, S, (uint32_t)i, 0, 1)) : 0);
        sp.off[i] = off;
        float n1, n2, n3, n4;
        box_muller(u24c(w.y), u24c(w.z), n1, n2);
        box_muller(u24c(w.w), u24c(w2.x), n3, n4);
        sp.vx[i] = vth * n1;
        sp.vy[i] = vth * n2;
        sp.vz[i] = vth * n3;
        sp.id[i] = (uint32_t)i;
        if (R.scheme == 2 || R.scheme == 3) sp.abar[i] = 0.0f;
    }
}

// abar = (q/m) E(x) for the implicit scheme's first step.
__global__ void k_set_abar(Run R) {
    const DevState *st = R.st;
    const int par = st->parity;
    for (int S = 0; S < 2; ++S) {
        const Species sp = R.buf[par][S];
        const long long n = st->n_slots[S];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            if (sp.cell[i] < 0) continue;
            const int cell = sp.cell[i] & (int)kCellMask;
            const float off = sp.off[i];
            float e;
            if (R.scheme == 3) {  // node field, linear weights
                e = (1.0f - off) * R.e_gather[cell] + off * R.e_gather[cell + 1];
            } else {
                const int j = cell + (off >= 0.5f ? 1 : 0);
                const float w1 = off >= 0.5f ? off - 0.5f : off + 0.5f;
                e = (1.0f - w1) * R.e_gather[j] + w1 * R.e_gather[j + 1];
                if (R.stretched) e *= R.hw[cell].y;  // voltage drops over the cell width
            }
            sp.abar[i] = R.qm[S] * e;
        }
    }
}

// Validation of uploaded particles (pic_set_particles).
__global__ void k_check_particles(const int32_t *__restrict__ cell, const float *__restrict__ off, long long n,
                                  int n_cells, unsigned int *flag) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = cell[i];
        const float o = off[i];
        bad |= c < 0 || c >= n_cells || !(o >= 0.0f) || !(o < 1.0f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

cudaError_t launch_check_particles(const int32_t *cell, const float *off, long long n, int n_cells,
                                   unsigned int *flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long grid = (n + 4 * kThreads - 1) / (4 * kThreads);
    if (grid > 4096) grid = 4096;
    k_check_particles<<<(int)grid, kThreads, 0, s>>>(cell, off, n, n_cells, flag);
    return cudaGetLastError();
}

// After the check (flag clear): the uploaded particles of one species from
// the idle buffer into the current one, and the species' counters.  A set
// flag leaves everything as it was; the caller reads the flag afterwards.
// With collisions every uploaded particle draws its first wait to a
// selection at the run's current step.  16-byte copies: every array starts
// 256-byte aligned.
__device__ __forceinline__ int32_t entry_word(const Run &R, int S, int32_t cell, uint32_t id, long long step) {
    return R.mcc ? cell | (int32_t)wait_bits(draw_wait(R, R.wait_tab, S, id, step, 1)) : cell;
}

__global__ void k_apply_particles(Run R, Species dst, Species src, long long n, bool abar_given,
                                  const unsigned int *flag, int S, unsigned int next_id) {
    if (*flag) return;
    DevState *st = R.st;
    const long long step = st->step;
    const long long n4 = n >> 2, stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long j = t0; j < n4; j += stride) {
        int4 c = reinterpret_cast<const int4 *>(src.cell)[j];
        const uint4 id = reinterpret_cast<const uint4 *>(src.id)[j];
        c.x = entry_word(R, S, c.x, id.x, step);
        c.y = entry_word(R, S, c.y, id.y, step);
        c.z = entry_word(R, S, c.z, id.z, step);
        c.w = entry_word(R, S, c.w, id.w, step);
        reinterpret_cast<int4 *>(dst.cell)[j] = c;
        reinterpret_cast<float4 *>(dst.off)[j] = reinterpret_cast<const float4 *>(src.off)[j];
        reinterpret_cast<float4 *>(dst.vx)[j] = reinterpret_cast<const float4 *>(src.vx)[j];
        reinterpret_cast<float4 *>(dst.vy)[j] = reinterpret_cast<const float4 *>(src.vy)[j];
        reinterpret_cast<float4 *>(dst.vz)[j] = reinterpret_cast<const float4 *>(src.vz)[j];
        reinterpret_cast<uint4 *>(dst.id)[j] = id;
        if (dst.abar)
            reinterpret_cast<float4 *>(dst.abar)[j] =
                abar_given ? reinterpret_cast<const float4 *>(src.abar)[j] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    for (long long i = 4 * n4 + t0; i < n; i += stride) {
        dst.cell[i] = entry_word(R, S, src.cell[i], src.id[i], step);
        dst.off[i] = src.off[i];
        dst.vx[i] = src.vx[i];
        dst.vy[i] = src.vy[i];
        dst.vz[i] = src.vz[i];
        dst.id[i] = src.id[i];
        if (dst.abar) dst.abar[i] = abar_given ? src.abar[i] : 0.0f;
    }
    if (t0 == 0) {
        st->n_slots[S] = n;
        st->n_live[S] = n;
        st->next_id[S] = next_id;
    }
}

cudaError_t launch_apply_particles(const Run &r, const Species &dst, const Species &src, long long n,
                                   bool abar_given, const unsigned int *flag, int S, unsigned int next_id,
                                   cudaStream_t s) {
    long long grid = (n / 4 + kThreads - 1) / kThreads;
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    k_apply_particles<<<(int)grid, kThreads, 0, s>>>(r, dst, src, n, abar_given, flag, S, next_id);
    return cudaGetLastError();
}

// Kinetic energy of the transverse velocities (diagnostics only): four
// particles a thread per pass with 16-byte loads (slot arrays are 256-byte
// aligned), their FP32 sum added in FP64.
__global__ void k_perp_energy(Run R) {
    const DevState *st = R.st;
    const int par = st->parity;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    for (int S = 0; S < 2; ++S) {
        const Species sp = R.buf[par][S];
        const long long n = st->n_slots[S], n4 = n >> 2;
        double acc = 0.0;
        for (long long j = t0; j < n4; j += stride) {
            const int4 c = reinterpret_cast<const int4 *>(sp.cell)[j];
            const float4 y = reinterpret_cast<const float4 *>(sp.vy)[j];
            const float4 z = reinterpret_cast<const float4 *>(sp.vz)[j];
            const float e = (c.x >= 0 ? y.x * y.x + z.x * z.x : 0.0f) + (c.y >= 0 ? y.y * y.y + z.y * z.y : 0.0f) +
                            (c.z >= 0 ? y.z * y.z + z.z * z.z : 0.0f) + (c.w >= 0 ? y.w * y.w + z.w * z.w : 0.0f);
            acc += (double)e;
        }
        for (long long i = 4 * n4 + t0; i < n; i += stride) {
            if (sp.cell[i] < 0) continue;
            const float vy = sp.vy[i], vz = sp.vz[i];
            acc += (double)(vy * vy + vz * vz);
        }
        const double tot = warp_sum(acc);
        if ((threadIdx.x & 31) == 0 && tot != 0.0) atomicAdd(&R.st->ke_perp[S], tot * R.half_m_w[S]);
    }
}

__global__ void k_philox_fill(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                              uint32_t c3, long long n, uint32_t *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), k0, k1);
        reinterpret_cast<uint4 *>(out)[i] = w;
    }
}

// ---------------------------------------------------------------------------
// Batched runs: one persistent launch per phase over many independent runs of
// uneven size.  Work items are (run, species, chunk of `chunk` particles),
// claimed dynamically from a global counter; every block derives the same
// item table from the per-run work counts, which only change at the very
// end of a launch.  The block that finishes a run's last item runs that
// run's tail inside the same launch, so one run's serial field solve
// overlaps other runs' particle work.  Phases: 0 = explicit step or
// implicit pass 1; 1 = implicit pass 2; 2 = counting sort.
// ---------------------------------------------------------------------------
template <int MODE>
__device__ void batch_item(const Run &R, unsigned char *smem, const Ring &g, int S, long long b, long long e,
                           unsigned int items_r, int r, int &loaded_run, uint32_t *wtab) {
    using MI = ModeInfo<MODE>;
    __shared__ bool s_last;
    DevState *st = R.st;
    const int n = R.n_cells;
    const SmemMain sm = carve_main(smem, n, R.eedf_bins, false, wtab);
    const long long step = st->step;
    const bool diag = MI::push && R.diag_period > 0 && (step % R.diag_period) == 0;
    if (loaded_run != r) {
        if (MI::needs_field)
            for (int k = threadIdx.x; k < n + 2; k += kThreads) sm.e[k] = R.e_gather[k];
        if (MI::push || MI::pass2) load_wait_tab(R, wtab);
        for (int k = threadIdx.x; k <= n; k += kThreads) {
            sm.acc.cnt[k] = 0u;
            sm.acc.a[k] = 0u;
            sm.acc.bh[k] = 0u;
            sm.acc.bl[k] = 0u;
        }
        loaded_run = r;
    }
    if (diag) {
        for (int k = threadIdx.x; k < n; k += kThreads) sm.heat[k] = 0.0f;
        for (int k = threadIdx.x; k <= R.eedf_bins; k += kThreads) sm.eedf[k] = 0u;
    }
    if (threadIdx.x == 0) *sm.q.n = 0u;
    __syncthreads();
    if (b < e) {
        Tally t = {0.0f, 0.0f, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        const Species sp = R.buf[st->parity][S];
        for (long long sb = b; sb < e; sb += kFlushEvery) {
            const long long se = sb + kFlushEvery < e ? sb + kFlushEvery : e;
            if (S == 0)
                process_segment<MODE, 0>(R, sm, g, sp, sb, se, diag, step, t);
            else
                process_segment<MODE, 1>(R, sm, g, sp, sb, se, diag, step, t);
            flush_species(R, sm, S, MI::count_only);
        }
        if (MI::push) flush_tally(R, S, t);
        if (diag) {
            __syncthreads();
            for (int k = threadIdx.x; k < n; k += kThreads) {
                const float h = sm.heat[k];
                if (h != 0.0f) atomicAdd(&R.heat[S][k], (double)h / R.dx);
            }
            for (int k = threadIdx.x; k <= R.eedf_bins; k += kThreads)
                if (sm.eedf[k]) atomicAdd(&R.eedf[k], (unsigned long long)sm.eedf[k]);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->blocks_done, 1u) == items_r - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        tail<MODE>(R, (unsigned char *)g.buf + tail_stage_bytes(n), (unsigned char *)g.buf, diag, false, false, wtab);
        loaded_run = -1;  // the tail reused the shared memory
        __syncthreads();
    }
}

__device__ void batch_sort_item(const Run &R, int S, long long b, long long e, unsigned int items_r) {
    __shared__ bool s_last;
    DevState *st = R.st;
    if (b < e) sort_chunk(R, st->parity, S, b, e);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->sort_blocks_done, 1u) == items_r - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) sort_finish(R);
        __syncthreads();
    }
}

template <int PHASE>
__global__ void __launch_bounds__(kThreads, 2) k_batch(const Run *__restrict__ runs, int nruns,
                                                       long long *work, BatchState *bs, long long chunk,
                                                       int table_off) {
    extern __shared__ __align__(128) unsigned char smem_all[];
    __shared__ unsigned int sc_u[33];
    __shared__ unsigned int s_item;
    __shared__ bool s_glast;
    __shared__ __align__(8) unsigned long long s_bar[kStages];
    __shared__ unsigned int s_uses;
    __shared__ uint32_t s_wtab[kWaitTab];
    unsigned int *table = (unsigned int *)(smem_all + table_off);  // [2 nruns + 1] item prefix
    Ring g;
    g.buf = (uint32_t *)smem_all;
    g.bar = s_bar;
    g.uses = &s_uses;
    g.nf = kMaxFields;
    unsigned char *smem = smem_all + ring_bytes(true);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[s], 1u);
        s_uses = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int nj = 2 * nruns;
    // items per (run, species); a run with no particles still gets one empty
    // item so that its tail (field solve, step counter) runs
    const int per = (nj + kThreads - 1) / kThreads;
    const int j0 = threadIdx.x * per;
    unsigned int run_sum = 0;
    for (int q = 0; q < per; ++q) {
        const int j = j0 + q;
        if (j >= nj) break;
        const Run &R = runs[j >> 1];
        const bool part = PHASE == 1 ? (R.scheme == 2 || R.scheme == 3) : true;
        const int S = j & 1;
        const long long nn = (S == 1 && !R.ions_mobile) ? 0 : work[j];
        unsigned int it = part ? (unsigned int)((nn + chunk - 1) / chunk) : 0u;
        if (part && S == 0 && it == 0) {
            const long long n1 = R.ions_mobile ? work[j + 1] : 0;
            if (n1 == 0) it = 1u;
        }
        table[j] = it;
        run_sum += it;
    }
    unsigned int total;
    unsigned int ex = block_exclusive_scan<unsigned int>(run_sum, sc_u, total);
    for (int q = 0; q < per; ++q) {
        const int j = j0 + q;
        if (j >= nj) break;
        const unsigned int it = table[j];
        table[j] = ex;
        ex += it;
    }
    if (threadIdx.x == 0) table[nj] = total;
    __syncthreads();
    int loaded_run = -1;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&bs->next_item, 1u);
        __syncthreads();
        const unsigned int item = s_item;
        __syncthreads();
        if (item >= total) break;
        int lo = 0, hi = nj - 1;  // largest j with table[j] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid] <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int j = lo, r = j >> 1, S = j & 1;
        const Run &R = runs[r];
        const unsigned int items_r = table[2 * r + 2] - table[2 * r];
        const long long nn = (S == 1 && !R.ions_mobile) ? 0 : work[j];
        const long long b0 = (long long)(item - table[j]) * chunk;
        const long long b = b0 < nn ? b0 : nn;
        const long long e = b0 + chunk < nn ? b0 + chunk : nn;
        if (PHASE == 2) {
            batch_sort_item(R, S, b, e, items_r);
        } else if (PHASE == 1) {
            if (R.scheme == 3)
                batch_item<kImplicit2MC>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
            else
                batch_item<kImplicit2>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
        } else if (R.scheme == 0) {
            batch_item<kExplicitEC>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
        } else if (R.scheme == 1) {
            batch_item<kExplicitMC>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
        } else if (R.scheme == 2) {
            batch_item<kImplicit1>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
        } else {
            batch_item<kImplicit1MC>(R, smem, g, S, b, e, items_r, r, loaded_run, s_wtab);
        }
    }
    // the last block of the launch publishes the work counts of the next one
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_glast = atomicAdd(&bs->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_glast) return;
    __threadfence();
    for (int j = threadIdx.x; j < nj; j += kThreads) work[j] = runs[j >> 1].st->n_slots[j & 1];
    if (threadIdx.x == 0) {
        bs->next_item = 0u;
        bs->blocks_done = 0u;
        bs->launches += 1;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int block_smem_bytes(const Run &r) {
    const bool implicit = r.scheme == 2 || r.scheme == 3, ec3 = r.scheme == 4;
    const size_t a = ring_bytes(implicit) + main_smem_bytes(r.n_cells, r.eedf_bins, ec3, r.stretched != 0);
    const size_t b = tail_stage_bytes(r.n_cells, ec3) + tail_smem_bytes(r.n_cells);
    return (int)(a > b ? a : b);
}

// The dynamic shared-memory limit of every mode is raised once by
// occupancy_grid() before any launch (never during stream capture).
template <int MODE>
static cudaError_t launch_mode(const Run &r, int grid, cudaStream_t s) {
    const int smem = block_smem_bytes(r);
    k_particles<MODE><<<grid, kThreads, smem, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_particles(const Run &r, Mode m, int grid, cudaStream_t s) {
    switch (m) {
        case kExplicitEC: return launch_mode<kExplicitEC>(r, grid, s);
        case kExplicitMC: return launch_mode<kExplicitMC>(r, grid, s);
        case kDepositEC: return launch_mode<kDepositEC>(r, grid, s);
        case kDepositMC: return launch_mode<kDepositMC>(r, grid, s);
        case kImplicit1: return launch_mode<kImplicit1>(r, grid, s);
        case kImplicit2: return launch_mode<kImplicit2>(r, grid, s);
        case kImplicit1MC: return launch_mode<kImplicit1MC>(r, grid, s);
        case kImplicit2MC: return launch_mode<kImplicit2MC>(r, grid, s);
        case kExplicitEC3: return launch_mode<kExplicitEC3>(r, grid, s);
        case kDepositEC3: return launch_mode<kDepositEC3>(r, grid, s);
        case kExplicitNU: return launch_mode<kExplicitNU>(r, grid, s);
        case kImplicit1NU: return launch_mode<kImplicit1NU>(r, grid, s);
        case kImplicit2NU: return launch_mode<kImplicit2NU>(r, grid, s);
        case kExplicitEC3NU: return launch_mode<kExplicitEC3NU>(r, grid, s);
    }
    return cudaErrorInvalidValue;
}

// A kernel's dynamic shared-memory limit only ever rises (per device):
// handles of different sizes live side by side in one process, and each
// launch asks for its own size.
static cudaError_t raise_smem_limit(const void *func, int smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> raised;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &cur = raised[std::make_pair(func, dev)];
    if (smem <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

template <int MODE>
static cudaError_t occ(const Run &r, int *per_sm) {
    const int smem = block_smem_bytes(r);
    const cudaError_t e = raise_smem_limit((const void *)k_particles<MODE>, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_particles<MODE>, kThreads, smem);
}

cudaError_t occupancy_grid(const Run &r, Mode m, int *grid) {
    int dev = 0, sms = 0, per = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 14; ++k) {  // raise the shared-memory limit of every mode
        int dummy = 0;
        switch (k) {
            case 0: e = occ<kExplicitEC>(r, &dummy); break;
            case 1: e = occ<kExplicitMC>(r, &dummy); break;
            case 2: e = occ<kDepositEC>(r, &dummy); break;
            case 3: e = occ<kDepositMC>(r, &dummy); break;
            case 4: e = occ<kImplicit1>(r, &dummy); break;
            case 5: e = occ<kImplicit2>(r, &dummy); break;
            case 6: e = occ<kImplicit1MC>(r, &dummy); break;
            case 7: e = occ<kImplicit2MC>(r, &dummy); break;
            case 8: e = occ<kExplicitEC3>(r, &dummy); break;
            case 9: e = occ<kDepositEC3>(r, &dummy); break;
            case 10: e = occ<kExplicitNU>(r, &dummy); break;
            case 11: e = occ<kImplicit1NU>(r, &dummy); break;
            case 12: e = occ<kImplicit2NU>(r, &dummy); break;
            default: e = occ<kExplicitEC3NU>(r, &dummy); break;
        }
        if (e != cudaSuccess) return e;
    }
    switch (m) {
        case kExplicitEC: e = occ<kExplicitEC>(r, &per); break;
        case kExplicitMC: e = occ<kExplicitMC>(r, &per); break;
        case kDepositEC: e = occ<kDepositEC>(r, &per); break;
        case kDepositMC: e = occ<kDepositMC>(r, &per); break;
        case kImplicit1: e = occ<kImplicit1>(r, &per); break;
        case kImplicit2: e = occ<kImplicit2>(r, &per); break;
        case kImplicit1MC: e = occ<kImplicit1MC>(r, &per); break;
        case kImplicit2MC: e = occ<kImplicit2MC>(r, &per); break;
        case kExplicitEC3: e = occ<kExplicitEC3>(r, &per); break;
        case kDepositEC3: e = occ<kDepositEC3>(r, &per); break;
        case kExplicitNU: e = occ<kExplicitNU>(r, &per); break;
        case kImplicit1NU: e = occ<kImplicit1NU>(r, &per); break;
        case kImplicit2NU: e = occ<kImplicit2NU>(r, &per); break;
        case kExplicitEC3NU: e = occ<kExplicitEC3NU>(r, &per); break;
    }
    if (e != cudaSuccess) return e;
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

cudaError_t launch_finalize(const Run &r, cudaStream_t s) {
    k_finalize<<<1, kThreads, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Run &r, int grid, cudaStream_t s) {
    k_sort<<<grid, kThreads, 0, s>>>(r);
    return cudaGetLastError();
}

// Grid of the sort: as many resident blocks as fit (the scatter is latency-bound).
cudaError_t sort_grid(int *grid) {
    int dev = 0, sms = 0, per = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sort, kThreads, 0);
    if (e != cudaSuccess) return e;
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

cudaError_t launch_set_abar(const Run &r, cudaStream_t s) {
    k_set_abar<<<1024, kThreads, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_perp_energy(const Run &r, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_perp_energy<<<sms * 4, kThreads, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                               uint32_t c3, long long n, uint32_t *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_philox_fill<<<1024, kThreads, 0, s>>>(k0, k1, c0, c1, c2, c3, n, out);
    return cudaGetLastError();
}

size_t batch_smem_bytes(int max_cells, int max_bins, int nruns, int *table_off) {
    const size_t a = ring_bytes(true) + main_smem_bytes(max_cells, max_bins, false);
    const size_t b = tail_stage_bytes(max_cells) + tail_smem_bytes(max_cells);
    const size_t off = ((a > b ? a : b) + 15) & ~size_t(15);
    *table_off = (int)off;
    return off + 4 * (size_t)(2 * nruns + 1);
}

template <int PHASE>
static cudaError_t batch_attr(int smem) {
    return raise_smem_limit((const void *)k_batch<PHASE>, smem);
}

cudaError_t batch_prepare(int smem, int *grid) {
    cudaError_t e = batch_attr<0>(smem);
    if (e == cudaSuccess) e = batch_attr<1>(smem);
    if (e == cudaSuccess) e = batch_attr<2>(smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per0 = 1, per1 = 1;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per0, k_batch<0>, kThreads, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_batch<1>, kThreads, smem);
    if (e != cudaSuccess) return e;
    int per = per0 < per1 ? per0 : per1;
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

cudaError_t launch_batch(int phase, const Run *runs, int nruns, long long *work, BatchState *bs,
                         long long chunk, int grid, int smem, int table_off, cudaStream_t s) {
    if (phase == 0)
        k_batch<0><<<grid, kThreads, smem, s>>>(runs, nruns, work, bs, chunk, table_off);
    else if (phase == 1)
        k_batch<1><<<grid, kThreads, smem, s>>>(runs, nruns, work, bs, chunk, table_off);
    else
        k_batch<2><<<grid, kThreads, smem, s>>>(runs, nruns, work, bs, chunk, table_off);
    return cudaGetLastError();
}

cudaError_t launch_load(const Run &r, int species, long long n, float vth, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_load<<<1024, kThreads, 0, s>>>(r, species, n, vth);
    return cudaGetLastError();
}

}  // namespace pic

// ===========================================================================
// Charge assignment without caller-provided scratch (pic_deposit_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// charge density: code running inside another framework's memory pool that
// forbids foreign allocations, real-time loops that must not hit the
// allocator, or tools that only hold the particle arrays.  For them the
// per-node sums live in this file-scope device array, sized for the largest
// grid the library accepts.  Every GPU that loads the library keeps it
// (about 25 KB) until the process exits.  All calls on a device share it, so
// calls that overlap on the GPU (different streams, or a second call
// enqueued before the first finished on another stream) race; calls on one
// stream are ordered and safe.
// ===========================================================================
namespace pic {
namespace noalloc {

constexpr int kScratchKeys = kMaxCells + 1;
// [0, 3*kScratchKeys): count, sum a, sum a^2 per key; then the arrival counter
static __device__ __align__(256) unsigned long long g_scratch[3 * kScratchKeys + 32];

__global__ void __launch_bounds__(kThreads) k_deposit(const int32_t *__restrict__ cell,
                                                      const float *__restrict__ off, long long n,
                                                      int n_cells, int periodic, int s1,
                                                      unsigned long long *scratch, long long *out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ bool s_last;
    unsigned long long *C = scratch, *A = scratch + kScratchKeys, *B = scratch + 2 * kScratchKeys;
    unsigned int *done = (unsigned int *)(scratch + 3 * kScratchKeys);
    Acc acc;
    acc.cnt = (unsigned int *)smem;
    acc.a = acc.cnt + kScratchKeys;
    acc.bh = acc.a + kScratchKeys;
    acc.bl = acc.bh + kScratchKeys;
    const int n1 = n_cells + 1;
    for (int k = threadIdx.x; k < n1; k += kThreads) {
        acc.cnt[k] = 0u;
        acc.a[k] = 0u;
        acc.bh[k] = 0u;
        acc.bl[k] = 0u;
    }
    __syncthreads();
    const long long G = gridDim.x;
    long long ch = (n + G - 1) / G;
    ch = (ch + 31) & ~31ll;
    const long long c0 = (long long)blockIdx.x * ch;
    const long long c1 = c0 + ch < n ? c0 + ch : n;
    for (long long sb = c0; sb < c1; sb += kFlushEvery) {
        const long long se = sb + kFlushEvery < c1 ? sb + kFlushEvery : c1;
        for (long long base = sb; base < se; base += (long long)kThreads * kUnroll) {
            int key[kUnroll];
            uint32_t a[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const long long i = base + (long long)u * kThreads + threadIdx.x;
                key[u] = -1;
                a[u] = 0u;
                if (i < se) {
                    // an entry off the grid (cell outside 0..n_cells-1, or an
                    // offset outside [0, 1), NaN included) assigns nothing
                    const int c = cell[i];
                    const float f = off[i];
                    if (c >= 0 && c < n_cells && f >= 0.0f && f < 1.0f)
                        key[u] = s1 ? deposit_key_s1(c, f, a[u]) : deposit_key_s2(c, f, a[u]);
                }
            }
            deposit_tile(key, a, acc, false);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n1; k += kThreads) {
            if (acc.cnt[k]) {
                atomicAdd(&C[k], (unsigned long long)acc.cnt[k]);
                atomicAdd(&A[k], (unsigned long long)acc.a[k]);
                atomicAdd(&B[k], ((unsigned long long)acc.bh[k] << 16) + acc.bl[k]);
                acc.cnt[k] = 0u;
                acc.a[k] = 0u;
                acc.bh[k] = 0u;
                acc.bl[k] = 0u;
            }
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // node charges from the per-key sums (the same reassembly as the step tail)
    for (int g = threadIdx.x; g <= n_cells; g += kThreads) {
        unsigned long long q = 0;
        if (s1) {
            if (!(periodic && g == n_cells)) {
                if (g < n_cells) q += (C[g] << 16) - A[g];
                const int gl = periodic ? (g - 1 + n_cells) % n_cells : g - 1;
                if (gl >= 0 && gl < n_cells) q += A[gl];
                q <<= 17;
            }
        } else if (!(periodic && g == n_cells)) {
            unsigned long long c[3], aa[3], bb[3];
            for (int d = 0; d < 3; ++d) {
                int k = g - 1 + d;
                c[d] = aa[d] = bb[d] = 0ull;
                if (periodic) {
                    k = ((k % n_cells) + n_cells) % n_cells;
                    c[d] = C[k] + (k == 0 ? C[n_cells] : 0ull);
                    aa[d] = A[k] + (k == 0 ? A[n_cells] : 0ull);
                    bb[d] = B[k] + (k == 0 ? B[n_cells] : 0ull);
                } else if (k >= 0 && k <= n_cells) {
                    c[d] = C[k];
                    aa[d] = A[k];
                    bb[d] = B[k];
                }
            }
            q = (c[1] << 32) + (aa[1] << 17) - 2ull * bb[1] + bb[0] + (c[2] << 32) - (aa[2] << 17) + bb[2];
            if (!periodic) {
                if (g == 0) q += (c[1] << 32) - (aa[1] << 17) + bb[1];
                if (g == n_cells) q += bb[1];
            }
        }
        out[g] = (long long)q;
    }
}

// Device address of the scratch array, looked up once per device.
struct DeviceSlot {
    bool ready;
    unsigned long long *ptr;
};
static DeviceSlot g_slots[64];
static std::mutex g_slots_mutex;

}  // namespace noalloc
}  // namespace pic

extern "C" int pic_deposit_noalloc(int32_t scheme, int32_t boundary, int32_t n_cells,
                                   const int32_t *cell, const float *off, int64_t n,
                                   int64_t *rho_q_out, void *stream) {
    using namespace pic;
    using namespace pic::noalloc;
    if (scheme < 0 || scheme > 3 || (boundary != 0 && boundary != 1)) {  // m = 3 (scheme 4): runs only
        set_last_error("pic_deposit_noalloc: unknown scheme or boundary");
        return -1;
    }
    if (n_cells < 2 || n_cells > kMaxCells) {  // the scratch holds at most kMaxCells + 1 keys
        set_last_error("pic_deposit_noalloc: n_cells outside 2..1024 (size of the static scratch)");
        return -1;
    }
    if (n < 0 || n >= (1ll << 29) || !rho_q_out || (n > 0 && (!cell || !off))) {
        set_last_error("pic_deposit_noalloc: n outside 0..2^29-1 or a NULL array");
        return -1;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_last_error("pic_deposit_noalloc: no current CUDA device");
        return -5;
    }
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_slots_mutex);
        if (!g_slots[dev].ready) {
            // set-up on this device (the current one): the host-side name of a
            // __device__ array is not a device address; ask the runtime for it
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                set_last_error("pic_deposit_noalloc: cudaGetSymbolAddress failed");
                return -5;
            }
            g_slots[dev].ptr = (unsigned long long *)p;
            g_slots[dev].ready = true;
        }
        scratch = g_slots[dev].ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto cuda_fail = [](const char *what, cudaError_t e) {
        std::string m = std::string("pic_deposit_noalloc: ") + what + ": " + cudaGetErrorString(e);
        set_last_error(m.c_str());
        return -5;
    };
    // the array keeps the previous call's sums: clear it on this stream first
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (3 * kScratchKeys + 32), s);
    if (e != cudaSuccess) return cuda_fail("clearing the static scratch", e);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute", e);
    long long grid = (n + 8191) / 8192;
    if (grid < 1) grid = 1;
    if (grid > 4ll * sms) grid = 4ll * sms;
    const int smem = 16 * kScratchKeys;
    k_deposit<<<(int)grid, kThreads, smem, s>>>(cell, off, (long long)n, n_cells, boundary == 1,
                                               scheme == 1 || scheme == 3, scratch, (long long *)rho_q_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("kernel launch", e);
    return 0;
}

// ===========================================================================
// Adjoint of the collisionless EC explicit step (reverse mode).
//
// Electrons on a frozen ion background, no collisions.  The forward kernel is
// the explicit EC step of Sec. 2 (scheme (2)) built from the same device
// functions as k_particles<kExplicitEC> -- gather, push, renormalisation,
// fixed-point S_2 assignment and the Gauss-law field solve -- so a state
// advanced here is bit-identical to the same state advanced by pic_step.  It
// reads time level n from one slot and writes level n+1 to another, keeps
// absorbed particles in place with cell = -1 (the absorption step is the
// event the derivative holds fixed), and sums per step the objectives
//   P^n = sum_p q w E_p vbar_p             (power absorbed by the electrons)
//   G^n = sum_p w vbar_p S_1(xi_p - 1/2)/dx (current density at the centre of
//                                            the first cell)
// with vbar = (v^{n-1/2} + v^{n+1/2}) / 2.
//
// The reverse kernel of level n (one launch per step, last block runs the
// field part) finishes the position adjoint of level n+1 with the adjoint
// field of that level, then takes the adjoint of the push of level n:
//   lv' = lv + dt lx + dJ/dv,   lE = (q/m) dt lv' + dJ/dE_p,
//   lx' = lx + (lE dE_p/dx + dJ/dx),   lv <- lv' + dJ/dv (v^{n-1/2} term),
// scattering lE to the cell centres with the S_1 weights of the gather (the
// transpose of Eq. 3).  The field part transposes the Gauss-law solve: the
// cell-centred field is E_c = d0 + kappa P_c (+ background), P_c the prefix
// of the node charge and d0 fixed by the electrode voltage (or the zero-mean
// field of the periodic box), so with L_c the scattered sensitivities
//   dJ/dq_g = kappa sum_{c >= g} (L_c - mean L),  dJ/dV_left = sum L / (n dx).
// Differences of dJ/dq_g along the grid are again a cell-centred table, so the
// derivative of the S_2 assignment at a particle is an EC gather (Eq. 3) of
//   Lambda_c = (e w / eps0) (L_c - mean L):   lx += gather(Lambda)/dx,
// which is the discrete F = -dU/dx structure of the scheme read backwards.
// ===========================================================================
namespace pic {

// S_1(xi - 1/2) with its periodic image, and its derivative in xi: the EC
// gather (Eq. 3) of a table holding 1 in the first cell.
__device__ __forceinline__ float flux_weight(int n, int periodic, int cell, float off, float &deriv) {
    if (cell == 0) {
        deriv = off >= 0.5f ? -1.0f : 1.0f;
        return off >= 0.5f ? 1.5f - off : 0.5f + off;
    }
    if (cell == 1 && off < 0.5f) {
        deriv = -1.0f;
        return 0.5f - off;
    }
    if (periodic && cell == n - 1 && off >= 0.5f) {
        deriv = 1.0f;
        return off - 0.5f;
    }
    deriv = 0.0f;
    return 0.0f;
}

// A slot entry counts as a particle only with cell in [0, n) and off in [0, 1).
__device__ __forceinline__ int adj_valid_cell(int cell, float off, int n) {
    return (cell >= 0 && cell < n && off >= 0.0f && off < 1.0f) ? cell : -1;
}

template <int U, typename T>
__device__ __forceinline__ void adj_load(const T *p, long long i0, long long np, T (&o)[kUnroll], T fill) {
    if (i0 + U <= np) {
        ldv<U>(p + i0, o);
    } else {
#pragma unroll
        for (int q = 0; q < U; ++q) o[q] = i0 + q < np ? p[i0 + q] : fill;
    }
}

template <int U, typename T>
__device__ __forceinline__ void adj_store(T *p, long long i0, long long np, const T (&o)[kUnroll]) {
    if (i0 + U <= np) {
        stv<U>(p + i0, o);
    } else {
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (i0 + q < np) p[i0 + q] = o[q];
    }
}

template <bool PUSH>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_adj_fwd(Run R, AdjFwd A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ bool s_last;
    __shared__ double s_obj[2][kThreads / 32];
    constexpr int U = kUnroll;
    const int n = R.n_cells;
    const SmemMain sm = carve_main(smem, n, 0, false, nullptr);
    if (PUSH)
        for (int k = threadIdx.x; k < n + 2; k += kThreads) sm.e[k] = A.e_in[k];
    for (int k = threadIdx.x; k <= n; k += kThreads) {
        sm.acc.cnt[k] = 0u;
        sm.acc.a[k] = 0u;
        sm.acc.bh[k] = 0u;
        sm.acc.bl[k] = 0u;
    }
    __syncthreads();
    const long long tile = (long long)kThreads * U;
    double pw_acc = 0.0, fl_acc = 0.0;
    long long added = 0;  // particles this block assigned since its last flush
    for (long long t0 = (long long)blockIdx.x * tile; t0 < A.np; t0 += (long long)gridDim.x * tile) {
        const long long i0 = t0 + (long long)threadIdx.x * U;
        int cell[U];
        float off[U], vx[U];
        adj_load<U>(A.in.cell, i0, A.np, cell, -1);
        adj_load<U>(A.in.off, i0, A.np, off, 0.0f);
        if (PUSH) adj_load<U>(A.in.vx, i0, A.np, vx, 0.0f);
        int key[U];
        uint32_t a[U];
        float pw = 0.0f, fl = 0.0f;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            key[q] = -1;
            a[q] = 0u;
            cell[q] = adj_valid_cell(cell[q], off[q], n);
            if (cell[q] < 0) continue;
            if (PUSH) {
                // the explicit EC step of k_particles<kExplicitEC>, collisionless
                const float e_field = gather_ec(sm.e, cell[q], off[q]);
                const float v_new = fmaf(R.qm_dt[0], e_field, vx[q]);
                const float vb = 0.5f * (vx[q] + v_new);
                float dfl;
                pw += R.qw[0] * e_field * vb;
                fl += flux_weight(n, R.periodic, cell[q], off[q], dfl) * vb;
                float s = fmaf(v_new, R.dt_dx, off[q]);
                if (!(fabsf(s) < 1.0e6f)) s = (float)(2 * n + 2);
                int c = cell[q];
                renormalise(c, s);
                vx[q] = v_new;
                off[q] = s;
                if (R.periodic) {
                    if (c < 0 || c >= n) c = ((c % n) + n) % n;
                } else if (c < 0 || c >= n) {
                    cell[q] = -1;  // absorbed by an electrode (Sec. 3)
                    continue;
                }
                cell[q] = c;
            }
            key[q] = deposit_key_s2(cell[q], off[q], a[q]);
        }
        if (PUSH) {
            adj_store<U>(A.out.cell, i0, A.np, cell);
            adj_store<U>(A.out.off, i0, A.np, off);
            adj_store<U>(A.out.vx, i0, A.np, vx);
        }
        pw_acc += (double)pw;
        fl_acc += (double)fl;
        deposit_tile(key, a, sm.acc, false);
        added += tile;
        if (added + tile > 65536) {  // keep the 32-bit block sums exact
            flush_species(R, sm, 0, false);
            added = 0;
        }
    }
    flush_species(R, sm, 0, false);
    if (PUSH) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const double p = warp_sum(pw_acc), f = warp_sum(fl_acc);
        if (lane == 0) {
            s_obj[0][wid] = p;
            s_obj[1][wid] = f;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            double acc = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) acc += s_obj[threadIdx.x][w];
            if (acc != 0.0) atomicAdd(&A.obj[threadIdx.x], threadIdx.x == 0 ? acc : acc * (double)R.weight * R.inv_dx);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&R.st->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    Run Rt = R;
    Rt.e_gather = A.e_out;
    tail_field<kDepositEC>(Rt, global_keys(R), smem, A.level, false, false, false, Volt{0.0, 0.0f, 0.0f}, false, 0.0,
                           false);
    tail_reset(R);
    __syncthreads();
    if (threadIdx.x == 0) R.st->blocks_done = 0u;
}

// Field part of the reverse step (last block): fold the ghost cells, the
// transposed Gauss-law solve, dJ/dV0, and the table Lambda of this level.
__device__ void tail_adjoint(const Run &R, const AdjRev &A, unsigned char *smem) {
    __shared__ double sc_d[kThreads / 32 + 1];
    const int n = R.n_cells;
    double *L = (double *)smem;  // [n]
    for (int c = threadIdx.x; c < n; c += kThreads) {
        double v = A.le[c + 1];
        if (R.periodic) {
            if (c == 0) v += A.le[n + 1];      // right ghost = cell 0
            if (c == n - 1) v += A.le[0];      // left ghost = cell n-1
        }
        L[c] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n + 2; k += kThreads) A.le[k] = 0.0;
    double s = 0.0;
    for (int c = threadIdx.x; c < n; c += kThreads) s += L[c];
    s = block_sum_lean(s, sc_d);
    const double mean = s / (double)n;
    if (threadIdx.x == 0 && !R.periodic)
        *A.dv0 += sin(2.0 * 3.14159265358979323846 * R.rf_freq * ((double)A.level * R.dt)) * s / ((double)n * R.dx);
    for (int c = threadIdx.x; c < n; c += kThreads) {
        A.lam_out[c + 1] = (float)(A.lam_scale * (L[c] - mean));
        if (c == 0) A.lam_out[n + 1] = R.periodic ? (float)(A.lam_scale * (L[0] - mean)) : 0.0f;
        if (c == n - 1) A.lam_out[0] = R.periodic ? (float)(A.lam_scale * (L[n - 1] - mean)) : 0.0f;
    }
    __syncthreads();
}

// Add a warp's scatter contributions to shared memory: each thread folded its
// particles into the three table entries k0, k0+1, k0+2 (k0 < 0: none; k0 is
// at most n_cells, and entry n_cells+2 is a padding slot that only receives
// zeros).
__device__ __forceinline__ void adj_scatter(float *sle, int k0, float v0, float v1, float v2) {
    const int kw = __shfl_sync(FULL_MASK, k0, 0);
    if (__all_sync(FULL_MASK, k0 == kw) && kw >= 0) {
        v0 = warp_sum(v0);
        v1 = warp_sum(v1);
        v2 = warp_sum(v2);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&sle[kw], v0);
            atomicAdd(&sle[kw + 1], v1);
            atomicAdd(&sle[kw + 2], v2);
        }
        return;
    }
    if (k0 >= 0) {
        if (v0 != 0.0f) atomicAdd(&sle[k0], v0);
        if (v1 != 0.0f) atomicAdd(&sle[k0 + 1], v1);
        if (v2 != 0.0f) atomicAdd(&sle[k0 + 2], v2);
    }
}

__global__ void __launch_bounds__(kThreads, kMinBlocks) k_adj_rev(Run R, AdjRev A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ bool s_last;
    constexpr int U = kUnroll;
    const int n = R.n_cells;
    float *se = (float *)smem;     // [n+2] E of level n
    float *slam = se + (n + 2);    // [n+2] Lambda of level n+1
    float *sle = slam + (n + 2);   // [n+3] scattered sensitivities of this block (last: padding)
    for (int k = threadIdx.x; k < n + 3; k += kThreads) {
        if (k < n + 2) {
            se[k] = A.a_part ? A.e[k] : 0.0f;
            slam[k] = A.lam_in ? A.lam_in[k] : 0.0f;
        }
        sle[k] = 0.0f;
    }
    __syncthreads();
    const float dt = (float)R.dt, inv_dx = (float)R.inv_dx, qm_dt = R.qm_dt[0], qw = R.qw[0];
    const long long tile = (long long)kThreads * U;
    for (long long t0 = (long long)blockIdx.x * tile; t0 < A.np; t0 += (long long)gridDim.x * tile) {
        const long long i0 = t0 + (long long)threadIdx.x * U;
        int hc[U];
        float ho[U], lx[U], lv[U];
        adj_load<U>(A.hi.cell, i0, A.np, hc, -1);
        adj_load<U>(A.hi.off, i0, A.np, ho, 0.0f);
        adj_load<U>(A.lx, i0, A.np, lx, 0.0f);
        adj_load<U>(A.lv, i0, A.np, lv, 0.0f);
        // finish the position adjoint of level n+1: derivative of its charge assignment
#pragma unroll
        for (int q = 0; q < U; ++q) {
            hc[q] = adj_valid_cell(hc[q], ho[q], n);
            if (hc[q] < 0) {
                lx[q] = 0.0f;
            } else if (A.lam_in) {
                lx[q] += gather_ec(slam, hc[q], ho[q]) * inv_dx;
            }
        }
        int k0 = -1;
        float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
        if (A.a_part) {
            int lc[U];
            float lo[U], vm[U], vp[U];
            adj_load<U>(A.lo.cell, i0, A.np, lc, -1);
            adj_load<U>(A.lo.off, i0, A.np, lo, 0.0f);
            adj_load<U>(A.lo.vx, i0, A.np, vm, 0.0f);
            adj_load<U>(A.hi.vx, i0, A.np, vp, 0.0f);
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int c = adj_valid_cell(lc[q], lo[q], n);
                if (c < 0) {
                    lx[q] = 0.0f;
                    lv[q] = 0.0f;
                    continue;
                }
                // gather of level n and its slope in xi (table entries j, j+1)
                const float off = lo[q];
                const int j = c + (off >= 0.5f ? 1 : 0);
                const float w1 = off >= 0.5f ? off - 0.5f : off + 0.5f;
                const float ej = se[j], ej1 = se[j + 1];
                const float e_field = (1.0f - w1) * ej + w1 * ej1;
                const float de = ej1 - ej;
                float dfl;
                const float fl = flux_weight(n, R.periodic, c, off, dfl);
                const float vb = 0.5f * (vm[q] + vp[q]);
                const float dj_dv = 0.5f * (A.c_pw * qw * e_field + A.c_fl * A.w_dx * fl);
                const float dj_de = A.c_pw * qw * vb;
                const float dj_dxi = A.c_fl * A.w_dx * vb * dfl;
                const float lvp = lv[q] + dt * lx[q] + dj_dv;     // x^{n+1} = x^n + dt v^{n+1/2}
                const float le = qm_dt * lvp + dj_de;             // v^{n+1/2} = v^{n-1/2} + qm dt E_p
                lv[q] = lvp + dj_dv;
                lx[q] = lx[q] + (le * de + dj_dxi) * inv_dx;
                // transpose of the gather: le (1 - w1) to entry j, le w1 to entry j+1
                const float a0 = le * (1.0f - w1), a1 = le * w1;
                if (k0 < 0) k0 = j;
                if (j == k0) {
                    v0 += a0;
                    v1 += a1;
                } else if (j == k0 + 1) {
                    v1 += a0;
                    v2 += a1;
                } else {
                    atomicAdd(&sle[j], a0);
                    atomicAdd(&sle[j + 1], a1);
                }
            }
        }
        adj_store<U>(A.lx, i0, A.np, lx);
        if (A.a_part) adj_store<U>(A.lv, i0, A.np, lv);
        if (A.a_part) adj_scatter(sle, k0, v0, v1, v2);
    }
    if (!A.a_part) return;
    __syncthreads();
    for (int k = threadIdx.x; k < n + 2; k += kThreads)
        if (sle[k] != 0.0f) atomicAdd(&A.le[k], (double)sle[k]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&R.st->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    tail_adjoint(R, A, smem);
    if (threadIdx.x == 0) R.st->blocks_done = 0u;
}

int adj_fwd_smem_bytes(int n_cells) {
    const size_t a = main_smem_bytes(n_cells, 0, false);
    const size_t b = tail_smem_bytes(n_cells);
    return (int)(a > b ? a : b);
}

int adj_rev_smem_bytes(int n_cells) {
    const size_t a = 4 * (3 * (size_t)(n_cells + 2) + 1);
    const size_t b = 8 * (size_t)n_cells;
    return (int)(((a > b ? a : b) + 15) & ~size_t(15));
}

cudaError_t adj_prepare(int n_cells, int *grid) {
    int dev = 0, sms = 0, per = 1, per_r = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int sf = adj_fwd_smem_bytes(n_cells), sr = adj_rev_smem_bytes(n_cells);
    if ((e = raise_smem_limit((const void *)k_adj_fwd<true>, sf)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void *)k_adj_fwd<false>, sf)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void *)k_adj_rev, sr)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_fwd<true>, kThreads, sf)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_r, k_adj_rev, kThreads, sr)) != cudaSuccess) return e;
    per = per < per_r ? per : per_r;
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

cudaError_t launch_adj_fwd(const Run &r, const AdjFwd &a, bool push, int grid, cudaStream_t s) {
    const int smem = adj_fwd_smem_bytes(r.n_cells);
    if (push)
        k_adj_fwd<true><<<grid, kThreads, smem, s>>>(r, a);
    else
        k_adj_fwd<false><<<grid, kThreads, smem, s>>>(r, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_rev(const Run &r, const AdjRev &a, int grid, cudaStream_t s) {
    k_adj_rev<<<grid, kThreads, adj_rev_smem_bytes(r.n_cells), s>>>(r, a);
    return cudaGetLastError();
}

}  // namespace pic

// ===========================================================================
// Self-test of the bounded waits (see pic.h): one launch of k_wait_selftest.
// ===========================================================================
namespace pic {
namespace selftest {
struct WaitResult {
    unsigned long long waited_ns;
    unsigned int status;
    unsigned int pad;
};
static __device__ WaitResult g_wait_result;
}  // namespace selftest
}  // namespace pic

extern "C" int pic_selftest_wait(int64_t limit_ns, uint32_t *status, double *waited_s, void *stream) {
    using namespace pic;
    if (limit_ns < 0 || limit_ns > 10ll * 1000000000ll || !status || !waited_s) {
        set_last_error("pic_selftest_wait: limit_ns outside 0..1e10 or a NULL output");
        return -1;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, selftest::g_wait_result) != cudaSuccess || !p) {
        set_last_error("pic_selftest_wait: cudaGetSymbolAddress failed");
        return -5;
    }
    selftest::WaitResult *d = (selftest::WaitResult *)p;
    cudaStream_t s = (cudaStream_t)stream;
    k_wait_selftest<<<1, 32, 0, s>>>((unsigned long long)limit_ns, &d->status, &d->waited_ns);
    selftest::WaitResult h{};
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_last_error("pic_selftest_wait: launch or read-back failed");
        return -5;
    }
    *status = h.status;
    *waited_s = 1e-9 * (double)h.waited_ns;
    return h.status ? -6 : 0;
}
