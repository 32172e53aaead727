// pic_batch.cu -- many independent discharges in one caller-owned arena,
// advanced together by persistent launches over all runs (k_batch in
// pic_kernels.cu), whole sort cycles replayed from a captured CUDA graph, and
// an autotuner for the work-item size and the sort period.  Implements the
// pic_batch_* part of include/pic.h.
#include "pic.h"
#include "pic_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pic;

struct pic_batch {
    int nruns;
    std::vector<pic_config> cfgs;
    std::vector<Layout> layouts;
    std::vector<size_t> offsets;
    std::vector<Run> runs;
    unsigned char *arena;
    size_t arena_bytes;
    Run *runs_d;
    long long *work_d;
    BatchState *bs_d;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    cudaGraphExec_t graph;
    int graph_len;
    int grid, smem, table_off;
    long long chunk;
    int sort_period;
    long long host_step;
    bool any_implicit;
    std::string err;
};

namespace {

constexpr int kMaxRuns = 1024;

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchLayout {
    size_t bs, work, runs, total;
    std::vector<size_t> run_off;
    std::vector<Layout> L;
};

int fail_b(pic_batch *b, int code, const char *msg) {
    set_last_error(msg);
    if (b) b->err = msg;
    return code;
}

int cuda_fail_b(pic_batch *b, cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return fail_b(b, PIC_ECUDA, buf);
}

#define CKB(b, call)                                               \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail_b((b), e_, #call); \
    } while (0)

int batch_layout(const pic_config *cfgs, int nruns, BatchLayout *out) {
    if (!cfgs || nruns < 1 || nruns > kMaxRuns) return fail_b(nullptr, PIC_EINVAL, "nruns outside 1..1024");
    size_t o = 0;
    out->bs = o;
    o = a256(o + sizeof(BatchState));
    out->work = o;
    o = a256(o + 16 * (size_t)nruns);
    out->runs = o;
    o = a256(o + sizeof(Run) * (size_t)nruns);
    out->run_off.resize(nruns);
    out->L.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        int code = validate_run_config(&cfgs[r]);
        if (code) return code;
        if (cfgs[r].scheme == PIC_EC3_EXPLICIT || cfgs[r].cell_width) {
            char msg[96];
            snprintf(msg, sizeof msg, "run %d: the m = 3 scheme and non-uniform grids run through pic_init only", r);
            return fail_b(nullptr, PIC_EINVAL, msg);
        }
        out->L[r] = make_run_layout(cfgs[r]);
        out->run_off[r] = o;
        o = a256(o + out->L[r].total);
    }
    out->total = o;
    return PIC_OK;
}

int enqueue_batch_step(pic_batch *b, long long step_index, cudaStream_t s) {
    CKB(b, launch_batch(0, b->runs_d, b->nruns, b->work_d, b->bs_d, b->chunk, b->grid, b->smem, b->table_off, s));
    if (b->any_implicit)
        CKB(b, launch_batch(1, b->runs_d, b->nruns, b->work_d, b->bs_d, b->chunk, b->grid, b->smem,
                            b->table_off, s));
    if (b->sort_period > 0 && (step_index + 1) % b->sort_period == 0)
        CKB(b, launch_batch(2, b->runs_d, b->nruns, b->work_d, b->bs_d, b->chunk, b->grid, b->smem,
                            b->table_off, s));
    return PIC_OK;
}

void drop_graph(pic_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_len = 0;
}

int capture_cycle(pic_batch *b) {
    const int len = b->sort_period > 0 ? b->sort_period : 16;
    if (!b->capture_stream) CKB(b, cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CKB(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    int r = PIC_OK;
    for (int k = 0; k < len && r == PIC_OK; ++k) r = enqueue_batch_step(b, k, b->capture_stream);
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
    if (r) return r;
    if (e != cudaSuccess) return cuda_fail_b(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail_b(b, e, "cudaGraphInstantiate");
    b->graph_len = len;
    return PIC_OK;
}

int step_batch(pic_batch *b, long long n) {
    const int K = b->sort_period > 0 ? b->sort_period : 16;
    while (n > 0) {
        if (b->host_step % K == 0 && n >= K) {
            if (!b->graph) {
                int r = capture_cycle(b);
                if (r) return r;
            }
            CKB(b, cudaGraphLaunch(b->graph, b->stream));
            b->host_step += K;
            n -= K;
        } else {
            int r = enqueue_batch_step(b, b->host_step, b->stream);
            if (r) return r;
            b->host_step += 1;
            n -= 1;
        }
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_required_sizes(const pic_config *cfgs, int32_t nruns, pic_sizes *out) {
    if (!out) return fail_b(nullptr, PIC_EINVAL, "out is NULL");
    BatchLayout BL;
    int r = batch_layout(cfgs, nruns, &BL);
    if (r) return r;
    out->arena_bytes = BL.total;
    out->snapshot_bytes = 0;
    return PIC_OK;
}

int pic_batch_init(const pic_config *cfgs, int32_t nruns, const pic_buffers *bufs, void *stream,
                   pic_batch **out) {
    if (!bufs || !out) return fail_b(nullptr, PIC_EINVAL, "bufs/out is NULL");
    BatchLayout BL;
    int r = batch_layout(cfgs, nruns, &BL);
    if (r) return r;
    if (!bufs->arena || bufs->arena_bytes < BL.total) {
        char m[200];
        snprintf(m, sizeof m, "arena of %zu bytes, %zu needed", bufs->arena_bytes, BL.total);
        return fail_b(nullptr, PIC_ENOMEM, m);
    }
    if (((uintptr_t)bufs->arena & 255u) != 0) return fail_b(nullptr, PIC_ENOMEM, "arena not 256-byte aligned");
    pic_batch *b = new pic_batch();
    b->nruns = nruns;
    b->cfgs.assign(cfgs, cfgs + nruns);
    b->layouts = BL.L;
    b->offsets = BL.run_off;
    b->runs.resize(nruns);
    b->arena = (unsigned char *)bufs->arena;
    b->arena_bytes = BL.total;
    b->bs_d = (BatchState *)(b->arena + BL.bs);
    b->work_d = (long long *)(b->arena + BL.work);
    b->runs_d = (Run *)(b->arena + BL.runs);
    b->stream = (cudaStream_t)stream;
    b->capture_stream = nullptr;
    b->graph = nullptr;
    b->graph_len = 0;
    b->host_step = 0;
    b->chunk = 16384;
    b->any_implicit = false;
    int sort_period = 0, max_cells = 2, max_bins = 1, big = 0;
    for (int k = 0; k < nruns; ++k) {
        derive_run(cfgs[k], BL.L[k], b->arena + BL.run_off[k], b->runs[k]);
        b->any_implicit |= implicit_scheme(cfgs[k]);
        if (cfgs[k].sort_period > 0 && (sort_period == 0 || cfgs[k].sort_period < sort_period))
            sort_period = cfgs[k].sort_period;
        if (cfgs[k].n_cells > max_cells) {
            max_cells = cfgs[k].n_cells;
            big = k;
        }
        max_bins = std::max(max_bins, (int)cfgs[k].eedf_bins);
    }
    b->sort_period = sort_period > 0 ? sort_period : 16;
    auto bail = [&](int code) {
        delete b;
        return code;
    };
    // per-run kernels for the initial load: the run with the widest grid sets
    // the shared-memory limit and the grid (with the implicit runs' wider ring
    // if there are any)
    Run widest = b->runs[big];
    widest.eedf_bins = max_bins;
    if (b->any_implicit) widest.scheme = PIC_EC_IMPLICIT;
    int grid = 0;
    cudaError_t e = occupancy_grid(widest, kExplicitEC, &grid);
    if (e != cudaSuccess) return bail(cuda_fail_b(nullptr, e, "occupancy"));
    e = cudaMemsetAsync(b->arena, 0, BL.total, b->stream);
    if (e != cudaSuccess) return bail(cuda_fail_b(nullptr, e, "cudaMemsetAsync(arena)"));
    for (int k = 0; k < nruns; ++k) {
        r = init_run_state(cfgs[k], b->runs[k], b->arena + BL.run_off[k], BL.L[k].total, grid, b->stream, &b->err);
        if (r) return bail(r);
    }
    std::vector<long long> work(2 * (size_t)nruns);
    for (int k = 0; k < nruns; ++k) {
        work[2 * k] = cfgs[k].np_init;
        work[2 * k + 1] = cfgs[k].ions_mobile ? cfgs[k].np_init : 0;
    }
    e = cudaMemcpyAsync(b->runs_d, b->runs.data(), sizeof(Run) * nruns, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->work_d, work.data(), 8 * work.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(cuda_fail_b(nullptr, e, "batch upload"));
    b->smem = (int)batch_smem_bytes(max_cells, max_bins, nruns, &b->table_off);
    e = batch_prepare(b->smem, &b->grid);
    if (e != cudaSuccess) return bail(cuda_fail_b(nullptr, e, "batch_prepare"));
    *out = b;
    return PIC_OK;
}

int pic_batch_step(pic_batch *b, int64_t n) {
    if (!b || n < 0) return fail_b(b, PIC_EINVAL, "bad argument");
    return step_batch(b, n);
}

int pic_batch_diag(pic_batch *b, int32_t run, pic_diag_t *out, int reset_avg) {
    if (!b || !out || run < 0 || run >= b->nruns) return fail_b(b, PIC_EINVAL, "bad argument");
    return run_diag(b->runs[run], b->cfgs[run], b->layouts[run], b->arena + b->offsets[run], b->stream, out,
                    reset_avg, &b->err);
}

int pic_batch_get_particles(pic_batch *b, int32_t run, int species, pic_host_particles *out) {
    if (!b || !out || run < 0 || run >= b->nruns || species < 0 || species > 1)
        return fail_b(b, PIC_EINVAL, "bad argument");
    return run_get_particles(b->runs[run], b->stream, species, out, &b->err);
}

int pic_batch_profiles(pic_batch *b, int32_t run, double *ne, double *ni, double *phi, double *heat_e,
                       double *heat_i, uint64_t *eedf) {
    if (!b || run < 0 || run >= b->nruns) return fail_b(b, PIC_EINVAL, "bad argument");
    return run_profiles(b->runs[run], b->cfgs[run], b->stream, ne, ni, phi, heat_e, heat_i, eedf, &b->err);
}

int pic_batch_set_schedule(pic_batch *b, int64_t chunk, int32_t sort_period) {
    if (!b || chunk < 256 || chunk > (1ll << 24) || sort_period < 0)
        return fail_b(b, PIC_EINVAL, "chunk outside 256..2^24 or negative sort period");
    CKB(b, cudaStreamSynchronize(b->stream));
    b->chunk = (chunk + 31) & ~31ll;
    b->sort_period = sort_period;
    drop_graph(b);
    return PIC_OK;
}

int pic_batch_autotune(pic_batch *b, int32_t trial_steps, int64_t *chunk, int32_t *sort_period,
                       double *ms_per_step) {
    if (!b || trial_steps < 1) return fail_b(b, PIC_EINVAL, "bad argument");
    // Every candidate schedule gives bit-identical particles (charge sums are
    // integers and draws are keyed on (id, step)), so the trial steps are
    // ordinary steps of the runs.
    const long long chunks[] = {4096, 8192, 16384, 32768, 65536};
    const int periods[] = {4, 8, 16, 32};
    cudaEvent_t e0, e1;
    CKB(b, cudaEventCreate(&e0));
    CKB(b, cudaEventCreate(&e1));
    double best = 1e300;
    long long best_chunk = b->chunk;
    int best_period = b->sort_period;
    for (long long ch : chunks) {
        for (int sp : periods) {
            int r = pic_batch_set_schedule(b, ch, sp);
            if (r) return r;
            // align to a sort cycle, then time whole cycles
            long long align = (sp - b->host_step % sp) % sp;
            if (align) {
                r = step_batch(b, align);
                if (r) return r;
            }
            const long long steps = ((trial_steps + sp - 1) / sp) * sp;
            CKB(b, cudaEventRecord(e0, b->stream));
            r = step_batch(b, steps);
            if (r) return r;
            CKB(b, cudaEventRecord(e1, b->stream));
            CKB(b, cudaEventSynchronize(e1));
            float ms = 0.0f;
            CKB(b, cudaEventElapsedTime(&ms, e0, e1));
            const double per = ms / (double)steps;
            if (per < best) {
                best = per;
                best_chunk = ch;
                best_period = sp;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int r = pic_batch_set_schedule(b, best_chunk, best_period);
    if (r) return r;
    if (chunk) *chunk = best_chunk;
    if (sort_period) *sort_period = best_period;
    if (ms_per_step) *ms_per_step = best;
    return PIC_OK;
}

int pic_batch_status(pic_batch *b, uint32_t *status) {
    if (!b || !status) return fail_b(b, PIC_EINVAL, "NULL argument");
    CKB(b, cudaStreamSynchronize(b->stream));
    uint32_t s = 0;
    for (int k = 0; k < b->nruns; ++k) {
        DevState st;
        CKB(b, cudaMemcpy(&st, b->runs[k].st, sizeof st, cudaMemcpyDeviceToHost));
        s |= st.status;
    }
    *status = s;
    return PIC_OK;
}

void pic_batch_free(pic_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    delete b;
}

}  // extern "C"
