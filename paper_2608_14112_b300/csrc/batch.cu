// batch.cu -- many volumes of uneven sizes refined together, and the
// autotuner of the evaluator's launch shape.
//
// gve_refine_batch: each volume keeps its own binning (cell-free brick
// pairs, sort, ranges) in its own sub-context and stream; the evaluation and
// the update of all volumes are one persistent cooperative kernel
// (k_batch_iter in field.cu): its CTAs take global brick ids from one work
// counter, find each brick's volume in a table of brick offsets and run the
// fused forward + backward of that volume's brick; after a bounded grid-wide
// barrier the same launch reduces each volume's loss in a fixed order and
// applies the chain rule and Adam to every Gaussian of every volume.  One
// iteration -- bias corrections, the per-volume binning branches, the
// batch-wide capacity check, the persistent kernel, the step counter -- is
// captured once as a CUDA graph and replayed; the Adam step and the trace
// index come from device-side state.  All volumes advance in lockstep: if any
// volume's pair count exceeds its capacity, every volume skips that iteration
// and the host, after growing the scratch, replays from it.  A grid-barrier
// wait that runs out (about a second; it only can when the grid is not
// co-resident) sets a device flag: every later launch of the call does
// nothing and the call returns GVE_E_TIMEOUT.
//
// gve_autotune: times one loss-and-gradient pass (no parameter update) of the
// batch -- binning plus the persistent kernel -- for every brick edge in
// {4, 8, 16} and every Gaussians-per-block in {32, 64}, and returns the
// fastest.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kMaxVol = 32;


struct StatePtrs {
    DevState* p[kMaxVol];
    int n;
};

__global__ void k_batch_reset(BatchState* b, int it0)
{
    b->it = it0;
    b->first = -1;
    b->next = 0;
    b->bar_count = 0;
    b->bar_gen = 0;
    b->err = 0;
}

// bounded waits: about one second of ~128 ns sleeps; the fault-injection
// hook GVE_FAULT=timeout makes the barrier wait for one CTA more than the
// grid holds, with a limit of a few milliseconds, so the wait runs out
constexpr long long kSpinLimit = 8000000;
constexpr long long kSpinLimitTest = 20000;

bool fault(const char* what)
{
    const char* f = getenv("GVE_FAULT");
    return f && strcmp(f, what) == 0;
}

__global__ void k_batch_bc(BatchState* b, int step0, float b1, float b2)
{
    const int step = step0 + b->it + 1;
    b->bc[0] = (float)(1.0 - pow((double)b1, step));
    b->bc[1] = (float)(1.0 - pow((double)b2, step));
}

__global__ void k_batch_overflow(StatePtrs sp, BatchState* b)
{
    int any = 0;
    for (int v = 0; v < sp.n; ++v) any |= sp.p[v]->overflow;
    if (!any) return;
    if (b->first < 0) b->first = b->it;
    for (int v = 0; v < sp.n; ++v) sp.p[v]->overflow = 1;
}

__global__ void k_batch_inc(BatchState* b) { b->it += 1; }

gve_status make_sub(gve_ctx* c, gve_ctx** out)
{
    gve_ctx* s = new gve_ctx();
    s->device = c->device;
    if (cudaMallocHost(&s->hstate, sizeof(DevState)) != cudaSuccess) {
        delete s;
        return fail(c, GVE_E_NOMEM, "pinned host state");
    }
    if (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess) {
        cudaFreeHost(s->hstate);
        delete s;
        return cuda_fail(c, cudaGetLastError(), "event create");
    }
    *out = s;
    return GVE_OK;
}

gve_status ensure_batch(gve_ctx* c, int nvol)
{
    if (!c->gstream) {
        if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "stream create");
        if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "event create");
    }
    while ((int)c->sub.size() < nvol) {
        gve_ctx* s = nullptr;
        gve_status st = make_sub(c, &s);
        if (st != GVE_OK) return st;
        c->sub.push_back(s);
        cudaStream_t vs = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "stream create");
        c->vstream.push_back(vs);
        c->vjoin.push_back(ev);
    }
    gve_status st = ensure(c, c->bstate, sizeof(BatchState), c->gstream);
    if (st != GVE_OK) return st;
    return ensure(c, c->btab, sizeof(BrickArgs) * kMaxVol + sizeof(long long) * (kMaxVol + 1) +
                                  sizeof(double) * kMaxVol * 3, c->gstream);
}

struct Vol {
    Call k;
    const float* field;
    float* prims;
    long long goff;   // first Gaussian of the volume in the concatenated records
    double inv_m;
};

// device tables of one batch: evaluator arguments, brick offsets, 1 / voxels, SSE
struct Tables {
    BrickArgs* vargs;
    long long* boff;
    double* inv_m;
    double* sse;
};

Tables tables(gve_ctx* c)
{
    Tables t;
    char* b = (char*)c->btab.p;
    t.vargs = reinterpret_cast<BrickArgs*>(b);
    t.boff = reinterpret_cast<long long*>(b + sizeof(BrickArgs) * kMaxVol);
    t.inv_m = reinterpret_cast<double*>(b + sizeof(BrickArgs) * kMaxVol + sizeof(long long) * (kMaxVol + 1));
    t.sse = t.inv_m + kMaxVol;
    return t;
}

gve_status check_batch(gve_ctx* c, int nvol, const gve_volume* vols, const float* prims, const gve_eval_opts* o)
{
    if (!c) return GVE_E_INVALID;
    if (nvol < 1 || nvol > kMaxVol || !vols) return fail(c, GVE_E_INVALID, "volume count must be 1..32");
    if (!prims || (reinterpret_cast<uintptr_t>(prims) & 15u)) return fail(c, GVE_E_INVALID, "bad primitive pointer");
    for (int v = 0; v < nvol; ++v) {
        if (!vols[v].field_dev) return fail(c, GVE_E_INVALID, "null field in batch");
        gve_status st = check_common(c, prims, vols[v].n, vols[v].dims, o);
        if (st != GVE_OK) return st;
    }
    return GVE_OK;
}

// Build the per-volume calls (sub-contexts, streams) and size their scratch.
gve_status setup_vols(gve_ctx* c, int nvol, const gve_volume* vols, float* prims, const gve_eval_opts* o,
                      Vol* V, long long* ntot, cudaStream_t caller)
{
    gve_status st = ensure_batch(c, nvol);
    if (st != GVE_OK) return st;
    if (cudaEventRecord(c->fork, caller) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "event");
    long long off = 0;
    for (int v = 0; v < nvol; ++v) {
        if (cudaStreamWaitEvent(c->vstream[v], c->fork, 0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "wait");
        Vol& vo = V[v];
        st = begin(c->sub[v], vo.k, vols[v].n, vols[v].dims, o, c->vstream[v]);
        if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
        vo.field = vols[v].field_dev;
        vo.prims = prims + 12 * off;
        vo.goff = off;
        vo.inv_m = 1.0 / ((double)vols[v].dims.nx * vols[v].dims.ny * vols[v].dims.nz);
        st = size_pairs(vo.k, vo.prims, o);
        if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
        off += vols[v].n;
    }
    *ntot = off;
    return ensure(c, c->acc, sizeof(float) * 12 * (off > 0 ? off : 1), c->gstream);
}

// The persistent kernel's arguments; uploads the volume tables (their
// pointers change only when the scratch grows).
gve_status batch_args(gve_ctx* c, int nvol, Vol* V, const gve_eval_opts* o, const gve_schedule* sc, long long ntot,
                      float* prims, float* m, float* v, float* grad, double* trace, BatchIterArgs* out)
{
    Tables t = tables(c);
    BrickArgs va[kMaxVol];
    long long boff[kMaxVol + 1];
    double inv_m[kMaxVol];
    boff[0] = 0;
    for (int i = 0; i < nvol; ++i) {
        va[i] = brick_args(V[i].k, o);
        va[i].field = V[i].field;
        va[i].mask_thresh = sc ? sc->mask_thresh : -1.f;
        va[i].acc = (float*)c->acc.p + 12 * V[i].goff;
        boff[i + 1] = boff[i] + V[i].k.g.nbricks;
        inv_m[i] = V[i].inv_m;
    }
    cudaStream_t g = c->gstream;
    if (cudaMemcpyAsync(t.vargs, va, sizeof(BrickArgs) * nvol, cudaMemcpyHostToDevice, g) != cudaSuccess ||
        cudaMemcpyAsync(t.boff, boff, sizeof(long long) * (nvol + 1), cudaMemcpyHostToDevice, g) != cudaSuccess ||
        cudaMemcpyAsync(t.inv_m, inv_m, sizeof(double) * nvol, cudaMemcpyHostToDevice, g) != cudaSuccess ||
        cudaStreamSynchronize(g) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "batch tables");
    const int grid = batch_iter_grid(o->brick, o->gaussians_per_block == 32 ? 32 : 64);
    if (grid <= 0) return fail(c, GVE_E_CUDA, "the device cannot launch the persistent kernel cooperatively");
    BatchIterArgs p{};
    p.vargs = t.vargs;
    p.boff = t.boff;
    p.inv_m = t.inv_m;
    p.nvol = nvol;
    p.nbricks = boff[nvol];
    p.ntot = ntot;
    p.bs = (BatchState*)c->bstate.p;
    p.acc = (float*)c->acc.p;
    p.prims = prims;
    p.m = m;
    p.v = v;
    p.grad = grad;
    p.do_adam = sc != nullptr;
    if (sc) {
        p.ad.lr = sc->lr; p.ad.b1 = sc->beta1; p.ad.b2 = sc->beta2; p.ad.eps = sc->eps;
        p.ad.bc_dev = p.bs->bc;
    }
    p.trace = trace;
    p.sse = t.sse;
    const bool inject = fault("timeout");
    p.expect = (unsigned)grid + (inject ? 1u : 0u);
    p.spin_limit = inject ? kSpinLimitTest : kSpinLimit;
    *out = p;
    return GVE_OK;
}

// One iteration of the batch on c->gstream: bias corrections, every
// volume's binning on its own stream, the capacity check, the persistent
// kernel, the step counter.
gve_status issue_iteration(gve_ctx* c, int nvol, Vol* V, const gve_eval_opts* o, const gve_schedule* sc,
                           const BatchIterArgs& p, unsigned grid)
{
    BatchState* bs = (BatchState*)c->bstate.p;
    StatePtrs sp{};
    sp.n = nvol;
    for (int v = 0; v < nvol; ++v) sp.p[v] = dstate(c->sub[v]);
    cudaStream_t g = c->gstream;
    if (sc) k_batch_bc<<<1, 1, 0, g>>>(bs, sc->step0, sc->beta1, sc->beta2);
    cudaEventRecord(c->fork, g);
    for (int v = 0; v < nvol; ++v) {
        cudaStreamWaitEvent(c->vstream[v], c->fork, 0);
        bin_all(V[v].k, V[v].prims, o, 0);
        cudaEventRecord(c->vjoin[v], c->vstream[v]);
        cudaStreamWaitEvent(g, c->vjoin[v], 0);
    }
    k_batch_overflow<<<1, 1, 0, g>>>(sp, bs);
    cudaError_t e = launch_batch_iter(o->brick, o->gaussians_per_block == 32 ? 32 : 64, p, grid, g);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent batch kernel");
    k_batch_inc<<<1, 1, 0, g>>>(bs);
    return GVE_OK;
}

// The iteration as a CUDA graph (nullptr in *exec when the capture is not
// possible: the iteration is then issued directly every time).
gve_status capture_iteration(gve_ctx* c, int nvol, Vol* V, const gve_eval_opts* o, const gve_schedule* sc,
                             const BatchIterArgs& p, unsigned grid, cudaGraphExec_t* exec)
{
    *exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t g = c->gstream;
    if (cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "begin capture");
    gve_status st = issue_iteration(c, nvol, V, o, sc, p, grid);
    cudaError_t e = cudaStreamEndCapture(g, &graph);
    if (st != GVE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        c->err.clear();
        return GVE_OK;   // issued directly instead
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();
    }
    return GVE_OK;
}

gve_status run_iteration(gve_ctx* c, cudaGraphExec_t exec, int nvol, Vol* V, const gve_eval_opts* o,
                         const gve_schedule* sc, const BatchIterArgs& p, unsigned grid)
{
    if (exec) {
        if (cudaGraphLaunch(exec, c->gstream) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "graph launch");
        return GVE_OK;
    }
    return issue_iteration(c, nvol, V, o, sc, p, grid);
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_refine_batch(gve_ctx* c, int32_t nvol, const gve_volume* vols, float* prims,
                                       const gve_schedule* sc, float* adam_state, double* trace, double* psnr_out,
                                       gve_stats* stats, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!sc) return fail(c, GVE_E_INVALID, "null schedule");
    const gve_eval_opts* o = &sc->eval;
    gve_status st = check_batch(c, nvol, vols, prims, o);
    if (st != GVE_OK) return st;
    if (sc->iters < 0 || !(sc->lr >= 0.f) || !(sc->beta1 >= 0.f && sc->beta1 < 1.f) ||
        !(sc->beta2 >= 0.f && sc->beta2 < 1.f) || !(sc->eps >= 0.f) || sc->step0 < 0)
        return fail(c, GVE_E_INVALID, "bad schedule");
    if (adam_state && (reinterpret_cast<uintptr_t>(adam_state) & 15u)) return fail(c, GVE_E_INVALID, "adam alignment");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t caller = (cudaStream_t)stream;
    Vol V[kMaxVol];
    long long ntot = 0;
    st = setup_vols(c, nvol, vols, prims, o, V, &ntot, caller);
    if (st != GVE_OK) return st;
    float* m = adam_state;
    if (!m) {
        st = ensure(c, c->adam, sizeof(float) * 24 * (ntot > 0 ? ntot : 1), c->gstream);
        if (st != GVE_OK) return st;
        m = (float*)c->adam.p;
        if (cudaMemsetAsync(m, 0, sizeof(float) * 24 * (ntot > 0 ? ntot : 1), c->gstream) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "memset adam");
    }
    float* vmom = m + 12 * ntot;
    for (int v = 0; v < nvol; ++v) {
        cudaEventRecord(c->vjoin[v], V[v].k.s);
        cudaStreamWaitEvent(c->gstream, c->vjoin[v], 0);
    }
    if (cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "memset acc");
    double* tr = trace;
    if (!tr) {
        st = ensure(c, c->trace, sizeof(double) * ((size_t)sc->iters * nvol + 1), c->gstream);
        if (st != GVE_OK) return st;
        tr = (double*)c->trace.p;
    }
    BatchState* bs = (BatchState*)c->bstate.p;
    BatchIterArgs p{};
    st = batch_args(c, nvol, V, o, sc, ntot, prims, m, vmom, nullptr, tr, &p);
    if (st != GVE_OK) return st;
    const unsigned grid = p.expect - (fault("timeout") ? 1u : 0u);
    cudaGraphExec_t exec = nullptr;
    st = capture_iteration(c, nvol, V, o, sc, p, grid, &exec);
    if (st != GVE_OK) return st;
    cudaEventRecord(c->ev0, c->gstream);
    k_batch_reset<<<1, 1, 0, c->gstream>>>(bs, 0);
    int it = 0, retries = 0;
    const int seg = 64;
    while (it < sc->iters) {
        const int end = it + seg < sc->iters ? it + seg : sc->iters;
        for (int t = it; t < end; ++t) {
            st = run_iteration(c, exec, nvol, V, o, sc, p, grid);
            if (st != GVE_OK) {
                if (exec) cudaGraphExecDestroy(exec);
                return st;
            }
        }
        BatchState hb{};
        if (cudaMemcpyAsync(&hb, bs, sizeof(hb), cudaMemcpyDeviceToHost, c->gstream) != cudaSuccess ||
            cudaStreamSynchronize(c->gstream) != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            return cuda_fail(c, cudaGetLastError(), "batch state");
        }
        if (hb.err) {
            if (exec) cudaGraphExecDestroy(exec);
            return fail(c, GVE_E_TIMEOUT, "a grid-wide wait of the persistent batch kernel ran out");
        }
        if (hb.first >= 0) {
            if (++retries > 8) {
                if (exec) cudaGraphExecDestroy(exec);
                return fail(c, GVE_E_CAPACITY, "batch capacity retries");
            }
            if (exec) cudaGraphExecDestroy(exec);
            exec = nullptr;
            // every volume grows to half again what it has needed so far, so
            // that volumes close to their capacity do not each force a replay
            for (int v = 0; v < nvol; ++v) {
                DevState h;
                st = read_state(V[v].k, &h);
                const unsigned long long n1 = h.max_total1 > h.total1 ? h.max_total1 : h.total1;
                const unsigned long long n2 = h.max_total > h.total ? h.max_total : h.total;
                if (st == GVE_OK) st = grow_pairs(V[v].k, n1 + n1 / 2, n2 + n2 / 2);
                if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
                reset_state(V[v].k);
                if (cudaStreamSynchronize(V[v].k.s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "sync");
            }
            st = batch_args(c, nvol, V, o, sc, ntot, prims, m, vmom, nullptr, tr, &p);
            if (st != GVE_OK) return st;
            st = capture_iteration(c, nvol, V, o, sc, p, grid, &exec);
            if (st != GVE_OK) return st;
            // the skipped iteration left the sums as the kernel found them
            if (cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream) != cudaSuccess)
                return cuda_fail(c, cudaGetLastError(), "memset acc");
            k_batch_reset<<<1, 1, 0, c->gstream>>>(bs, hb.first);
            it = hb.first;
            continue;
        }
        it = end;
    }
    cudaEventRecord(c->ev1, c->gstream);
    if (exec) cudaGraphExecDestroy(exec);
    // final evaluation of every volume after its last update
    double psnr_min = INFINITY;
    long long pairs = 0;
    for (int v = 0; v < nvol; ++v) {
        cudaStreamWaitEvent(V[v].k.s, c->ev1, 0);
        st = bin_all(V[v].k, V[v].prims, o, sc->iters);
        if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
        BrickArgs a = brick_args(V[v].k, o);
        a.field = V[v].field;
        a.mask_thresh = sc->mask_thresh;
        launch_brick(kModeLoss, a, V[v].k.s);
        launch_sse_reduce(a.part, V[v].k.g.nbricks, dstate(c->sub[v]), nullptr, 0, V[v].inv_m, V[v].k.s);
        DevState h;
        st = read_state(V[v].k, &h);
        if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
        if (h.overflow) return fail(c, GVE_E_CAPACITY, "final evaluation overflowed");
        const double M = 1.0 / V[v].inv_m;
        const double p = h.sse[1] > 0.0 ? 10.0 * std::log10(M / h.sse[1]) : INFINITY;
        if (psnr_out) psnr_out[v] = p;
        psnr_min = p < psnr_min ? p : psnr_min;
        pairs += (long long)h.total;
    }
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        memset(stats, 0, sizeof(*stats));
        stats->psnr_final = psnr_min;
        stats->brick_pairs = pairs;
        stats->iters_done = sc->iters;
        stats->retries = retries;
        stats->ms_total = ms;
        long long per_iter = 4;   // bias corrections, capacity check, persistent kernel, step counter
        for (int v = 0; v < nvol; ++v) per_iter += (V[v].k.n > 0 ? 3 : 0) + 4 + 5 * ((V[v].k.g.key_bits + 7) / 8) + 1;
        stats->launches = per_iter * sc->iters;
        if (sc->iters > 0 && trace) {
            double first = 0, last = 0;
            cudaMemcpy(&first, tr, sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(&last, tr + (size_t)(sc->iters - 1) * nvol, sizeof(double), cudaMemcpyDeviceToHost);
            stats->loss_first = first;
            stats->loss_last = last;
        }
    }
    // the caller's stream continues after the batch
    cudaEventRecord(c->fork, c->gstream);
    for (int v = 0; v < nvol; ++v) {
        cudaEventRecord(c->vjoin[v], V[v].k.s);
        cudaStreamWaitEvent(caller, c->vjoin[v], 0);
    }
    cudaStreamWaitEvent(caller, c->fork, 0);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "batch");
    return GVE_OK;
}

extern "C" gve_status gve_autotune(gve_ctx* c, int32_t nvol, const gve_volume* vols, const float* prims,
                                   gve_eval_opts* opts, float* ms_out, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!opts) return fail(c, GVE_E_INVALID, "null options");
    const int bricks[3] = {4, 8, 16};
    const int chunks[2] = {32, 64};
    gve_eval_opts best = *opts;
    float best_ms = INFINITY;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t caller = (cudaStream_t)stream;
    int idx = 0;
    for (int bi = 0; bi < 3; ++bi)
        for (int ci = 0; ci < 2; ++ci, ++idx) {
            gve_eval_opts o = *opts;
            o.brick = bricks[bi];
            o.gaussians_per_block = chunks[ci];
            gve_status st = check_batch(c, nvol, vols, prims, &o);
            if (st != GVE_OK) return st;
            Vol V[kMaxVol];
            long long ntot = 0;
            st = setup_vols(c, nvol, vols, const_cast<float*>(prims), &o, V, &ntot, caller);
            if (st != GVE_OK) return st;
            st = ensure(c, c->adam, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream);
            if (st != GVE_OK) return st;
            for (int v = 0; v < nvol; ++v) {
                cudaEventRecord(c->vjoin[v], V[v].k.s);
                cudaStreamWaitEvent(c->gstream, c->vjoin[v], 0);
            }
            cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream);
            BatchIterArgs p{};
            // gradient only: the records stay as they are, the gradient goes to scratch
            st = batch_args(c, nvol, V, &o, nullptr, ntot, const_cast<float*>(prims), nullptr, nullptr,
                            (float*)c->adam.p, nullptr, &p);
            if (st != GVE_OK) return st;
            const unsigned grid = p.expect - (fault("timeout") ? 1u : 0u);
            k_batch_reset<<<1, 1, 0, c->gstream>>>((BatchState*)c->bstate.p, 0);
            float total = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(c->ev0, c->gstream);
                st = issue_iteration(c, nvol, V, &o, nullptr, p, grid);
                if (st != GVE_OK) return st;
                cudaEventRecord(c->ev1, c->gstream);
                if (cudaEventSynchronize(c->ev1) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "sync");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, c->ev0, c->ev1);
                if (rep > 0) total += ms;  // first repetition warms up
            }
            BatchState hb{};
            if (cudaMemcpy(&hb, c->bstate.p, sizeof(hb), cudaMemcpyDeviceToHost) != cudaSuccess)
                return cuda_fail(c, cudaGetLastError(), "batch state");
            if (hb.err) return fail(c, GVE_E_TIMEOUT, "a grid-wide wait of the persistent batch kernel ran out");
            if (hb.first >= 0) return fail(c, GVE_E_CAPACITY, "autotune pass overflowed its pair capacity");
            const float per = total / 2.f;
            if (ms_out) ms_out[idx] = per;
            if (per < best_ms) { best_ms = per; best = o; }
        }
    *opts = best;
    for (int v = 0; v < nvol && v < (int)c->vstream.size(); ++v) {
        cudaEventRecord(c->vjoin[v], c->vstream[v]);
        cudaStreamWaitEvent(caller, c->vjoin[v], 0);
    }
    return GVE_OK;
}
