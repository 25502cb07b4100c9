// batch.cu -- many volumes of uneven sizes refined together, and the
// autotuner of the evaluator's launch shape.
//
// gve_refine_batch: the volumes' records are one concatenated set; one
// binning covers all of them (bin.cu with a table of the volumes: each
// Gaussian is binned into the tiles and bricks of its own volume, tiles and
// bricks numbered volume after volume), so every stage runs once over the
// whole batch.  The evaluation and the update of all volumes are one
// persistent cooperative kernel (k_batch_iter in field.cu): its CTAs take
// global brick ids from one work counter, find each brick's volume in the
// table of brick offsets and run the fused forward + backward of that
// volume's brick; after a bounded grid-wide barrier the same launch reduces
// each volume's loss in a fixed order and applies the chain rule and Adam to
// every Gaussian of every volume.  One iteration -- bias corrections, the
// binning, the capacity check, the persistent kernel, the step counter -- is
// captured once as a CUDA graph and replayed; the Adam step and the trace
// index come from device-side state.  If the pairs exceed their capacity the
// iteration is skipped on the device and the host, after growing the
// scratch, replays from it.  A grid-barrier wait that runs out (about a
// second; it only can when the grid is not co-resident) sets a device flag:
// every later launch of the call does nothing and the call returns
// GVE_E_TIMEOUT.
//
// gve_autotune: times one loss-and-gradient pass (no parameter update) of the
// batch -- binning plus the persistent kernel -- for every brick edge in
// {4, 8, 16} and every Gaussians-per-block in {32, 64}, and returns the
// fastest.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kMaxVol = 32;

__global__ void k_batch_reset(BatchState* b, int it0)
{
    b->it = it0;
    b->first = -1;
    b->next = 0;
    b->bar_count = 0;
    b->bar_gen = 0;
    b->err = 0;
    b->done = 0;
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

__global__ void k_batch_overflow(const DevState* st, BatchState* b)
{
    if (st->overflow && b->first < 0) b->first = b->it;
}

__global__ void k_batch_inc(BatchState* b) { b->it += 1; }

gve_status ensure_batch(gve_ctx* c)
{
    if (!c->gstream) {
        if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "stream create");
        if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "event create");
    }
    gve_status st = ensure(c, c->bstate, sizeof(BatchState), c->gstream);
    if (st != GVE_OK) return st;
    return ensure(c, c->btab, sizeof(double) * kMaxVol * 2, c->gstream);
}

struct Vol {
    BinGeom g;
    const float* field;
    long long goff;   // first Gaussian of the volume in the concatenated records
    double inv_m;
};

gve_status check_batch(gve_ctx* c, int nvol, const gve_volume* vols, const float* prims, const gve_eval_opts* o)
{
    if (!c) return GVE_E_INVALID;
    if (nvol < 1 || nvol > kMaxVol || !vols) return fail(c, GVE_E_INVALID, "volume count must be 1..32");
    if (!prims || (reinterpret_cast<uintptr_t>(prims) & 15u)) return fail(c, GVE_E_INVALID, "bad primitive pointer");
    long long total = 0;
    for (int v = 0; v < nvol; ++v) {
        if (!vols[v].field_dev) return fail(c, GVE_E_INVALID, "null field in batch");
        gve_status st = check_common(c, prims, vols[v].n, vols[v].dims, o);
        if (st != GVE_OK) return st;
        total += vols[v].n;
    }
    if (total > (long long)kGidMask + 1) return fail(c, GVE_E_INVALID, "more than 2^24 primitives in the batch");
    return GVE_OK;
}

// One batch: its volumes and the call whose binning covers all of them.
struct Batch {
    int nvol;
    Vol V[kMaxVol];
    Call k;            // the whole batch: n = all Gaussians, vt = the volumes
    long long ntot;
};

// Build the batch's volume table on the context's batch stream and size the
// binning scratch for it.
gve_status setup_vols(gve_ctx* c, int nvol, const gve_volume* vols, float* prims, const gve_eval_opts* o,
                      Batch* b, cudaStream_t caller)
{
    gve_status st = ensure_batch(c);
    if (st != GVE_OK) return st;
    if (cudaEventRecord(c->fork, caller) != cudaSuccess || cudaStreamWaitEvent(c->gstream, c->fork, 0) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "event");
    b->nvol = nvol;
    Call& k = b->k;
    k.c = c;
    k.s = c->gstream;
    VolTab& vt = k.vt;
    vt = VolTab{};
    vt.nvol = nvol;
    long long off = 0;
    for (int v = 0; v < nvol; ++v) {
        Vol& vo = b->V[v];
        vo.g = make_geom(vols[v].dims, o->brick);
        vo.field = vols[v].field_dev;
        vo.goff = off;
        vo.inv_m = 1.0 / ((double)vols[v].dims.nx * vols[v].dims.ny * vols[v].dims.nz);
        vt.g[v] = vo.g;
        vt.goff[v] = off;
        vt.toff[v + 1] = vt.toff[v] + vo.g.ntiles;
        vt.boff[v + 1] = vt.boff[v] + vo.g.nbricks;
        off += vols[v].n;
    }
    vt.goff[nvol] = off;
    if (vt.toff[nvol] > (long long)INT_MAX || vt.boff[nvol] > (long long)INT_MAX)
        return fail(c, GVE_E_INVALID, "the batch has too many bricks");
    b->ntot = off;
    k.n = off;
    k.g = vt.g[0];
    c->launches = 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    st = ensure(c, c->state, sizeof(DevState), k.s);
    if (st != GVE_OK) return st;
    st = size_pairs(k, prims, o);
    if (st != GVE_OK) return st;
    return ensure(c, c->acc, sizeof(float) * 12 * (off > 0 ? off : 1), c->gstream);
}

// evaluator arguments of volume v over the batch's binning: its geometry,
// its bricks' ranges and SSE partials; Gaussian indices are global
BrickArgs vol_args(const Batch& b, int v, const gve_eval_opts* o, float mask_thresh)
{
    Call k = b.k;
    gve_ctx* c = k.c;
    BrickArgs a = brick_args(k, o);
    const long long nb = k.vt.boff[k.vt.nvol], b0 = k.vt.boff[v];
    a.g = b.V[v].g;
    a.start = (const uint32_t*)c->ranges.p + b0;
    a.end = (const uint32_t*)c->ranges.p + nb + b0;
    a.part = (float2*)c->part.p + b0;
    a.inv_m = (float)b.V[v].inv_m;
    a.field = b.V[v].field;
    a.mask_thresh = mask_thresh;
    a.acc = (float*)c->acc.p;
    return a;
}

// The persistent kernel's arguments, the volume tables included (rebuilt
// when the scratch grows).
gve_status batch_args(gve_ctx* c, const Batch& b, const gve_eval_opts* o, const gve_schedule* sc, float* prims,
                      float* m, float* v, float* grad, double* trace, BatchIterArgs* out)
{
    const int nvol = b.nvol;
    static_assert(kMaxVol <= kMaxBatchVol, "volume table size");
    const int grid = batch_iter_grid(o->brick, o->gaussians_per_block == 32 ? 32 : 64);
    if (grid <= 0) return fail(c, GVE_E_CUDA, "the device cannot launch the persistent kernel cooperatively");
    BatchIterArgs p{};
    for (int i = 0; i < nvol; ++i) {
        p.va[i] = vol_args(b, i, o, sc ? sc->mask_thresh : -1.f);
        p.inv_m[i] = b.V[i].inv_m;
    }
    for (int i = 0; i <= nvol; ++i) p.boff[i] = b.k.vt.boff[i];
    p.coff[0] = 0;
    for (int i = 0; i < nvol; ++i) p.coff[i + 1] = p.coff[i] + (b.V[i].g.nbricks + kSseChunk - 1) / kSseChunk;
    p.nchunks = p.coff[nvol];
    gve_status st = ensure(c, c->csum, sizeof(double2) * (p.nchunks > 0 ? p.nchunks : 1), c->gstream);
    if (st != GVE_OK) return st;
    p.csum = (double2*)c->csum.p;
    p.nvol = nvol;
    p.nbricks = p.boff[nvol];
    p.ntot = b.ntot;
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
    p.sse = (double*)c->btab.p;
    const bool inject = fault("timeout");
    p.expect = (unsigned)grid + (inject ? 1u : 0u);
    p.spin_limit = inject ? kSpinLimitTest : kSpinLimit;
    *out = p;
    return GVE_OK;
}

// One iteration of the batch on c->gstream: bias corrections, the binning of
// all volumes, the capacity check, the persistent kernel, the step counter.
gve_status issue_iteration(gve_ctx* c, Batch& b, const gve_eval_opts* o, const gve_schedule* sc, float* prims,
                           const BatchIterArgs& p, unsigned grid)
{
    BatchState* bs = (BatchState*)c->bstate.p;
    cudaStream_t g = c->gstream;
    if (sc) k_batch_bc<<<1, 1, 0, g>>>(bs, sc->step0, sc->beta1, sc->beta2);
    gve_status st = bin_all(b.k, prims, o, 0);
    if (st != GVE_OK) return st;
    k_batch_overflow<<<1, 1, 0, g>>>(dstate(c), bs);
    cudaError_t e = launch_batch_iter(o->brick, o->gaussians_per_block == 32 ? 32 : 64, p, grid, g);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent batch kernel");
    k_batch_inc<<<1, 1, 0, g>>>(bs);
    return GVE_OK;
}

// The iteration as a CUDA graph (nullptr in *exec when the capture is not
// possible: the iteration is then issued directly every time).
gve_status capture_iteration(gve_ctx* c, Batch& b, const gve_eval_opts* o, const gve_schedule* sc, float* prims,
                             const BatchIterArgs& p, unsigned grid, cudaGraphExec_t* exec)
{
    *exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t g = c->gstream;
    if (cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "begin capture");
    gve_status st = issue_iteration(c, b, o, sc, prims, p, grid);
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

gve_status run_iteration(gve_ctx* c, cudaGraphExec_t exec, Batch& b, const gve_eval_opts* o, const gve_schedule* sc,
                         float* prims, const BatchIterArgs& p, unsigned grid)
{
    if (exec) {
        if (cudaGraphLaunch(exec, c->gstream) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "graph launch");
        return GVE_OK;
    }
    return issue_iteration(c, b, o, sc, prims, p, grid);
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
    Batch b;
    st = setup_vols(c, nvol, vols, prims, o, &b, caller);
    if (st != GVE_OK) return st;
    const long long ntot = b.ntot;
    float* m = adam_state;
    if (!m) {
        st = ensure(c, c->adam, sizeof(float) * 24 * (ntot > 0 ? ntot : 1), c->gstream);
        if (st != GVE_OK) return st;
        m = (float*)c->adam.p;
        if (cudaMemsetAsync(m, 0, sizeof(float) * 24 * (ntot > 0 ? ntot : 1), c->gstream) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "memset adam");
    }
    float* vmom = m + 12 * ntot;
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
    st = batch_args(c, b, o, sc, prims, m, vmom, nullptr, tr, &p);
    if (st != GVE_OK) return st;
    const unsigned grid = p.expect - (fault("timeout") ? 1u : 0u);
    cudaGraphExec_t exec = nullptr;
    const long long l0 = c->launches;
    st = capture_iteration(c, b, o, sc, prims, p, grid, &exec);
    if (st != GVE_OK) return st;
    const long long per_iter = c->launches - l0 + 4;   // + bias corrections, check, persistent kernel, counter
    cudaEventRecord(c->ev0, c->gstream);
    k_batch_reset<<<1, 1, 0, c->gstream>>>(bs, 0);
    int it = 0, retries = 0;
    const int seg = 64;
    while (it < sc->iters) {
        const int end = it + seg < sc->iters ? it + seg : sc->iters;
        for (int t = it; t < end; ++t) {
            st = run_iteration(c, exec, b, o, sc, prims, p, grid);
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
            // grow to half again what the batch has needed so far, so that a
            // slowly growing pair count does not force a replay each time
            DevState h;
            st = read_state(b.k, &h);
            if (st != GVE_OK) return st;
            const unsigned long long n1 = h.max_total1 > h.total1 ? h.max_total1 : h.total1;
            const unsigned long long n2 = h.max_total > h.total ? h.max_total : h.total;
            st = grow_pairs(b.k, n1 + n1 / 2, n2 + n2 / 2);
            if (st != GVE_OK) return st;
            reset_state(b.k);
            st = batch_args(c, b, o, sc, prims, m, vmom, nullptr, tr, &p);
            if (st != GVE_OK) return st;
            st = capture_iteration(c, b, o, sc, prims, p, grid, &exec);
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
    // final evaluation of every volume after its last update: one binning,
    // then each volume's loss
    double psnr_min = INFINITY;
    long long pairs = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        reset_state(b.k);
        st = bin_all(b.k, prims, o, sc->iters);
        if (st != GVE_OK) return st;
        DevState h;
        st = read_state(b.k, &h);
        if (st != GVE_OK) return st;
        if (!h.overflow) {
            pairs = (long long)h.total;
            break;
        }
        if (attempt == 1) return fail(c, GVE_E_CAPACITY, "final evaluation overflowed");
        st = grow_pairs(b.k, h.total1, h.total);
        if (st != GVE_OK) return st;
    }
    for (int v = 0; v < nvol; ++v) {
        BrickArgs a = vol_args(b, v, o, sc->mask_thresh);
        launch_brick(kModeLoss, a, c->gstream);
        launch_sse_reduce(a.part, b.V[v].g.nbricks, dstate(c), nullptr, 0, b.V[v].inv_m, c->gstream);
        DevState h;
        st = read_state(b.k, &h);
        if (st != GVE_OK) return st;
        const double M = 1.0 / b.V[v].inv_m;
        const double q = h.sse[1] > 0.0 ? 10.0 * std::log10(M / h.sse[1]) : INFINITY;
        if (psnr_out) psnr_out[v] = q;
        psnr_min = q < psnr_min ? q : psnr_min;
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
    cudaStreamWaitEvent(caller, c->fork, 0);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "batch");
    return GVE_OK;
}

// Concurrent allocation of a batch's volumes: up to kAllocWorkers host
// threads, each with its own context (scratch) and stream, take volumes
// largest first from a shared counter; volume v's records go to rows
// [off_v, off_v + n_v) of prims.  Each volume's result is exactly that of
// gve_allocate on it alone.
constexpr int kAllocWorkers = 8;

extern "C" gve_status gve_allocate_batch(gve_ctx* c, int32_t nvol, const gve_volume* vols,
                                         const gve_alloc_opts* o, float* prims, gve_alloc_info* infos,
                                         void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (nvol < 1 || nvol > kMaxVol || !vols || !o) return fail(c, GVE_E_INVALID, "volume count must be 1..32");
    if (!prims || (reinterpret_cast<uintptr_t>(prims) & 15u)) return fail(c, GVE_E_INVALID, "bad primitive pointer");
    long long off[kMaxVol + 1];
    off[0] = 0;
    for (int v = 0; v < nvol; ++v) {
        if (!vols[v].field_dev || vols[v].n < 0) return fail(c, GVE_E_INVALID, "bad volume in batch");
        off[v + 1] = off[v] + vols[v].n;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    const int nw = std::min(nvol, kAllocWorkers);
    while ((int)c->asub.size() < nw) {
        gve_ctx* w = nullptr;
        gve_status st = gve_ctx_create(&w, c->device);
        if (st != GVE_OK) return fail(c, st, "allocation worker context");
        cudaStream_t as = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&as, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            gve_ctx_destroy(w);
            return cuda_fail(c, cudaGetLastError(), "allocation worker stream");
        }
        c->asub.push_back(w);
        c->astream.push_back(as);
        c->ajoin.push_back(ev);
    }
    gve_status st = ensure_batch(c);
    if (st != GVE_OK) return st;
    cudaStream_t caller = (cudaStream_t)stream;
    if (cudaEventRecord(c->fork, caller) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "event");
    for (int w = 0; w < nw; ++w)
        if (cudaStreamWaitEvent(c->astream[w], c->fork, 0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "wait");
    // largest volumes first
    int order[kMaxVol];
    for (int v = 0; v < nvol; ++v) order[v] = v;
    auto voxels = [&](int v) { return (long long)vols[v].dims.nx * vols[v].dims.ny * vols[v].dims.nz; };
    std::stable_sort(order, order + nvol, [&](int a, int b) { return voxels(a) > voxels(b); });
    std::vector<gve_status> status(nvol, GVE_OK);
    std::vector<std::string> msg(nvol);
    std::atomic<int> next{0};
    auto work = [&](int w) {
        cudaSetDevice(c->device);
        for (int k = next.fetch_add(1); k < nvol; k = next.fetch_add(1)) {
            const int v = order[k];
            gve_alloc_info info{};
            const gve_status s = gve_allocate(c->asub[w], vols[v].field_dev, vols[v].dims, vols[v].n, o,
                                              prims + 12 * off[v], nullptr, &info, c->astream[w]);
            status[v] = s;
            if (s != GVE_OK) msg[v] = c->asub[w]->err;
            if (infos) infos[v] = info;
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(work, w);
    work(0);
    for (std::thread& t : pool) t.join();
    for (int w = 0; w < nw; ++w) {
        cudaEventRecord(c->ajoin[w], c->astream[w]);
        cudaStreamWaitEvent(caller, c->ajoin[w], 0);
    }
    for (int v = 0; v < nvol; ++v)
        if (status[v] != GVE_OK) {
            char buf[64];
            snprintf(buf, sizeof(buf), "volume %d: ", v);
            c->err = std::string(buf) + msg[v];
            return status[v];
        }
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "allocate batch");
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
    float* P = const_cast<float*>(prims);
    int idx = 0;
    for (int bi = 0; bi < 3; ++bi)
        for (int ci = 0; ci < 2; ++ci, ++idx) {
            gve_eval_opts o = *opts;
            o.brick = bricks[bi];
            o.gaussians_per_block = chunks[ci];
            gve_status st = check_batch(c, nvol, vols, prims, &o);
            if (st != GVE_OK) return st;
            Batch b;
            st = setup_vols(c, nvol, vols, P, &o, &b, caller);
            if (st != GVE_OK) return st;
            const long long ntot = b.ntot;
            st = ensure(c, c->adam, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream);
            if (st != GVE_OK) return st;
            cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (ntot > 0 ? ntot : 1), c->gstream);
            BatchIterArgs p{};
            // gradient only: the records stay as they are, the gradient goes to scratch
            st = batch_args(c, b, &o, nullptr, P, nullptr, nullptr, (float*)c->adam.p, nullptr, &p);
            if (st != GVE_OK) return st;
            const unsigned grid = p.expect - (fault("timeout") ? 1u : 0u);
            k_batch_reset<<<1, 1, 0, c->gstream>>>((BatchState*)c->bstate.p, 0);
            float total = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(c->ev0, c->gstream);
                st = issue_iteration(c, b, &o, nullptr, P, p, grid);
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
    cudaEventRecord(c->fork, c->gstream);
    cudaStreamWaitEvent(caller, c->fork, 0);
    return GVE_OK;
}
