// batch.cu -- many volumes of uneven sizes refined together, and the
// autotuner of the evaluator's launch shape.
//
// gve_refine_batch: each volume keeps its own pipeline (binning, brick
// evaluator, SSE, chain rule + Adam) on its own stream and scratch; one
// refinement iteration of all volumes is captured once as a CUDA graph (fork
// into one branch per volume for the binning, a batch-wide capacity check,
// fork again for evaluation and update, join) and the graph is replayed for
// every iteration: one launch per iteration for the whole batch, with small
// and large volumes sharing the GPU.  The Adam step and the trace index come
// from a device-side counter, so the replayed graph needs no per-iteration
// arguments.  All volumes advance in lockstep: if any volume's pair count
// exceeds its capacity, every volume skips that iteration and the host,
// after growing the scratch, replays from it.
//
// gve_autotune: times one loss-and-gradient pass (no parameter update) of the
// batch for every brick edge in {4, 8, 16} and every Gaussians-per-block in
// {32, 64}, and returns the fastest.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kMaxVol = 32;

struct BatchState {
    int it;        // iteration index within the call
    int first;     // first iteration that overflowed, -1 if none
    float bc[2];   // Adam bias corrections of the current step
};

struct StatePtrs {
    DevState* p[kMaxVol];
    int n;
};

__global__ void k_batch_reset(BatchState* b, int it0)
{
    b->it = it0;
    b->first = -1;
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
    return ensure(c, c->bstate, sizeof(BatchState), c->gstream);
}

struct Vol {
    Call k;
    const float* field;
    float* prims;
    float* m;
    float* v;
    double inv_m;
};

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
        vo.inv_m = 1.0 / ((double)vols[v].dims.nx * vols[v].dims.ny * vols[v].dims.nz);
        st = size_pairs(vo.k, vo.prims, o);
        if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
        off += vols[v].n;
    }
    *ntot = off;
    return GVE_OK;
}

void launch_eval_update(Vol& vo, const gve_eval_opts* o, const gve_schedule* sc, double* trace, int nvol, int col,
                        BatchState* bs, bool update)
{
    gve_ctx* sc_ctx = vo.k.c;
    BrickArgs a = brick_args(vo.k, o);
    a.field = vo.field;
    a.mask_thresh = sc ? sc->mask_thresh : -1.f;
    a.acc = (float*)sc_ctx->acc.p;
    launch_brick(kModeLoss, a, vo.k.s);
    launch_sse_reduce(a.part, vo.k.g.nbricks, dstate(sc_ctx), trace, 0, vo.inv_m, vo.k.s, bs ? &bs->it : nullptr,
                      nvol, col);
    if (update) {
        AdamArgs ad{};
        ad.lr = sc->lr; ad.b1 = sc->beta1; ad.b2 = sc->beta2; ad.eps = sc->eps;
        ad.bc_dev = bs->bc;
        launch_chain((float*)sc_ctx->acc.p, (float*)sc_ctx->acc.p, vo.prims, vo.k.n, nullptr, vo.m, vo.v, &ad,
                     dstate(sc_ctx), vo.k.s);
    } else {
        // gradient without update: written into the first moment slot as scratch
        launch_chain((float*)sc_ctx->acc.p, (float*)sc_ctx->acc.p, vo.prims, vo.k.n, vo.m, nullptr, nullptr, nullptr,
                     dstate(sc_ctx), vo.k.s);
    }
}

gve_status capture_iteration(gve_ctx* c, int nvol, Vol* V, const gve_eval_opts* o, const gve_schedule* sc,
                             double* trace, cudaGraphExec_t* exec)
{
    BatchState* bs = (BatchState*)c->bstate.p;
    StatePtrs sp{};
    sp.n = nvol;
    for (int v = 0; v < nvol; ++v) sp.p[v] = dstate(c->sub[v]);
    cudaGraph_t graph = nullptr;
    cudaStream_t g = c->gstream;
    if (cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "begin capture");
    k_batch_bc<<<1, 1, 0, g>>>(bs, sc->step0, sc->beta1, sc->beta2);
    cudaEventRecord(c->fork, g);
    for (int v = 0; v < nvol; ++v) {
        cudaStreamWaitEvent(c->vstream[v], c->fork, 0);
        bin_all(V[v].k, V[v].prims, o, 0);
        cudaEventRecord(c->vjoin[v], c->vstream[v]);
        cudaStreamWaitEvent(g, c->vjoin[v], 0);
    }
    k_batch_overflow<<<1, 1, 0, g>>>(sp, bs);
    cudaEventRecord(c->fork, g);
    for (int v = 0; v < nvol; ++v) {
        cudaStreamWaitEvent(c->vstream[v], c->fork, 0);
        launch_eval_update(V[v], o, sc, trace, nvol, v, bs, true);
        cudaEventRecord(c->vjoin[v], c->vstream[v]);
        cudaStreamWaitEvent(g, c->vjoin[v], 0);
    }
    k_batch_inc<<<1, 1, 0, g>>>(bs);
    cudaError_t e = cudaStreamEndCapture(g, &graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    return GVE_OK;
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
    {
        long long off = 0;
        for (int v = 0; v < nvol; ++v) {
            V[v].m = m + 12 * off;
            V[v].v = m + 12 * ntot + 12 * off;
            off += V[v].k.n;
            gve_ctx* s = c->sub[v];
            if (cudaMemsetAsync(s->acc.p, 0, sizeof(float) * 12 * (V[v].k.n > 0 ? V[v].k.n : 1), V[v].k.s) !=
                cudaSuccess)
                return cuda_fail(c, cudaGetLastError(), "memset acc");
            cudaEventRecord(c->vjoin[v], V[v].k.s);
            cudaStreamWaitEvent(c->gstream, c->vjoin[v], 0);
        }
    }
    double* tr = trace;
    if (!tr) {
        st = ensure(c, c->trace, sizeof(double) * ((size_t)sc->iters * nvol + 1), c->gstream);
        if (st != GVE_OK) return st;
        tr = (double*)c->trace.p;
    }
    BatchState* bs = (BatchState*)c->bstate.p;
    cudaGraphExec_t exec = nullptr;
    st = capture_iteration(c, nvol, V, o, sc, tr, &exec);
    if (st != GVE_OK) return st;
    cudaEventRecord(c->ev0, c->gstream);
    k_batch_reset<<<1, 1, 0, c->gstream>>>(bs, 0);
    int it = 0, retries = 0;
    const int seg = 64;
    while (it < sc->iters) {
        const int end = it + seg < sc->iters ? it + seg : sc->iters;
        for (int t = it; t < end; ++t) {
            if (cudaGraphLaunch(exec, c->gstream) != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return cuda_fail(c, cudaGetLastError(), "graph launch");
            }
        }
        BatchState hb{};
        if (cudaMemcpyAsync(&hb, bs, sizeof(hb), cudaMemcpyDeviceToHost, c->gstream) != cudaSuccess ||
            cudaStreamSynchronize(c->gstream) != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_fail(c, cudaGetLastError(), "batch state");
        }
        if (hb.first >= 0) {
            if (++retries > 8) { cudaGraphExecDestroy(exec); return fail(c, GVE_E_CAPACITY, "batch capacity retries"); }
            cudaGraphExecDestroy(exec);
            exec = nullptr;
            for (int v = 0; v < nvol; ++v) {
                DevState h;
                st = read_state(V[v].k, &h);
                if (st == GVE_OK) st = grow_pairs(V[v].k, h.max_total > h.total ? h.max_total : h.total);
                if (st != GVE_OK) { c->err = c->sub[v]->err; return st; }
                reset_state(V[v].k);
                if (cudaStreamSynchronize(V[v].k.s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "sync");
            }
            st = capture_iteration(c, nvol, V, o, sc, tr, &exec);
            if (st != GVE_OK) return st;
            k_batch_reset<<<1, 1, 0, c->gstream>>>(bs, hb.first);
            it = hb.first;
            continue;
        }
        it = end;
    }
    cudaEventRecord(c->ev1, c->gstream);
    cudaGraphExecDestroy(exec);
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
        long long per_iter = 3;
        for (int v = 0; v < nvol; ++v)
            per_iter += (V[v].k.n > 0 ? 3 : 0) + 4 + 5 * ((V[v].k.g.key_bits + 7) / 8) + 1 + 1 + 2 + (V[v].k.n > 0 ? 1 : 0);
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
            st = ensure(c, c->adam, sizeof(float) * 24 * (ntot > 0 ? ntot : 1), c->gstream);
            if (st != GVE_OK) return st;
            long long off = 0;
            for (int v = 0; v < nvol; ++v) {
                V[v].m = (float*)c->adam.p + 12 * off;
                V[v].v = nullptr;
                off += V[v].k.n;
                cudaMemsetAsync(c->sub[v]->acc.p, 0, sizeof(float) * 12 * (V[v].k.n > 0 ? V[v].k.n : 1), V[v].k.s);
            }
            float total = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                for (int v = 0; v < nvol; ++v) {
                    gve_ctx* s = c->sub[v];
                    cudaEventRecord(s->ev0, V[v].k.s);
                    bin_all(V[v].k, V[v].prims, &o, 0);
                    launch_eval_update(V[v], &o, nullptr, nullptr, nvol, v, nullptr, false);
                    cudaEventRecord(s->ev1, V[v].k.s);
                }
                for (int v = 0; v < nvol; ++v) {
                    if (cudaStreamSynchronize(V[v].k.s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "sync");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, c->sub[v]->ev0, c->sub[v]->ev1);
                    if (rep > 0) total += ms;  // first repetition warms up
                }
            }
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
