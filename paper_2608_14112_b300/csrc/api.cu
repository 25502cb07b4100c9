// api.cu -- the C ABI of libgve (see include/gve.h): argument checks, context
// scratch, and the launch sequences of evaluation, gradient and refinement.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "gve_int.cuh"

namespace gve {

int num_sms()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        return 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

gve_status cuda_fail(gve_ctx* c, cudaError_t e, const char* what)
{
    if (c) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
        c->err = buf;
    }
    return GVE_E_CUDA;
}

gve_status fail(gve_ctx* c, gve_status s, const char* msg)
{
    if (c) c->err = msg;
    return s;
}

gve_status ensure(gve_ctx* c, Buf& b, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return GVE_OK;
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "sync before regrow");
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    // fault-injection hook (host side): GVE_FAULT=alloc makes every scratch
    // allocation fail as an exhausted device would
    if (const char* f = getenv("GVE_FAULT"))
        if (strcmp(f, "alloc") == 0) return fail(c, GVE_E_NOMEM, "device scratch allocation failed (injected)");
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, GVE_E_NOMEM, "device scratch allocation failed");
    }
    b.bytes = want;
    return GVE_OK;
}

// split the sorted values into Gaussian ids and (optionally) sub-brick masks
__global__ void k_strip_mask(uint32_t* v, uint8_t* masks, unsigned long long n)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t x = v[i];
        if (masks) masks[i] = (uint8_t)(x >> kGidBits);
        v[i] = x & kGidMask;
    }
}

__global__ void k_reset_state(DevState* st)
{
    st->total = 0;
    st->max_total = 0;
    st->total1 = 0;
    st->max_total1 = 0;
    st->overflow = 0;
    st->first_overflow_iter = INT_MAX;
    st->err = 0;
    st->sse[0] = 0.0;
    st->sse[1] = 0.0;
    st->kept = 0;
    st->cand = 0;
    st->listed = 0;
}

}  // namespace gve

using namespace gve;

#define GVE_TRY(x)                               \
    do {                                         \
        gve_status _s = (x);                     \
        if (_s != GVE_OK) return _s;             \
    } while (0)
#define GVE_CUDA(x, what)                                  \
    do {                                                   \
        cudaError_t _e = (x);                              \
        if (_e != cudaSuccess) return cuda_fail(c, _e, what); \
    } while (0)

namespace gve {

DevState* dstate(gve_ctx* c) { return reinterpret_cast<DevState*>(c->state.p); }

gve_status check_common(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o)
{
    if (!c) return GVE_E_INVALID;
    if (!o) return fail(c, GVE_E_INVALID, "null options");
    if (n < 0 || n > (int64_t)kGidMask + 1) return fail(c, GVE_E_INVALID, "primitive count out of range (max 2^24)");
    if (n > 0 && !prims) return fail(c, GVE_E_INVALID, "null primitive pointer");
    if (prims && (reinterpret_cast<uintptr_t>(prims) & 15u)) return fail(c, GVE_E_INVALID, "primitives not 16-byte aligned");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    // the conservative brick cover's float32 margins hold for coordinates below 2^14
    if (d.nx > (1 << 14) || d.ny > (1 << 14) || d.nz > (1 << 14))
        return fail(c, GVE_E_INVALID, "grid axis above 2^14 voxels (evaluation limit)");
    if (o->brick != 4 && o->brick != 8 && o->brick != 16) return fail(c, GVE_E_INVALID, "brick edge must be 4, 8 or 16");
    if (o->gaussians_per_block != 0 && o->gaussians_per_block != 32 && o->gaussians_per_block != 64)
        return fail(c, GVE_E_INVALID, "gaussians_per_block must be 0, 32 or 64");
    if (!(o->trunc_k > 0.f) || !std::isfinite(o->trunc_k)) return fail(c, GVE_E_INVALID, "trunc_k must be positive");
    if (o->normalized && !(o->rho0 > 0.f)) return fail(c, GVE_E_INVALID, "rho0 must be positive");
    BinGeom g = make_geom(d, o->brick);
    if (g.nbricks > (long long)INT_MAX || g.key_bits > 31) return fail(c, GVE_E_INVALID, "grid too large");
    return GVE_OK;
}

gve_status reset_state(Call& k)
{
    k_reset_state<<<1, 1, 0, k.s>>>(dstate(k.c));
    k.c->launches += 1;
    return GVE_OK;
}

gve_status read_state(Call& k, DevState* out)
{
    gve_ctx* c = k.c;
    GVE_CUDA(cudaMemcpyAsync(c->hstate, c->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, k.s), "state readback");
    GVE_CUDA(cudaStreamSynchronize(k.s), "state sync");
    *out = *c->hstate;
    return GVE_OK;
}

// per-Gaussian, per-tile and per-brick scratch
gve_status size_static(Call& k)
{
    gve_ctx* c = k.c;
    long long n = k.n > 0 ? k.n : 1;
    GVE_TRY(ensure(c, c->rec, sizeof(float4) * 3 * n, k.s));
    GVE_TRY(ensure(c, c->binrec, sizeof(BinRec) * n, k.s));
    GVE_TRY(ensure(c, c->counts, sizeof(uint32_t) * n, k.s));
    GVE_TRY(ensure(c, c->offsets, sizeof(unsigned long long) * (n + 1), k.s));
    GVE_TRY(ensure(c, c->acc, sizeof(float) * 12 * n, k.s));
    GVE_TRY(ensure(c, c->scanp, sizeof(unsigned long long) * kScanBlocks, k.s));
    const long long nt = k.vt.toff[k.vt.nvol], nb = k.vt.boff[k.vt.nvol];
    GVE_TRY(ensure(c, c->trange, sizeof(uint32_t) * 2 * nt, k.s));
    GVE_TRY(ensure(c, c->cbase, sizeof(uint32_t) * 64 * cbase_chunks(c->cap1, nt), k.s));
    GVE_TRY(ensure(c, c->bcount, sizeof(uint32_t) * nb, k.s));
    GVE_TRY(ensure(c, c->boff, sizeof(unsigned long long) * (nb + 1), k.s));
    GVE_TRY(ensure(c, c->ranges, sizeof(uint32_t) * 2 * nb, k.s));
    GVE_TRY(ensure(c, c->part, sizeof(double2) * (nb + 1024), k.s));
    return GVE_OK;
}

namespace {
// capacity for `need` pairs plus headroom for Gaussians that grow during
// refinement: 1/4 for brick pairs, 1/1 for the ten times fewer tile pairs
// (whose count follows the boxes' volume more steeply)
unsigned long long grown(unsigned long long need, bool tiles)
{
    unsigned long long cap = need + (tiles ? need : need / 4) + 65536;
    return cap > 0xFFFFFFFFull ? 0xFFFFFFFFull : cap;
}
}  // namespace

gve_status grow_pairs(Call& k, unsigned long long need1, unsigned long long need2)
{
    gve_ctx* c = k.c;
    if (need1 > c->cap1 || !c->keys[0].p) {
        const unsigned long long cap = grown(need1, true);
        if (need1 > cap) return fail(c, GVE_E_CAPACITY, "more than 2^32 tile pairs");
        for (int b = 0; b < 2; ++b) {
            GVE_TRY(ensure(c, c->keys[b], sizeof(uint32_t) * cap, k.s));
            GVE_TRY(ensure(c, c->vals[b], sizeof(uint32_t) * cap, k.s));
        }
        GVE_TRY(ensure(c, c->tmask, sizeof(unsigned long long) * cap, k.s));
        GVE_TRY(ensure(c, c->cbase, sizeof(uint32_t) * 64 * cbase_chunks(cap, k.vt.toff[k.vt.nvol]), k.s));
        GVE_TRY(ensure(c, c->hist, sizeof(uint32_t) * 256 * ((cap + kSortTile - 1) / kSortTile + 1), k.s));
        c->cap1 = cap;
    }
    if (need2 > c->cap || !c->pairs.p) {
        const unsigned long long cap = grown(need2, false);
        if (need2 > cap) return fail(c, GVE_E_CAPACITY, "more than 2^32 brick pairs");
        GVE_TRY(ensure(c, c->pairs, sizeof(uint32_t) * cap, k.s));
        c->cap = cap;
    }
    return GVE_OK;
}

// sizing: the binning runs until both pair buffers hold its totals (three
// runs at most: tile pairs, then brick pairs, are found too large)
// test hook: a logical pair capacity below what the binning needs, to
// exercise the overflow detection and replay of refinement
void test_pair_cap(gve_ctx* c)
{
    if (const char* tc = getenv("GVE_TEST_PAIR_CAP")) {
        const unsigned long long t = strtoull(tc, nullptr, 10);
        if (t > 0 && t < c->cap) c->cap = t;
    }
}

gve_status size_pairs(Call& k, const float* prims, const gve_eval_opts* o)
{
    gve_ctx* c = k.c;
    GVE_TRY(size_static(k));
    GVE_TRY(grow_pairs(k, 0, 0));
    for (int run = 0; run < 3; ++run) {
        reset_state(k);
        GVE_TRY(bin_all(k, prims, o, 0));
        DevState h;
        GVE_TRY(read_state(k, &h));
        if (!h.overflow) break;
        const bool tiles = h.total1 > c->cap1;
        GVE_TRY(grow_pairs(k, h.total1, tiles ? 0 : h.total));
        if (!tiles) break;  // the brick total was complete: both sizes known
    }
    test_pair_cap(c);
    reset_state(k);
    return GVE_OK;
}

// one binning of prims (tagged iteration 0) into pair buffers large enough
// for it: a context whose buffers already hold it bins once; otherwise the
// buffers grow and the binning runs again (four runs at most).  On return the
// device state holds that binning's totals and zero counters.
gve_status bin_sized(Call& k, const float* prims, const gve_eval_opts* o)
{
    gve_ctx* c = k.c;
    GVE_TRY(size_static(k));
    GVE_TRY(grow_pairs(k, 0, 0));
    for (int run = 0; run < 4; ++run) {
        reset_state(k);
        GVE_TRY(bin_all(k, prims, o, 0));
        DevState h;
        GVE_TRY(read_state(k, &h));
        if (!h.overflow) return GVE_OK;
        const bool tiles = h.total1 > c->cap1;
        GVE_TRY(grow_pairs(k, h.total1, tiles ? 0 : h.total));
    }
    return fail(c, GVE_E_CAPACITY, "pair count kept growing past capacity");
}

BinBufs bin_bufs(Call& k, uint32_t* gcount)
{
    gve_ctx* c = k.c;
    BinBufs b{};
    b.rec = (float4*)c->rec.p;
    b.br = (BinRec*)c->binrec.p;
    b.tcount = (uint32_t*)c->counts.p;
    b.toff = (unsigned long long*)c->offsets.p;
    b.scanp = c->scanp.p;
    for (int i = 0; i < 2; ++i) {
        b.tkeys[i] = (uint32_t*)c->keys[i].p;
        b.tvals[i] = (uint32_t*)c->vals[i].p;
    }
    b.hist = (uint32_t*)c->hist.p;
    b.tmask = (unsigned long long*)c->tmask.p;
    b.cbase = (uint32_t*)c->cbase.p;
    b.cap1 = c->cap1;
    b.trange = (uint32_t*)c->trange.p;
    b.bcount = (uint32_t*)c->bcount.p;
    b.boff = (unsigned long long*)c->boff.p;
    b.ranges = (uint32_t*)c->ranges.p;
    b.pairs = (uint32_t*)c->pairs.p;
    b.cap = c->cap;
    b.gcount = gcount;
    b.st = dstate(c);
    return b;
}

// full binning: prep, tile pairs and their sort, brick counts, ranges and
// the brick pairs
gve_status bin_all(Call& k, const float* prims, const gve_eval_opts* o, int iter, uint32_t* gcount)
{
    gve_ctx* c = k.c;
    c->launches += launch_binning(bin_bufs(k, gcount), prims, k.n, k.vt, o->trunc_k, iter, k.s);
    GVE_CUDA(cudaGetLastError(), "launch (binning)");
    return GVE_OK;
}

BrickArgs brick_args(Call& k, const gve_eval_opts* o)
{
    gve_ctx* c = k.c;
    BrickArgs a{};
    a.g = k.g;
    a.start = (const uint32_t*)c->ranges.p;
    a.end = a.start + k.g.nbricks;
    a.gids = (const uint32_t*)c->pairs.p;
    a.rec = (const float4*)c->rec.p;
    a.part = (float2*)c->part.p;
    a.st = dstate(c);
    double k2 = (double)o->trunc_k * (double)o->trunc_k;
    a.T = (float)(k2 * kNegHalfLog2e);
    a.rho0 = o->rho0;
    a.normalized = o->normalized;
    a.mask_thresh = -1.f;
    a.inv_m = (float)(1.0 / ((double)k.g.nx * k.g.ny * k.g.nz));
    a.chunk = o->gaussians_per_block;
    return a;
}

gve_status begin(gve_ctx* c, Call& k, int64_t n, gve_dims d, const gve_eval_opts* o, void* stream)
{
    k.c = c;
    k.s = (cudaStream_t)stream;
    k.n = n;
    k.g = make_geom(d, o->brick);
    k.vt = single_volume(k.g, n);
    c->launches = 0;
    GVE_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    GVE_TRY(ensure(c, c->state, sizeof(DevState), k.s));
    return GVE_OK;
}

}  // namespace gve

extern "C" {

const char* gve_status_str(gve_status s)
{
    switch (s) {
        case GVE_OK: return "ok";
        case GVE_E_INVALID: return "invalid argument";
        case GVE_E_BUDGET: return "infeasible budget";
        case GVE_E_NOMEM: return "out of device memory";
        case GVE_E_CUDA: return "CUDA error";
        case GVE_E_TIMEOUT: return "device wait timed out";
        case GVE_E_CAPACITY: return "pair capacity exceeded";
        case GVE_E_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char* gve_last_error(const gve_ctx* c) { return c ? c->err.c_str() : "null context"; }

gve_status gve_ctx_create(gve_ctx** out, int device)
{
    if (!out) return GVE_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GVE_E_INVALID;
    }
    if (cudaSetDevice(device) != cudaSuccess) return GVE_E_CUDA;
    gve_ctx* c = new gve_ctx();
    c->device = device;
    if (cudaMallocHost(&c->hstate, sizeof(DevState)) != cudaSuccess) {
        delete c;
        return GVE_E_NOMEM;
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        cudaFreeHost(c->hstate);
        delete c;
        return GVE_E_CUDA;
    }
    *out = c;
    return GVE_OK;
}

void gve_ctx_destroy(gve_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    Buf* bufs[] = {&c->rec, &c->binrec, &c->counts, &c->offsets, &c->acc, &c->adam, &c->keys[0], &c->keys[1],
                   &c->vals[0], &c->vals[1], &c->tmask, &c->trange, &c->cbase, &c->bcount, &c->csum, &c->boff, &c->pairs, &c->hist, &c->scanp, &c->ranges, &c->part, &c->state,
                   &c->a_g, &c->a_keys, &c->a_sel, &c->a_tmp, &c->a_cnt, &c->trace,
                   &c->s_hi, &c->s_mid, &c->s_cnt, &c->s_off, &c->s_pts, &c->s_cell, &c->s_order, &c->s_nd,
                   &c->s_gg, &c->s_loss, &c->s_inv, &c->s_ex, &c->s_terms, &c->s_ccnt, &c->s_cand, &c->r_rec, &c->r_cnt, &c->r_off, &c->r_keys[0], &c->r_keys[1],
                   &c->r_vals[0], &c->r_vals[1], &c->r_hist, &c->r_scanp, &c->r_rng, &c->r_crec, &c->r_state};
    for (Buf* b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->hstate) cudaFreeHost(c->hstate);
    if (c->sev_ready)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 64; ++b) cudaEventDestroy(c->sev[a][b]);
    for (gve_ctx* w : c->asub) gve_ctx_destroy(w);
    for (cudaStream_t as : c->astream) cudaStreamDestroy(as);
    for (cudaEvent_t ev : c->ajoin) cudaEventDestroy(ev);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->bstate.p) cudaFree(c->bstate.p);
    if (c->btab.p) cudaFree(c->btab.p);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

gve_status gve_evaluate(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                        float* field_out, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!field_out) return fail(c, GVE_E_INVALID, "null output field");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(bin_sized(k, prims, o));
    BrickArgs a = brick_args(k, o);
    a.field_out = field_out;
    launch_brick(kModeEval, a, k.s);
    GVE_CUDA(cudaGetLastError(), "launch (evaluate)");
    return GVE_OK;
}

gve_status gve_loss_grad(gve_ctx* c, const float* prims, int64_t n, const float* field, gve_dims d,
                         const gve_eval_opts* o, float mask_thresh, float* grad, double* sse_dev, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!field) return fail(c, GVE_E_INVALID, "null target field");
    if (n > 0 && !grad) return fail(c, GVE_E_INVALID, "null gradient output");
    if (grad && (reinterpret_cast<uintptr_t>(grad) & 15u)) return fail(c, GVE_E_INVALID, "gradient not 16-byte aligned");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(bin_sized(k, prims, o));
    GVE_CUDA(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (n > 0 ? n : 1), k.s), "memset acc");
    BrickArgs a = brick_args(k, o);
    a.field = field;
    a.mask_thresh = mask_thresh;
    a.acc = (float*)c->acc.p;
    launch_brick(kModeLoss, a, k.s);
    launch_sse_reduce(a.part, k.g.nbricks, dstate(c), nullptr, 0, 0.0, k.s);
    launch_chain((float*)c->acc.p, (float*)c->acc.p, const_cast<float*>(prims), n, grad, nullptr, nullptr, nullptr,
                 dstate(c), k.s);
    if (sse_dev)
        GVE_CUDA(cudaMemcpyAsync(sse_dev, dstate(c)->sse, 2 * sizeof(double), cudaMemcpyDeviceToDevice, k.s),
                 "copy sse");
    GVE_CUDA(cudaGetLastError(), "launch (loss_grad)");
    return GVE_OK;
}

gve_status gve_backward(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                        const float* grad_field, float* grad, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!grad_field) return fail(c, GVE_E_INVALID, "null upstream gradient");
    if (n > 0 && !grad) return fail(c, GVE_E_INVALID, "null gradient output");
    if (grad && (reinterpret_cast<uintptr_t>(grad) & 15u)) return fail(c, GVE_E_INVALID, "gradient not 16-byte aligned");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(bin_sized(k, prims, o));
    GVE_CUDA(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * (n > 0 ? n : 1), k.s), "memset acc");
    BrickArgs a = brick_args(k, o);
    a.upstream = grad_field;
    a.acc = (float*)c->acc.p;
    launch_brick(kModeBwd, a, k.s);
    launch_chain((float*)c->acc.p, (float*)c->acc.p, const_cast<float*>(prims), n, grad, nullptr, nullptr, nullptr,
                 dstate(c), k.s);
    GVE_CUDA(cudaGetLastError(), "launch (backward)");
    return GVE_OK;
}

gve_status gve_bin(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                   uint32_t* counts, uint32_t* keys, uint32_t* gids, uint8_t* masks, int64_t cap,
                   uint32_t* ranges, int64_t* n_pairs, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!n_pairs || (n > 0 && !counts) || !ranges || cap < 0) return fail(c, GVE_E_INVALID, "null output");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(size_pairs(k, prims, o));
    GVE_TRY(bin_all(k, prims, o, 0, n > 0 ? counts : nullptr));
    DevState h;
    GVE_TRY(read_state(k, &h));
    *n_pairs = (int64_t)h.total;
    if (h.overflow) return fail(c, GVE_E_INTERNAL, "pair buffer sized by the sizing pass overflowed");
    if ((int64_t)h.total > cap) return fail(c, GVE_E_CAPACITY, "output capacity below the pair count");
    if (h.total > 0) {
        if (!keys || !gids) return fail(c, GVE_E_INVALID, "null pair outputs");
        launch_fill_keys((const uint32_t*)c->ranges.p, k.g.nbricks, keys, k.s);
        GVE_CUDA(cudaMemcpyAsync(gids, c->pairs.p, sizeof(uint32_t) * h.total, cudaMemcpyDeviceToDevice, k.s), "copy");
        k_strip_mask<<<4 * num_sms(), 256, 0, k.s>>>(gids, masks, h.total);
    }
    GVE_CUDA(cudaMemcpyAsync(ranges, c->ranges.p, sizeof(uint32_t) * 2 * k.g.nbricks, cudaMemcpyDeviceToDevice, k.s), "copy");
    GVE_CUDA(cudaStreamSynchronize(k.s), "sync");
    return GVE_OK;
}

gve_status gve_count_pairs(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                           int64_t* kept, int64_t* cand, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!kept || !cand) return fail(c, GVE_E_INVALID, "null output");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(bin_sized(k, prims, o));
    BrickArgs a = brick_args(k, o);
    launch_brick(kModeCount, a, k.s);
    GVE_CUDA(cudaGetLastError(), "launch (count)");
    DevState h;
    GVE_TRY(read_state(k, &h));
    *kept = (int64_t)h.kept;
    *cand = (int64_t)h.cand;
    return GVE_OK;
}

gve_status gve_kept_pairs(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                          uint64_t* pairs, int64_t cap, int64_t* n_pairs, void* stream)
{
    GVE_TRY(check_common(c, prims, n, d, o));
    if (!n_pairs || cap < 0 || (cap > 0 && !pairs)) return fail(c, GVE_E_INVALID, "null output");
    if ((int64_t)d.nx * d.ny * d.nz > ((int64_t)1 << 40)) return fail(c, GVE_E_INVALID, "grid above 2^40 voxels");
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    GVE_TRY(bin_sized(k, prims, o));
    BrickArgs a = brick_args(k, o);
    a.pairs = reinterpret_cast<unsigned long long*>(pairs);
    a.pairs_cap = (unsigned long long)cap;
    launch_brick(kModeCount, a, k.s);
    GVE_CUDA(cudaGetLastError(), "launch (kept pairs)");
    DevState h;
    GVE_TRY(read_state(k, &h));
    *n_pairs = (int64_t)h.listed;
    if (h.listed > (unsigned long long)cap) return fail(c, GVE_E_CAPACITY, "more kept pairs than the output holds");
    return GVE_OK;
}

gve_status gve_refine(gve_ctx* c, float* prims, int64_t n, const float* field, gve_dims d, const gve_schedule* sc,
                      float* adam_state, double* trace, gve_stats* stats, void* stream)
{
    if (!sc) return fail(c, GVE_E_INVALID, "null schedule");
    GVE_TRY(check_common(c, prims, n, d, &sc->eval));
    if (!field) return fail(c, GVE_E_INVALID, "null target field");
    if (sc->iters < 0) return fail(c, GVE_E_INVALID, "negative iteration count");
    if (!(sc->lr >= 0.f) || !(sc->beta1 >= 0.f && sc->beta1 < 1.f) || !(sc->beta2 >= 0.f && sc->beta2 < 1.f) ||
        !(sc->eps >= 0.f) || sc->step0 < 0)
        return fail(c, GVE_E_INVALID, "bad Adam hyper-parameters");
    if (adam_state && (reinterpret_cast<uintptr_t>(adam_state) & 15u))
        return fail(c, GVE_E_INVALID, "adam state not 16-byte aligned");
    const gve_eval_opts* o = &sc->eval;
    Call k;
    GVE_TRY(begin(c, k, n, d, o, stream));
    if (c->keys[0].p && c->pairs.p) {
        // pair buffers from an earlier call: the first iteration's binning
        // sizes them (an overflow grows them and replays from there)
        GVE_TRY(size_static(k));
        GVE_TRY(grow_pairs(k, 0, 0));
        test_pair_cap(c);
        reset_state(k);
    } else {
        GVE_TRY(size_pairs(k, prims, o));
    }
    long long nn = n > 0 ? n : 1;
    float* m = adam_state;
    if (!m) {
        GVE_TRY(ensure(c, c->adam, sizeof(float) * 24 * nn, k.s));
        m = (float*)c->adam.p;
        GVE_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * 24 * nn, k.s), "memset adam");
    }
    float* v = m + 12 * nn;
    if (adam_state) v = adam_state + 12 * n;
    double* tr = trace;
    if (!tr) {
        GVE_TRY(ensure(c, c->trace, sizeof(double) * (sc->iters + 1), k.s));
        tr = (double*)c->trace.p;
    }
    GVE_CUDA(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * nn, k.s), "memset acc");
    const bool timed = stats != nullptr;
    if (timed && !c->sev_ready) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 64; ++b) GVE_CUDA(cudaEventCreate(&c->sev[a][b]), "event create");
        c->sev_ready = true;
    }
    GVE_CUDA(cudaEventRecord(c->ev0, k.s), "event");
    const double inv_m = 1.0 / ((double)d.nx * d.ny * d.nz);
    int retries = 0;
    int it = 0;
    const int seg = 64;
    double ms_brick = 0.0, ms_bin = 0.0;
    while (it < sc->iters) {
        int end = it + seg < sc->iters ? it + seg : sc->iters;
        for (int t = it; t < end; ++t) {
            if (timed) GVE_CUDA(cudaEventRecord(c->sev[0][t - it], k.s), "event");
            GVE_TRY(bin_all(k, prims, o, t));
            if (timed) GVE_CUDA(cudaEventRecord(c->sev[1][t - it], k.s), "event");
            BrickArgs a = brick_args(k, o);
            a.field = field;
            a.mask_thresh = sc->mask_thresh;
            a.acc = (float*)c->acc.p;
            // the sums start from zero each iteration (a memset is cheaper
            // than clearing them in the chain-rule kernel after reading)
            GVE_CUDA(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * nn, k.s), "memset acc");
            launch_brick(kModeLoss, a, k.s);
            if (timed) GVE_CUDA(cudaEventRecord(c->sev[2][t - it], k.s), "event");
            launch_sse_reduce(a.part, k.g.nbricks, dstate(c), tr, t, inv_m, k.s);
            AdamArgs ad{};
            ad.lr = sc->lr; ad.b1 = sc->beta1; ad.b2 = sc->beta2; ad.eps = sc->eps;
            int step = sc->step0 + t + 1;
            ad.bc1 = (float)(1.0 - std::pow((double)sc->beta1, step));
            ad.bc2 = (float)(1.0 - std::pow((double)sc->beta2, step));
            launch_chain((float*)c->acc.p, nullptr, prims, n, nullptr, m, v, &ad, dstate(c), k.s);
            c->launches += 1 + 2 + (n > 0 ? 1 : 0);
        }
        GVE_CUDA(cudaGetLastError(), "launch (refine)");
        DevState h;
        GVE_TRY(read_state(k, &h));
        if (h.overflow) {
            if (++retries > 8) return fail(c, GVE_E_CAPACITY, "pair count kept growing past capacity");
            GVE_TRY(grow_pairs(k, h.max_total1, h.max_total));
            GVE_CUDA(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * 12 * nn, k.s), "memset acc");
            reset_state(k);
            it = h.first_overflow_iter;
            continue;
        }
        if (timed) {
            for (int t = it; t < end; ++t) {
                float a = 0.f, b = 0.f;
                cudaEventElapsedTime(&a, c->sev[0][t - it], c->sev[1][t - it]);
                cudaEventElapsedTime(&b, c->sev[1][t - it], c->sev[2][t - it]);
                ms_bin += a;
                ms_brick += b;
            }
        }
        it = end;
    }
    // final evaluation after the last update: the brick evaluator's forward
    // phase alone (no gradient sums), timed on its own
    GVE_TRY(bin_all(k, prims, o, sc->iters));
    DevState h;
    {
        BrickArgs a = brick_args(k, o);
        a.field = field;
        a.mask_thresh = sc->mask_thresh;
        a.acc = nullptr;
        if (timed) GVE_CUDA(cudaEventRecord(c->sev[0][0], k.s), "event");
        launch_brick(kModeLoss, a, k.s);
        if (timed) GVE_CUDA(cudaEventRecord(c->sev[1][0], k.s), "event");
        launch_sse_reduce(a.part, k.g.nbricks, dstate(c), nullptr, 0, inv_m, k.s);
        c->launches += 3;
    }
    GVE_CUDA(cudaEventRecord(c->ev1, k.s), "event");
    GVE_CUDA(cudaGetLastError(), "launch (refine final)");
    GVE_TRY(read_state(k, &h));
    bool fwd_timed = timed;
    if (h.overflow) {
        // the final evaluation alone overflowed: grow and redo it (untimed)
        fwd_timed = false;
        GVE_TRY(grow_pairs(k, h.max_total1, h.max_total));
        reset_state(k);
        GVE_TRY(bin_all(k, prims, o, sc->iters));
        BrickArgs a = brick_args(k, o);
        a.field = field;
        a.mask_thresh = sc->mask_thresh;
        launch_brick(kModeLoss, a, k.s);
        launch_sse_reduce(a.part, k.g.nbricks, dstate(c), nullptr, 0, inv_m, k.s);
        GVE_TRY(read_state(k, &h));
        if (h.overflow) return fail(c, GVE_E_CAPACITY, "final evaluation overflowed");
        ++retries;
    }
    if (stats) {
        double first = 0.0, last = 0.0;
        if (sc->iters > 0) {
            GVE_CUDA(cudaMemcpy(&first, tr, sizeof(double), cudaMemcpyDeviceToHost), "trace");
            GVE_CUDA(cudaMemcpy(&last, tr + sc->iters - 1, sizeof(double), cudaMemcpyDeviceToHost), "trace");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        stats->loss_first = first;
        stats->loss_last = last;
        stats->sse_final = h.sse[1];
        double M = (double)d.nx * d.ny * d.nz;
        stats->psnr_final = h.sse[1] > 0.0 ? 10.0 * std::log10(M / h.sse[1]) : INFINITY;
        stats->brick_pairs = (int64_t)h.total;
        stats->iters_done = sc->iters;
        stats->retries = retries;
        stats->ms_total = ms;
        stats->ms_brick = (float)ms_brick;
        stats->ms_bin = (float)ms_bin;
        float msf = 0.f;
        if (fwd_timed) cudaEventElapsedTime(&msf, c->sev[0][0], c->sev[1][0]);
        stats->ms_fwd = msf;
        stats->launches = c->launches;
    }
    return GVE_OK;
}

gve_status gve_structure_stats(gve_ctx* c, const float* field, gve_dims d, double* out, double* stage_ms,
                               void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!field || !out) return fail(c, GVE_E_INVALID, "null argument");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (d.nx > (1 << 24) || d.ny > (1 << 24) || d.nz > (1 << 24)) return fail(c, GVE_E_INVALID, "grid axis above 2^24");
    GVE_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    c->launches = 0;
    return gve::structure_stats(c, field, d, out, stage_ms, (cudaStream_t)stream);
}

gve_status gve_allocate(gve_ctx* c, const float* field, gve_dims d, int64_t budget, const gve_alloc_opts* o,
                        float* prims, int64_t* feasible_max, gve_alloc_info* info, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!field || !o) return fail(c, GVE_E_INVALID, "null argument");
    if (budget < 0 || budget > (int64_t)INT_MAX) return fail(c, GVE_E_INVALID, "budget out of range");
    if (budget > 0 && !prims) return fail(c, GVE_E_INVALID, "null primitive output");
    if (prims && (reinterpret_cast<uintptr_t>(prims) & 15u)) return fail(c, GVE_E_INVALID, "primitives not 16-byte aligned");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (d.nx > (1 << 24) || d.ny > (1 << 24) || d.nz > (1 << 24)) return fail(c, GVE_E_INVALID, "grid axis above 2^24");
    if (!(o->detail_frac >= 0.0 && o->detail_frac <= 1.0)) return fail(c, GVE_E_INVALID, "detail_frac outside [0,1]");
    if (!(o->w0 > 0.f && o->w0 < 1.f)) return fail(c, GVE_E_INVALID, "w0 outside (0,1)");
    GVE_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    return gve::allocate(c, field, d, budget, o, prims, feasible_max, info, (cudaStream_t)stream);
}

}  // extern "C"
