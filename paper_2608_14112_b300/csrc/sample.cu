// sample.cu -- stratified-sample refinement (Sec. III-F; Table III: 3,072
// jittered points per iteration, 35 / 40 / 25 % from high-value, occupied
// mid-range and all voxels): Eq. 3, the value loss and its gradient at the
// iteration's points, then the shared chain rule and Adam (optim.cu).
//
// The points are few (at most kMaxSamples), so they are bucketed into a
// coarse grid of cells (32^3 voxels, coarser for very large grids) by a
// counting sort (z-major cells, cstart[c] = the number of points in cells
// before c), and the Gaussians do the searching:
// one thread per Gaussian walks the (z, y) rows of cells its conservative
// box overlaps -- the points of a row's cell range are one contiguous run of
// the sorted points -- and tests each with the same float32 keep chain as
// the voxel path (kept iff t > T).  A Gaussian whose box spans more rows
// than half the number of points scans all points instead (training can
// grow a few Gaussians to cover the grid).  The forward adds w a G and w G into the
// point's sums with float atomics; the backward repeats the search and
// accumulates the Gaussian's sums A = sum G gn, H = sum h and the moments
// of h = G (a gn + gd) over d = p - mu in registers, then writes them to
// the accumulator layout the chain rule reads.  Nothing per pair is stored.
//
// Box of Gaussian i: centre mu, half-extent kb sqrt(Sigma_jj) with
// kb = k (1.001 + 1e-5 cond) (cond = (s_max / s_min)^2) plus 0.05 voxel,
// in float32: its margins cover the float32 rounding of the keep chain.
#include <cmath>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kMaxSamples = 8192;
constexpr long long kMaxCells = 1ll << 21;

struct CellGrid {
    int shift;  // cell edge = 2^shift voxels
    int ncx, ncy, ncz;
};

CellGrid make_cells(gve_dims d)
{
    CellGrid g{};
    for (g.shift = 5;; ++g.shift) {   // 32-voxel cells unless the grid needs more than kMaxCells
        g.ncx = ((d.nx - 1) >> g.shift) + 1;
        g.ncy = ((d.ny - 1) >> g.shift) + 1;
        g.ncz = ((d.nz - 1) >> g.shift) + 1;
        if ((long long)g.ncx * g.ncy * g.ncz <= kMaxCells) break;
    }
    return g;
}

// voxel coordinate floor(p) clamped to the grid, then its cell
__device__ __forceinline__ int cell_of(float p, int n, int shift, int nc)
{
    int v = (int)floorf(p);
    v = v < 0 ? 0 : (v > n - 1 ? n - 1 : v);
    const int c = v >> shift;
    return c < nc ? c : nc - 1;
}

// Points by cell: a counting sort (the order of points inside a cell does
// not matter: the forward adds into each point's sums atomically).  Count
// per cell, one CTA scans the counts into cstart[c] = the points in cells
// before c (c = 0 .. ncells), then each point takes a slot of its cell by
// counting the cell back down (the counters end at zero, ready for the next
// iteration).  Writes the sorted points, their original indices and the
// sorted position of each original index.
__device__ __forceinline__ uint32_t point_cell(const float4& q, int nx, int ny, int nz, const CellGrid& cg)
{
    const int cx = cell_of(q.x, nx, cg.shift, cg.ncx), cy = cell_of(q.y, ny, cg.shift, cg.ncy),
              cz = cell_of(q.z, nz, cg.shift, cg.ncz);
    return (uint32_t)(((long long)cz * cg.ncy + cy) * cg.ncx + cx);
}

__global__ void __launch_bounds__(256) k_cell_count(const float4* __restrict__ pts, int P, int nx, int ny, int nz,
                                                    CellGrid cg, uint32_t* __restrict__ ccnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) atomicAdd(&ccnt[point_cell(pts[i], nx, ny, nz, cg)], 1u);
}

// One CTA scans the counts in tiles of 4,096 cells: each thread takes four
// consecutive cells with one 16-byte load (so a warp's loads and stores are
// contiguous), then warp and block scans of the thread sums and a running
// carry between tiles.  The loads of four tiles are issued before the first
// is scanned.
constexpr int kScanThreads = 1024;
constexpr int kScanTiles = 4;

__device__ __forceinline__ uint4 scan_load(const uint32_t* __restrict__ ccnt, long long c, long long ncells)
{
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (c + 3 < ncells) {
        v = *reinterpret_cast<const uint4*>(ccnt + c);
    } else {
        if (c < ncells) v.x = ccnt[c];
        if (c + 1 < ncells) v.y = ccnt[c + 1];
        if (c + 2 < ncells) v.z = ccnt[c + 2];
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_cell_scan(const uint32_t* __restrict__ ccnt, long long ncells,
                                                            uint32_t* __restrict__ cstart)
{
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr long long tile = 4LL * kScanThreads;
    uint32_t carry = 0;
    for (long long base = 0; base < ncells; base += kScanTiles * tile) {
        uint4 vt[kScanTiles];
#pragma unroll
        for (int u = 0; u < kScanTiles; ++u) vt[u] = scan_load(ccnt, base + u * tile + 4LL * threadIdx.x, ncells);
#pragma unroll
        for (int u = 0; u < kScanTiles; ++u) {
            const long long c = base + u * tile + 4LL * threadIdx.x;
            if (base + u * tile >= ncells) break;          // uniform across the block
            const uint4 v = vt[u];
            const uint32_t s1 = v.x + v.y, s2 = s1 + v.z, s3 = s2 + v.w;
            uint32_t x = s3;                               // inclusive scan of the thread sums in the warp
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            if (lane == 31) wsum[w] = x;
            __syncthreads();
            if (w == 0) {                                  // inclusive scan of the warp sums
                uint32_t y = wsum[lane];
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
                    if (lane >= o) y += t;
                }
                wsum[lane] = y;
            }
            __syncthreads();
            const uint32_t e = carry + (w ? wsum[w - 1] : 0u) + x - s3;   // cells before this thread's first
            if (c + 3 < ncells) {
                *reinterpret_cast<uint4*>(cstart + c) = make_uint4(e, e + v.x, e + s1, e + s2);
            } else {
                if (c < ncells) cstart[c] = e;
                if (c + 1 < ncells) cstart[c + 1] = e + v.x;
                if (c + 2 < ncells) cstart[c + 2] = e + s1;
            }
            carry += wsum[kScanThreads / 32 - 1];
            __syncthreads();                               // wsum is rewritten by the next tile
        }
    }
    if (threadIdx.x == 0) cstart[ncells] = carry;
}

__global__ void __launch_bounds__(256) k_cell_scatter(const float4* __restrict__ pts, int P, int nx, int ny, int nz,
                                                      CellGrid cg, const uint32_t* __restrict__ cstart,
                                                      uint32_t* __restrict__ slot, float4* __restrict__ spts,
                                                      uint32_t* __restrict__ order, uint32_t* __restrict__ inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float4 q = pts[i];
    const uint32_t c = point_cell(q, nx, ny, nz, cg);
    const uint32_t pos = cstart[c] + atomicSub(&slot[c], 1u) - 1u;  // counts the cell back to zero
    spts[pos] = q;
    order[pos] = (uint32_t)i;
    inv[i] = pos;
}

struct SampleArgs {
    const float* prims;
    float4* rec;   // keep coefficients, written by the forward for Gaussians with candidates
    long long n;
    int nx, ny, nz;
    CellGrid cg;
    const uint32_t* cstart;   // [ncells + 1]
    int S;
    const float4* spts;
    float2* nd;          // per sorted point: (sum w a G, sum w G)
    const float2* gg;    // per sorted point: (dL/dnum, dL/dden)
    float* acc;          // [n][12] accumulators (backward)
    int4* cand;          // [0].x: count; then per listed Gaussian {i, lo}, {hi, 0}
    float k, T;
};

// Cell range of Gaussian i's conservative box; false for a record the
// preparation marks invalid (non-finite values, zero quaternion).
__device__ __forceinline__ bool gauss_cells(const SampleArgs& a, long long i, int lo[3], int hi[3])
{
    float mu[3], rad[3];
    const int kind = gauss_box(a.prims, i, a.k, mu, rad);
    if (kind == 0) return false;
    const int dims[3] = {a.nx, a.ny, a.nz};
    const int nc[3] = {a.cg.ncx, a.cg.ncy, a.cg.ncz};
    if (kind == 2) {  // scales beyond float range: every cell
        for (int j = 0; j < 3; ++j) { lo[j] = 0; hi[j] = nc[j] - 1; }
        return true;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float l = floorf(mu[j] - rad[j]), h = floorf(mu[j] + rad[j]);
        l = fminf(fmaxf(l, 0.f), (float)(dims[j] - 1));
        h = fminf(fmaxf(h, 0.f), (float)(dims[j] - 1));
        lo[j] = ((int)l) >> a.cg.shift;
        hi[j] = ((int)h) >> a.cg.shift;
    }
    return true;
}

// Calls f(s) for every sorted point s in the cells [lo, hi]: one contiguous
// run per (z, y) row of cells, or every point when the rows outnumber half
// the points.
template <class F>
__device__ __forceinline__ void for_candidates(const SampleArgs& a, const int lo[3], const int hi[3], F&& f)
{
    const long long rows = (long long)(hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    if (2 * rows >= a.S) {
        for (uint32_t s = 0; s < (uint32_t)a.S; ++s) f(s);
        return;
    }
    for (int cz = lo[2]; cz <= hi[2]; ++cz)
        for (int cy = lo[1]; cy <= hi[1]; ++cy) {
            const long long base = ((long long)cz * a.cg.ncy + cy) * a.cg.ncx;
            const uint32_t s0 = a.cstart[base + lo[0]], s1 = a.cstart[base + hi[0] + 1];
            for (uint32_t s = s0; s < s1; ++s) f(s);
        }
}

// whether any point lies in the cells [lo, hi] (the rows for_candidates walks)
__device__ __forceinline__ bool has_candidates(const SampleArgs& a, const int lo[3], const int hi[3])
{
    const long long rows = (long long)(hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    if (2 * rows >= a.S) return a.S > 0;
    for (int cz = lo[2]; cz <= hi[2]; ++cz)
        for (int cy = lo[1]; cy <= hi[1]; ++cy) {
            const long long base = ((long long)cz * a.cg.ncy + cy) * a.cg.ncx;
            if (a.cstart[base + hi[0] + 1] > a.cstart[base + lo[0]]) return true;
        }
    return false;
}

// The keep coefficients are computed here (float32, keep_coefficients, as
// in the voxel path's preparation), only for Gaussians whose box holds
// candidate points (about half of them at 1.4 M Gaussians against 6,144
// points), and stored for the gradient pass.  Those Gaussians (with a valid
// record) are listed with their cell box, so that the gradient pass visits
// only them.
__global__ void __launch_bounds__(128) k_sample_eval(const SampleArgs a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int lo[3], hi[3];
    if (!gauss_cells(a, i, lo, hi)) return;
    if (!has_candidates(a, lo, hi)) return;
    float pf[12];
    {
        const float4* p4 = reinterpret_cast<const float4*>(a.prims) + 3 * i;
        const float4 p0 = p4[0], p1 = p4[1], p2 = p4[2];
        const float q[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
        for (int j = 0; j < 12; ++j) pf[j] = q[j];
    }
    KeepCoef kc;
    keep_coefficients(pf, kc);
    const float4 r0 = kc.r0, r1 = kc.r1, r2 = kc.r2;
    a.rec[3 * i] = r0;
    a.rec[3 * i + 1] = r1;
    a.rec[3 * i + 2] = r2;
    if (!(r2.z > 0.f)) return;  // invalid record (weight zero)
    if (a.cand) {               // append to the list, one atomic per group of converged lanes
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
        unsigned slot = 0;
        if (lane == leader) slot = atomicAdd(reinterpret_cast<unsigned*>(a.cand), (unsigned)__popc(act));
        slot = __shfl_sync(act, slot, leader) + (unsigned)__popc(act & ((1u << lane) - 1u));
        a.cand[1 + 2 * (long long)slot] = make_int4((int)i, lo[0], lo[1], lo[2]);
        a.cand[2 + 2 * (long long)slot] = make_int4(hi[0], hi[1], hi[2], 0);
    }
    for_candidates(a, lo, hi, [&](uint32_t s) {
        const float4 q = a.spts[s];
        const float t = keep_t(r0, r1, r2, __fsub_rn(q.x, r0.x), __fsub_rn(q.y, r0.y), __fsub_rn(q.z, r0.z));
        if (!(t > a.T)) return;
        const float G = ex2_approx(t);
        atomicAdd(&a.nd[s].x, r2.y * G);
        atomicAdd(&a.nd[s].y, r2.z * G);
    });
}

// One thread per listed Gaussian (the others' sums stay zero: the caller
// clears acc); the grid covers all n, threads past the count return.
__global__ void __launch_bounds__(128) k_sample_grad(const SampleArgs a)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)(unsigned)a.cand[0].x) return;
    const int4 e0 = a.cand[1 + 2 * e], e1 = a.cand[2 + 2 * e];
    const long long i = e0.x;
    const int lo[3] = {e0.y, e0.z, e0.w}, hi[3] = {e1.x, e1.y, e1.z};
    float A = 0.f, H = 0.f, S1[3] = {0.f, 0.f, 0.f}, S2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float4 r0 = a.rec[3 * i], r1 = a.rec[3 * i + 1], r2 = a.rec[3 * i + 2];
    for_candidates(a, lo, hi, [&](uint32_t s) {
        const float4 q = a.spts[s];
        const float dx = __fsub_rn(q.x, r0.x), dy = __fsub_rn(q.y, r0.y), dz = __fsub_rn(q.z, r0.z);
        const float t = keep_t(r0, r1, r2, dx, dy, dz);
        if (!(t > a.T)) return;
        const float G = ex2_approx(t);
        const float2 g = a.gg[s];
        const float h = G * fmaf(r2.w, g.x, g.y);
        A = fmaf(G, g.x, A);
        H += h;
        S1[0] = fmaf(h, dx, S1[0]);
        S1[1] = fmaf(h, dy, S1[1]);
        S1[2] = fmaf(h, dz, S1[2]);
        S2[0] = fmaf(h * dx, dx, S2[0]);
        S2[1] = fmaf(h * dy, dy, S2[1]);
        S2[2] = fmaf(h * dz, dz, S2[2]);
        S2[3] = fmaf(h * dx, dy, S2[3]);
        S2[4] = fmaf(h * dx, dz, S2[4]);
        S2[5] = fmaf(h * dy, dz, S2[5]);
    });
    float4* o = reinterpret_cast<float4*>(a.acc) + 3 * i;
    o[0] = make_float4(A, H, S1[0], S1[1]);
    o[1] = make_float4(S1[2], S2[0], S2[1], S2[2]);
    o[2] = make_float4(S2[3], S2[4], S2[5], 0.f);
}

// One CTA: Vt = num / max(den, rho0) at each drawn sample and the terms of
// the objective that live at points, as FP64 sums: the masked value loss
// (1/S) sum 1[v > occ] (Vt - v)^2, the density term (1/S) sum 1[v > occ]
// (den - 1)^2 (den = rho = sum w G) and, with partners (the partner of
// sample j has original index S + j), the smoothness term (1/S) sum (den -
// den')^2.  Writes the upstream pair (dL/dnum, dL/dden) of every sorted
// point (a sample writes its partner's), the weighted total to loss and
// trace[iter], the unweighted terms to terms[0..2] (terms[3..5] cleared for
// the per-Gaussian terms), and vt_out (optional) by original index.
__global__ void __launch_bounds__(1024) k_sample_loss(const float4* __restrict__ spts, const uint32_t* __restrict__ order,
                                                      const uint32_t* __restrict__ inv, const float2* __restrict__ nd,
                                                      int S, int smooth, float rho0, float occ, float l_rho, float l_sm,
                                                      float2* __restrict__ gg, double* loss, double* trace, int iter,
                                                      float* vt_out, double* terms)
{
    __shared__ double part[3][32];
    double av = 0.0, ar = 0.0, as = 0.0;
    const float inv2 = 2.f / (float)S;
    const int P = smooth ? 2 * S : S;
    for (int s = threadIdx.x; s < P; s += blockDim.x) {
        const uint32_t o = order[s];
        if ((int)o >= S) continue;  // a partner: its sample writes it
        const float4 q = spts[s];
        const float2 v = nd[s];
        const float dd = fmaxf(v.y, rho0);
        const float vt = v.x / dd;
        const bool occd = q.w > occ;
        const float r = occd ? vt - q.w : 0.f;
        av += (double)r * (double)r;
        const float gn = inv2 * r / dd;
        float gd = v.y >= rho0 ? -vt * gn : 0.f;
        if (occd) {
            const float e = v.y - 1.f;
            ar += (double)e * (double)e;
            gd += l_rho * inv2 * e;
        }
        if (smooth) {
            const uint32_t pp = inv[o + S];
            const float e = v.y - nd[pp].y;
            as += (double)e * (double)e;
            gd += l_sm * inv2 * e;
            gg[pp] = make_float2(0.f, -l_sm * inv2 * e);
        }
        gg[s] = make_float2(gn, gd);
        if (vt_out) vt_out[o] = vt;
    }
    for (int o = 16; o > 0; o >>= 1) {
        av += __shfl_xor_sync(0xffffffffu, av, o);
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        as += __shfl_xor_sync(0xffffffffu, as, o);
    }
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = av;
        part[1][threadIdx.x >> 5] = ar;
        part[2][threadIdx.x >> 5] = as;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 3; ++k) t[k] += part[k][w];
        for (int k = 0; k < 3; ++k) t[k] /= (double)S;
        const double tot = t[0] + (double)l_rho * t[1] + (double)l_sm * t[2];
        if (loss) *loss = tot;
        if (trace) trace[iter] = tot;
        if (terms) {
            terms[0] = t[0]; terms[1] = t[1]; terms[2] = t[2];
            terms[3] = terms[4] = terms[5] = 0.0;
        }
    }
}

#define SMP_TRY(x)                               \
    do {                                         \
        gve_status st_ = (x);                    \
        if (st_ != GVE_OK) return st_;           \
    } while (0)
#define SMP_CUDA(x, what)                                     \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

struct SampleBufs {
    CellGrid cg;
    long long ncells;
    float4* pts;     // drawn (or caller's) points, then their partners
    float4* spts;    // sorted by cell
    uint32_t* order;
    uint32_t* inv;
    uint32_t* cstart;
    uint32_t* ccnt;
    float2* nd;
    float2* gg;
    double* loss;
    double* terms;
    float* extra;
    int4* cand;
};

// buffers for P points (samples and partners) and n records
gve_status sample_bufs(gve_ctx* c, gve_dims d, long long P, long long n, SampleBufs& b, cudaStream_t s)
{
    b.cg = make_cells(d);
    b.ncells = (long long)b.cg.ncx * b.cg.ncy * b.cg.ncz;
    const long long nn = n > 0 ? n : 1;
    SMP_TRY(ensure(c, c->s_pts, sizeof(float4) * 2 * P, s));
    SMP_TRY(ensure(c, c->s_order, sizeof(uint32_t) * P, s));
    SMP_TRY(ensure(c, c->s_inv, sizeof(uint32_t) * P, s));
    SMP_TRY(ensure(c, c->s_cell, sizeof(uint32_t) * (b.ncells + 1), s));
    SMP_TRY(ensure(c, c->s_ccnt, sizeof(uint32_t) * b.ncells, s));
    SMP_CUDA(cudaMemsetAsync(c->s_ccnt.p, 0, sizeof(uint32_t) * b.ncells, s), "memset cell counts");
    SMP_TRY(ensure(c, c->s_nd, sizeof(float2) * P, s));
    SMP_TRY(ensure(c, c->s_gg, sizeof(float2) * P, s));
    SMP_TRY(ensure(c, c->s_loss, sizeof(double), s));
    SMP_TRY(ensure(c, c->s_terms, sizeof(double) * 8, s));
    SMP_TRY(ensure(c, c->rec, sizeof(float4) * 3 * nn, s));
    SMP_TRY(ensure(c, c->binrec, sizeof(BinRec) * nn, s));
    SMP_TRY(ensure(c, c->acc, sizeof(float) * 12 * nn, s));
    SMP_TRY(ensure(c, c->s_ex, sizeof(float) * 12 * nn, s));
    SMP_TRY(ensure(c, c->s_cand, sizeof(int4) * (1 + 2 * nn), s));
    b.pts = (float4*)c->s_pts.p;
    b.spts = b.pts + P;
    b.order = (uint32_t*)c->s_order.p;
    b.inv = (uint32_t*)c->s_inv.p;
    b.cstart = (uint32_t*)c->s_cell.p;
    b.ccnt = (uint32_t*)c->s_ccnt.p;
    b.nd = (float2*)c->s_nd.p;
    b.gg = (float2*)c->s_gg.p;
    b.loss = (double*)c->s_loss.p;
    b.terms = (double*)c->s_terms.p;
    b.extra = (float*)c->s_ex.p;
    b.cand = (int4*)c->s_cand.p;
    return GVE_OK;
}

// weights of the point terms of one iteration
struct PointReg {
    float l_rho = 0.f, l_sm = 0.f;
    int smooth = 0;
};

// cells, forward and loss at the S samples (and, with pr.smooth, their S
// partners) in b.pts, the records prepared in c->rec; with `backward` the
// Gaussians' sums are written to c->acc
gve_status sample_pass(gve_ctx* c, const float* prims, long long n, gve_dims d, const gve_eval_opts* o, long long S,
                       const PointReg& pr, const SampleBufs& b, float occ, double* trace, int iter, float* vt_out,
                       bool backward, cudaStream_t s)
{
    const long long P = pr.smooth ? 2 * S : S;
    const unsigned pb = (unsigned)((P + 255) / 256);
    k_cell_count<<<pb, 256, 0, s>>>(b.pts, (int)P, d.nx, d.ny, d.nz, b.cg, b.ccnt);
    k_cell_scan<<<1, kScanThreads, 0, s>>>(b.ccnt, b.ncells, b.cstart);
    k_cell_scatter<<<pb, 256, 0, s>>>(b.pts, (int)P, d.nx, d.ny, d.nz, b.cg, b.cstart, b.ccnt, b.spts, b.order, b.inv);
    SMP_CUDA(cudaMemsetAsync(b.nd, 0, sizeof(float2) * P, s), "memset sums");
    SampleArgs a{};
    a.prims = prims;
    a.rec = (float4*)c->rec.p;
    a.n = n;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz;
    a.cg = b.cg;
    a.cstart = b.cstart;
    a.S = (int)P;
    a.spts = b.spts;
    a.nd = b.nd;
    a.gg = b.gg;
    a.acc = (float*)c->acc.p;
    a.k = o->trunc_k;
    a.T = (float)((double)o->trunc_k * (double)o->trunc_k * kNegHalfLog2e);
    const unsigned grid = (unsigned)((n + 127) / 128);
    if (backward && n > 0) {
        a.cand = b.cand;
        SMP_CUDA(cudaMemsetAsync(b.cand, 0, sizeof(int4), s), "memset candidate count");
        SMP_CUDA(cudaMemsetAsync(a.acc, 0, sizeof(float) * 12 * n, s), "memset sums");
    }
    if (n > 0) k_sample_eval<<<grid, 128, 0, s>>>(a);
    k_sample_loss<<<1, 1024, 0, s>>>(b.spts, b.order, b.inv, b.nd, (int)S, pr.smooth, o->rho0, occ, pr.l_rho, pr.l_sm,
                                     b.gg, b.loss, trace, iter, vt_out, b.terms);
    if (backward && n > 0) k_sample_grad<<<grid, 128, 0, s>>>(a);
    c->launches += 4 + (n > 0 ? 2 + (backward ? 1 : 0) : 0);
    SMP_CUDA(cudaGetLastError(), "launch (sampled pass)");
    return GVE_OK;
}

// the options of the full objective, checked; per-Gaussian weights and
// their logarithmic bounds
gve_status check_reg(gve_ctx* c, const gve_reg_opts* r, gve_dims d, const float* field, RegTerms& rt, bool& per_g)
{
    per_g = false;
    rt = RegTerms{0.f, 0.f, 0.f, 0.0, 0.0, 0.0};
    if (!r) return GVE_OK;
    const float w[6] = {r->lambda_rho, r->lambda_sm, r->lambda_sm_end, r->lambda_anc, r->lambda_aniso, r->lambda_cap};
    for (float x : w)
        if (!(x >= 0.f) || !std::isfinite(x)) return fail(c, GVE_E_INVALID, "regulariser weights must be finite and >= 0");
    if (r->anneal_iters < 0) return fail(c, GVE_E_INVALID, "negative annealing length");
    if (r->lambda_sm > 0.f && (!(r->partner_radius > 0.f) || !std::isfinite(r->partner_radius)))
        return fail(c, GVE_E_INVALID, "partner radius must be positive");
    if (!(r->aniso_max >= 1.f) || !std::isfinite(r->aniso_max)) return fail(c, GVE_E_INVALID, "aniso_max must be >= 1");
    const int mx = d.nx > d.ny ? (d.nx > d.nz ? d.nx : d.nz) : (d.ny > d.nz ? d.ny : d.nz);
    const double s_hi = r->s_hi > 0.f ? (double)r->s_hi : (double)mx / 16.0;
    if (!(r->s_lo > 0.f) || !((double)r->s_lo < s_hi)) return fail(c, GVE_E_INVALID, "need 0 < s_lo < s_hi");
    if (r->lambda_anc > 0.f && !field) return fail(c, GVE_E_INVALID, "the anchor term needs the field");
    rt.l_anc = r->lambda_anc;
    rt.l_aniso = r->lambda_aniso;
    rt.l_cap = r->lambda_cap;
    rt.ln_r = std::log((double)r->aniso_max);
    rt.ln_lo = std::log((double)r->s_lo);
    rt.ln_hi = std::log(s_hi);
    per_g = true;  // the unweighted terms are reported even where a weight is zero
    return GVE_OK;
}

// lambda_sm of iteration t: geometric decay to lambda_sm_end over
// anneal_iters iterations, then lambda_sm_end
double lambda_sm_at(const gve_reg_opts* r, int t)
{
    if (!r) return 0.0;
    const double l0 = r->lambda_sm, l1 = r->lambda_sm_end;
    const int A = r->anneal_iters;
    if (A <= 0 || !(l1 > 0.0) || !(l0 > 0.0)) return l0;
    const double f = t < A ? (double)t / (double)A : 1.0;
    return l0 * std::pow(l1 / l0, f);
}

// class lists of the field, then the split of S
gve_status sample_setup(gve_ctx* c, const float* field, gve_dims d, long long S, long long split[2], cudaStream_t s)
{
    SMP_TRY(sample_classes(c, field, d, s));
    split[0] = (long long)std::floor(0.35 * (double)S + 0.5);
    split[1] = (long long)std::floor(0.40 * (double)S + 0.5);
    return GVE_OK;
}

gve_status check_samples(gve_ctx* c, int64_t S, const gve_eval_opts* o, bool smooth = false)
{
    if (S < 1 || S > kMaxSamples) return fail(c, GVE_E_INVALID, "samples per iteration must be in [1, 8192]");
    if (smooth && 2 * S > kMaxSamples)
        return fail(c, GVE_E_INVALID, "with smoothness partners, samples per iteration must be in [1, 4096]");
    if (!o->normalized) return fail(c, GVE_E_INVALID, "sampled refinement evaluates Eq. 3 (normalized = 1)");
    return GVE_OK;
}

// full-grid SSE of the current records (the voxel path's loss pass)
gve_status full_grid_sse(gve_ctx* c, const float* prims, int64_t n, const float* field, gve_dims d,
                         const gve_eval_opts* o, void* stream, double* sse)
{
    Call k;
    SMP_TRY(begin(c, k, n, d, o, stream));
    SMP_TRY(size_pairs(k, prims, o));
    const double inv_m = 1.0 / ((double)d.nx * d.ny * d.nz);
    for (int attempt = 0; attempt < 4; ++attempt) {
        SMP_TRY(bin_all(k, prims, o, 0));
        BrickArgs a = brick_args(k, o);
        a.field = field;
        a.mask_thresh = -1.f;
        a.acc = nullptr;
        launch_brick(kModeLoss, a, k.s);
        launch_sse_reduce(a.part, k.g.nbricks, dstate(c), nullptr, 0, inv_m, k.s);
        DevState h;
        SMP_TRY(read_state(k, &h));
        if (!h.overflow) {
            *sse = h.sse[1];
            return GVE_OK;
        }
        SMP_TRY(grow_pairs(k, h.max_total1, h.max_total));
        reset_state(k);
    }
    return fail(c, GVE_E_CAPACITY, "final evaluation overflowed");
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_draw_samples(gve_ctx* c, const float* field, gve_dims d, int64_t S, uint64_t seed,
                                       uint32_t iter, float* pts_out, int64_t* vox_out, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!field || !pts_out) return fail(c, GVE_E_INVALID, "null argument");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (S < 1 || S > kMaxSamples) return fail(c, GVE_E_INVALID, "samples per iteration must be in [1, 8192]");
    if (reinterpret_cast<uintptr_t>(pts_out) & 15u) return fail(c, GVE_E_INVALID, "points not 16-byte aligned");
    SMP_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    long long split[2];
    SMP_TRY(sample_setup(c, field, d, S, split, s));
    launch_draw_samples(field, d, (const uint32_t*)c->s_hi.p, c->s_nh, (const uint32_t*)c->s_mid.p, c->s_nm, S,
                        split[0], split[1], seed, iter, reinterpret_cast<float4*>(pts_out),
                        reinterpret_cast<long long*>(vox_out), s);
    SMP_CUDA(cudaGetLastError(), "launch (draw)");
    return GVE_OK;
}

extern "C" gve_status gve_draw_partners(gve_ctx* c, const float* pts, int64_t S, gve_dims d, uint64_t seed,
                                        uint32_t iter, float radius, float* out, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!pts || !out) return fail(c, GVE_E_INVALID, "null argument");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (S < 1 || S > kMaxSamples) return fail(c, GVE_E_INVALID, "samples per iteration must be in [1, 8192]");
    if (!(radius > 0.f) || !std::isfinite(radius)) return fail(c, GVE_E_INVALID, "partner radius must be positive");
    if ((reinterpret_cast<uintptr_t>(pts) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u))
        return fail(c, GVE_E_INVALID, "points must be 16-byte aligned");
    SMP_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    c->launches = 1;
    launch_draw_partners(reinterpret_cast<const float4*>(pts), S, d, seed, iter, radius, reinterpret_cast<float4*>(out),
                         (cudaStream_t)stream);
    SMP_CUDA(cudaGetLastError(), "launch (partners)");
    return GVE_OK;
}

extern "C" gve_status gve_sample_loss_grad(gve_ctx* c, const float* prims, int64_t n, gve_dims d,
                                           const gve_eval_opts* o, const float* pts, int64_t S, float occ_thresh,
                                           const gve_reg_opts* reg, const float* field, float* grad_out,
                                           double* loss_dev, double* terms_dev, float* vt_out, void* stream)
{
    SMP_TRY(check_common(c, prims, n, d, o));
    PointReg pr;
    pr.l_rho = reg ? reg->lambda_rho : 0.f;
    pr.l_sm = reg ? reg->lambda_sm : 0.f;
    pr.smooth = pr.l_sm > 0.f;
    SMP_TRY(check_samples(c, S, o, pr.smooth != 0));
    RegTerms rt;
    bool per_g = false;
    SMP_TRY(check_reg(c, reg, d, field, rt, per_g));
    if (!pts) return fail(c, GVE_E_INVALID, "null points");
    if ((reinterpret_cast<uintptr_t>(pts) & 15u) || (grad_out && (reinterpret_cast<uintptr_t>(grad_out) & 15u)))
        return fail(c, GVE_E_INVALID, "points and gradient must be 16-byte aligned");
    SMP_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    const long long P = pr.smooth ? 2 * S : S;
    SampleBufs b;
    SMP_TRY(sample_bufs(c, d, P, n, b, s));
    SMP_CUDA(cudaMemcpyAsync(b.pts, pts, sizeof(float4) * P, cudaMemcpyDeviceToDevice, s), "copy points");
    SMP_TRY(sample_pass(c, prims, n, d, o, S, pr, b, occ_thresh, nullptr, 0, vt_out, grad_out != nullptr, s));
    if (per_g) {
        launch_reg(prims, n, field, d, rt, b.extra, b.terms, nullptr, b.loss, s);
        c->launches += 1;
    }
    if (loss_dev) SMP_CUDA(cudaMemcpyAsync(loss_dev, b.loss, sizeof(double), cudaMemcpyDeviceToDevice, s), "copy loss");
    if (terms_dev)
        SMP_CUDA(cudaMemcpyAsync(terms_dev, b.terms, sizeof(double) * 6, cudaMemcpyDeviceToDevice, s), "copy terms");
    if (grad_out && n > 0) {
        launch_chain((float*)c->acc.p, nullptr, const_cast<float*>(prims), n, grad_out, nullptr, nullptr, nullptr,
                     nullptr, s, per_g ? b.extra : nullptr);
        c->launches += 1;
    }
    SMP_CUDA(cudaGetLastError(), "launch (sampled gradient)");
    return GVE_OK;
}

extern "C" gve_status gve_refine_sampled(gve_ctx* c, float* prims, int64_t n, const float* field, gve_dims d,
                                         const gve_schedule* sc, int64_t S, uint64_t seed, const gve_reg_opts* reg,
                                         float* adam_state, double* trace, gve_stats* stats, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!sc) return fail(c, GVE_E_INVALID, "null schedule");
    SMP_TRY(check_common(c, prims, n, d, &sc->eval));
    const bool smooth = reg && reg->lambda_sm > 0.f;
    SMP_TRY(check_samples(c, S, &sc->eval, smooth));
    RegTerms rt;
    bool per_g = false;
    SMP_TRY(check_reg(c, reg, d, field, rt, per_g));
    if (!field) return fail(c, GVE_E_INVALID, "null target field");
    if (sc->iters < 0 || sc->step0 < 0) return fail(c, GVE_E_INVALID, "negative iteration count");
    if (!(sc->lr >= 0.f) || !(sc->beta1 >= 0.f && sc->beta1 < 1.f) || !(sc->beta2 >= 0.f && sc->beta2 < 1.f) ||
        !(sc->eps >= 0.f))
        return fail(c, GVE_E_INVALID, "bad Adam hyper-parameters");
    if (adam_state && (reinterpret_cast<uintptr_t>(adam_state) & 15u))
        return fail(c, GVE_E_INVALID, "adam state not 16-byte aligned");
    SMP_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    const gve_eval_opts* o = &sc->eval;
    const float occ = sc->mask_thresh >= 0.f ? sc->mask_thresh : 0.02f;
    long long split[2];
    SMP_TRY(sample_setup(c, field, d, S, split, s));
    SampleBufs b;
    SMP_TRY(sample_bufs(c, d, smooth ? 2 * S : S, n, b, s));
    const long long nn = n > 0 ? n : 1;
    float* m = adam_state;
    if (!m) {
        SMP_TRY(ensure(c, c->adam, sizeof(float) * 24 * nn, s));
        m = (float*)c->adam.p;
        SMP_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * 24 * nn, s), "memset adam");
    }
    float* v = adam_state ? adam_state + 12 * n : m + 12 * nn;
    SMP_TRY(ensure(c, c->state, sizeof(DevState), s));
    // stage events (with stats): before the preparation, before the draw,
    // before the chain rule; read back every 64 iterations
    const bool timed = stats != nullptr;
    if (timed && !c->sev_ready) {
        for (int q = 0; q < 3; ++q)
            for (int r = 0; r < 64; ++r) SMP_CUDA(cudaEventCreate(&c->sev[q][r]), "event create");
        c->sev_ready = true;
    }
    double ms_prep = 0.0, ms_search = 0.0;
    SMP_CUDA(cudaEventRecord(c->ev0, s), "event");
    for (int it0 = 0; it0 < sc->iters; it0 += 64) {
        const int end = it0 + 64 < sc->iters ? it0 + 64 : sc->iters;
        for (int it = it0; it < end; ++it) {
            const int step = sc->step0 + it;
            if (timed) SMP_CUDA(cudaEventRecord(c->sev[0][it - it0], s), "event");
            if (timed) SMP_CUDA(cudaEventRecord(c->sev[1][it - it0], s), "event");
            launch_draw_samples(field, d, (const uint32_t*)c->s_hi.p, c->s_nh, (const uint32_t*)c->s_mid.p, c->s_nm,
                                S, split[0], split[1], seed, (uint32_t)step, b.pts, nullptr, s);
            PointReg pr;
            if (reg) {
                pr.l_rho = reg->lambda_rho;
                pr.l_sm = (float)lambda_sm_at(reg, step);
                pr.smooth = smooth ? 1 : 0;
            }
            if (smooth) {
                launch_draw_partners(b.pts, S, d, seed, (uint32_t)step, reg->partner_radius, b.pts + S, s);
                c->launches += 1;
            }
            SMP_TRY(sample_pass(c, prims, n, d, o, S, pr, b, occ, trace, it, nullptr, true, s));
            if (per_g) {
                launch_reg(prims, n, field, d, rt, b.extra, b.terms, trace ? trace + it : nullptr, b.loss, s);
                c->launches += 1;
            }
            if (timed) SMP_CUDA(cudaEventRecord(c->sev[2][it - it0], s), "event");
            if (n > 0) {
                AdamArgs ad{};
                ad.lr = sc->lr; ad.b1 = sc->beta1; ad.b2 = sc->beta2; ad.eps = sc->eps;
                ad.bc1 = (float)(1.0 - std::pow((double)sc->beta1, step + 1));
                ad.bc2 = (float)(1.0 - std::pow((double)sc->beta2, step + 1));
                // the sums are cleared by the next pass's memset, not here
                launch_chain((float*)c->acc.p, nullptr, prims, n, nullptr, m, v, &ad, nullptr, s,
                             per_g ? b.extra : nullptr);
                c->launches += 1;
            }
            c->launches += 1;
        }
        if (timed) {
            SMP_CUDA(cudaEventSynchronize(c->sev[2][end - 1 - it0]), "sync");
            for (int it = it0; it < end; ++it) {
                float x = 0.f, y = 0.f;
                cudaEventElapsedTime(&x, c->sev[0][it - it0], c->sev[1][it - it0]);
                cudaEventElapsedTime(&y, c->sev[1][it - it0], c->sev[2][it - it0]);
                ms_prep += x;
                ms_search += y;
            }
        }
    }
    SMP_CUDA(cudaEventRecord(c->ev1, s), "event");
    SMP_CUDA(cudaGetLastError(), "launch (sampled refine)");
    if (stats) {
        float ms_loop = 0.f;
        SMP_CUDA(cudaEventSynchronize(c->ev1), "sync");
        cudaEventElapsedTime(&ms_loop, c->ev0, c->ev1);
        const long long launches = c->launches;
        double first = 0.0, last = 0.0;
        if (trace && sc->iters > 0) {
            SMP_CUDA(cudaMemcpy(&first, trace, sizeof(double), cudaMemcpyDeviceToHost), "trace");
            SMP_CUDA(cudaMemcpy(&last, trace + sc->iters - 1, sizeof(double), cudaMemcpyDeviceToHost), "trace");
        }
        double sse = 0.0;
        SMP_TRY(full_grid_sse(c, prims, n, field, d, o, stream, &sse));
        const double M = (double)d.nx * d.ny * d.nz;
        stats->loss_first = first;
        stats->loss_last = last;
        stats->sse_final = sse;
        stats->psnr_final = sse > 0.0 ? 10.0 * std::log10(M / sse) : INFINITY;
        stats->brick_pairs = 0;
        stats->iters_done = sc->iters;
        stats->retries = 0;
        stats->ms_total = ms_loop;
        stats->ms_brick = (float)ms_search;
        stats->ms_bin = (float)ms_prep;
        stats->ms_fwd = 0.f;
        stats->launches = launches + c->launches;
    }
    return GVE_OK;
}
