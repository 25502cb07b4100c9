// gve_int.cuh -- internal declarations of libgve (sm_103a).
//
// Data layout in HBM (per context):
//   prepped record  3 x float4 per Gaussian:
//       r0 = (mu_x, mu_y, mu_z, qxx)      r1 = (qyy, qzz, qxy2, qxz2)
//       r2 = (qyz2, alpha = w a, beta = w, a)
//     q.. = float32(-0.5 log2(e) Sigma^-1) entries (off-diagonals doubled),
//     from one fixed sequence of correctly rounded float32 operations
//     (keep_coefficients below).
//   bin record      20 words per Gaussian: whitening L (row-major 3x3),
//                   brick half-extent bound e[3], threshold K2, brick box
//                   lo[3] / hi[3], non-empty flag.
//   tile pairs      (tile key, Gaussian index) uint32 pairs, double-buffered
//                   for the radix sort, and a 64-bit brick pass mask per
//                   sorted pair (tile = kTile^3 bricks).
//   brick pairs     uint32 per pair, sorted by brick key then Gaussian index:
//                   Gaussian index in the low 24 bits, 8-bit sub-brick mask
//                   above.
//   ranges          uint32 start[nbricks], end[nbricks].
//   accumulators    float[12] per Gaussian: A = sum G gn, H = sum h, S1' (3),
//                   S2' (6: xx yy zz xy xz yz), 0 -- the per-Gaussian sums of
//                   the backward, h = G (a gn + gd).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/gve.h"

namespace gve {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanBlocks = 512;
constexpr int kScanThreads = 1024;
constexpr double kNegHalfLog2e = -0.72134752044448170367996234050095;
// sorted pair values: Gaussian index in the low 24 bits, sub-brick mask above
constexpr int kGidBits = 24;
constexpr uint32_t kGidMask = (1u << kGidBits) - 1u;
// bricks per tile edge of the two-level binning (64 bricks: one 64-bit mask)
constexpr int kTile = 4;

struct __align__(16) BinRec {
    float L[9];
    float e[3];
    float K2;
    int blo[3];
    int bhi[3];
    int nonempty;
};
static_assert(sizeof(BinRec) == 80, "bin record is 20 words");

// Device-side state of one call: pair totals and the sticky overflow flag.
struct DevState {
    unsigned long long total;        // brick pairs of the current binning
    unsigned long long max_total;    // largest total seen since reset
    unsigned long long total1;       // tile pairs of the current binning
    unsigned long long max_total1;   // largest total1 seen since reset
    int overflow;                    // sticky: an iteration needed more than cap pairs
    int first_overflow_iter;         // first iteration that overflowed
    int err;                         // internal consistency error
    int pad;
    double sse[2];                   // {masked, unmasked} SSE of the last reduction
    unsigned long long kept;         // kept (voxel, Gaussian) pairs (counting mode)
    unsigned long long cand;         // candidate pairs visited (counting mode)
    unsigned long long listed;       // kept pairs offered to the pair list (counting mode)
};

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace gve

struct gve_ctx {
    int device = 0;
    std::string err;
    gve::Buf rec, binrec, counts, offsets, acc, adam;
    gve::Buf keys[2], vals[2];       // tile pairs (radix double buffer)
    gve::Buf tmask, trange;          // brick pass mask per sorted tile pair; per-tile ranges
    gve::Buf cbase;                  // per chunk of 32 tile-list entries: earlier passes per brick
    uint64_t cap1 = 0;               // tile-pair capacity
    gve::Buf bcount, boff;           // per-brick pair counts and their exclusive scan
    gve::Buf pairs;                  // brick pairs in brick order
    uint64_t cap = 0;                // brick-pair capacity
    gve::Buf hist, scanp;
    gve::Buf ranges, part;
    gve::Buf state;
    gve::DevState* hstate = nullptr; // pinned host mirror
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // allocator scratch
    gve::Buf a_g, a_keys, a_sel, a_tmp, a_cnt;
    gve::Buf trace;                  // loss trace when the caller passes none
    // per-iteration stage events of one refine segment: before binning,
    // before the brick evaluator, after it
    cudaEvent_t sev[3][64] = {};
    bool sev_ready = false;
    long long launches = 0;          // kernels launched by the current call
    // batched allocation: one worker context, stream and join event per
    // concurrent allocation
    std::vector<gve_ctx*> asub;
    std::vector<cudaStream_t> astream;
    std::vector<cudaEvent_t> ajoin;
    // batched refinement: its stream and the event that joins it to the caller's
    cudaStream_t gstream = nullptr;
    cudaEvent_t fork = nullptr;
    gve::Buf bstate;                 // batch device state (BatchState)
    gve::Buf btab;                   // batch: per-volume {masked, unmasked} SSE of the last iteration
    gve::Buf csum;                   // batch: per-chunk partial sums of the loss
    // stratified-sample refinement: class lists, per-block counts and
    // offsets, samples, cell table, sorted sample order, per-sample sums and
    // upstream gradients, loss
    gve::Buf s_hi, s_mid, s_cnt, s_off, s_pts, s_cell, s_order, s_nd, s_gg, s_loss;
    gve::Buf s_inv, s_ex, s_terms;   // sorted position of each point, regulariser gradient, loss terms
    gve::Buf s_ccnt;                 // points per cell (the counting sort's counters)
    gve::Buf s_cand;                 // Gaussians with candidate points: count, then (index, cell box) pairs
    unsigned long long s_nh = 0, s_nm = 0;
    // ray marcher: keep coefficients, per-Gaussian cell counts and offsets,
    // (cell, Gaussian) pairs and their sort buffers, per-cell ranges, the
    // coefficients in cell order, device state
    gve::Buf r_rec, r_cnt, r_off, r_keys[2], r_vals[2], r_hist, r_scanp, r_rng, r_crec, r_state;
    int r_dims[3] = {0, 0, 0}, r_nc[3] = {0, 0, 0};
    float r_T = 0.f, r_rho0 = 0.f;
    int r_norm = 1;
    bool r_ready = false;
    unsigned long long r_pairs = 0;
};

namespace gve {

// ---- device helpers ------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The keep exponent t at a float32 offset d = p - mu from the prepared
// coefficients r0 = (mu, qxx), r1 = (qyy, qzz, qxy2, qxz2), r2 = (qyz2, ...):
// the voxel path's fixed chain (kept iff t > T).
__device__ __forceinline__ float keep_t(const float4& r0, const float4& r1, const float4& r2, float dx, float dy,
                                        float dz)
{
    const float b = __fmaf_rn(r1.z, dy, __fmul_rn(r1.w, dz));
    const float c = __fmaf_rn(dy, __fmaf_rn(r1.x, dy, __fmul_rn(r2.x, dz)), __fmul_rn(dz, __fmul_rn(r1.y, dz)));
    return __fmaf_rn(dx, __fmaf_rn(r0.w, dx, b), c);
}

// Conservative truncation box of raw record i (12 floats): centre mu and per
// axis half extent rad = kb sqrt(Sigma_jj) 1.0001 + 0.05 voxel with kb =
// k (1.001 + 1e-5 cond), cond = (s_max / s_min)^2, in float32; the margins
// cover the float32 rounding of the keep chain at any float32 point.
// Returns 0 for a record the preparation marks invalid (non-finite values,
// zero quaternion), 2 for scales beyond float range (the whole grid), else 1.
__device__ __forceinline__ int gauss_box(const float* prims, long long i, float k, float mu[3], float rad[3],
                                         float* kb_out = nullptr, float* cinv_out = nullptr)
{
    const float4* p4 = reinterpret_cast<const float4*>(prims) + 3 * i;
    const float4 p0 = p4[0], p1 = p4[1], p2 = p4[2];
    const float p[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 12; ++j) ok = ok && isfinite(p[j]);
    const float nq = sqrtf(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
    if (!ok || !(nq > 0.f) || !isfinite(nq)) return 0;
    const float qw = p[6] / nq, qx = p[7] / nq, qy = p[8] / nq, qz = p[9] / nq;
    const float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                           {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                           {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    float s[3];
    bool huge = false;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        s[j] = expf(p[3 + j]);
        huge = huge || !isfinite(s[j]);
        mu[j] = p[j];
    }
    if (huge) return 2;
    const float smax = fmaxf(s[0], fmaxf(s[1], s[2])), smin = fminf(s[0], fminf(s[1], s[2]));
    const float ratio = smin > 0.f ? smax / smin : 1e30f;
    const float kb = k * (1.001f + 1e-5f * fminf(ratio * ratio, 1e30f));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float var = R[j][0] * R[j][0] * s[0] * s[0] + R[j][1] * R[j][1] * s[1] * s[1] + R[j][2] * R[j][2] * s[2] * s[2];
        rad[j] = kb * sqrtf(var) * 1.0001f + 0.05f;
    }
    if (kb_out) *kb_out = kb;
    if (cinv_out) {  // Sigma^-1 = R diag(s^-2) R^T: xx, yy, zz, xy, xz, yz
        const float is[3] = {1.f / (s[0] * s[0]), 1.f / (s[1] * s[1]), 1.f / (s[2] * s[2])};
        const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int x = ab[q][0], y = ab[q][1];
            cinv_out[q] = R[x][0] * R[y][0] * is[0] + R[x][1] * R[y][1] * is[1] + R[x][2] * R[y][2] * is[2];
        }
    }
    return 1;
}

// FP64 with explicit rounding (no contraction whatever the compiler flags)
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }

// e^x in float32 by a fixed sequence of correctly rounded operations (the
// CPU reference runs the same sequence, so both agree bit for bit):
// Cody-Waite reduction x = n ln2 + r with ln2 split into a 16-bit head and a
// tail, a degree-7 Taylor polynomial of e^r in Horner form with fused
// multiply-adds, and the exact scaling by 2^n.  Relative error below 2^-22.
__device__ __forceinline__ float exp_fixed(float x)
{
    if (x != x) return x;
    if (x > 88.75f) return INFINITY;
    if (x < -103.5f) return 0.0f;
    const float n = rintf(__fmul_rn(x, 1.44269504f));
    float r = __fmaf_rn(-n, 0.693145751953125f, x);
    r = __fmaf_rn(-n, 1.42860677e-06f, r);
    float p = 1.98412698e-04f;
    p = __fmaf_rn(p, r, 1.38888889e-03f);
    p = __fmaf_rn(p, r, 8.33333333e-03f);
    p = __fmaf_rn(p, r, 4.16666667e-02f);
    p = __fmaf_rn(p, r, 1.66666667e-01f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    return ldexpf(p, (int)n);
}

// Keep-test coefficients of one raw record: the Eq. 2 activations and
// -log2(e)/2 Sigma^-1 = -log2(e)/2 R diag(s^-2) R^T in float32, one fixed
// sequence of correctly rounded operations (explicit intrinsics: no
// contraction whatever the file's flags), the scales by exp_fixed:
// r0 = (mu, qxx), r1 = (qyy, qzz, 2 qxy, 2 qxz), r2 = (2 qyz, w a, w, a);
// zero records when the record is invalid (non-finite values, zero
// quaternion or scale).
struct KeepCoef {
    float4 r0, r1, r2;
    float s[3];        // float32 scales exp_fixed(log s)
    float R[3][3];     // rotation of the normalised quaternion
    bool ok;
};

__device__ __forceinline__ void keep_coefficients(const float (&pf)[12], KeepCoef& o)
{
    o.r0 = o.r1 = o.r2 = make_float4(0.f, 0.f, 0.f, 0.f);
    o.ok = false;
    bool ok = true;
    for (int j = 0; j < 12; ++j) ok = ok && isfinite(pf[j]);
    if (!ok) return;
    float s[3];
    for (int j = 0; j < 3; ++j) s[j] = exp_fixed(pf[3 + j]);
    const float qw = pf[6], qx = pf[7], qy = pf[8], qz = pf[9];
    const float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(qw, qw), __fmul_rn(qx, qx)), __fmul_rn(qy, qy)),
                               __fmul_rn(qz, qz));
    const float nq = __fsqrt_rn(n2);
    if (!(nq > 0.0f) || !isfinite(nq)) return;
    for (int j = 0; j < 3; ++j)
        if (!(s[j] > 0.0f) || !isfinite(s[j])) return;
    const float w = __fdiv_rn(qw, nq), x = __fdiv_rn(qx, nq), y = __fdiv_rn(qy, nq), z = __fdiv_rn(qz, nq);
    float(&R)[3][3] = o.R;
    for (int j = 0; j < 3; ++j) o.s[j] = s[j];
    R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(y, y), __fmul_rn(z, z))));
    R[0][1] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    R[0][2] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    R[1][0] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(z, z))));
    R[1][2] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    R[2][0] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    R[2][1] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y))));
    float inv[3];
    for (int j = 0; j < 3; ++j) inv[j] = __fdiv_rn(1.0f, __fmul_rn(s[j], s[j]));
    const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    const float nhl = (float)kNegHalfLog2e;
    float Q[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int a = ab[q][0], b = ab[q][1];
        const float c = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(R[a][0], R[b][0]), inv[0]),
                                            __fmul_rn(__fmul_rn(R[a][1], R[b][1]), inv[1])),
                                  __fmul_rn(__fmul_rn(R[a][2], R[b][2]), inv[2]));
        Q[q] = __fmul_rn(c, nhl);
    }
    const float wd = __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_fixed(-pf[11])));
    o.r0 = make_float4(pf[0], pf[1], pf[2], Q[0]);
    o.r1 = make_float4(Q[1], Q[2], __fmul_rn(2.0f, Q[3]), __fmul_rn(2.0f, Q[4]));
    o.r2 = make_float4(__fmul_rn(2.0f, Q[5]), __fmul_rn(wd, pf[10]), wd, pf[10]);
    o.ok = true;
}

// ---- launchers (bin.cu) --------------------------------------------------
struct BinGeom {
    int nx, ny, nz, B, nbx, nby, nbz;
    long long nbricks;
    int key_bits;
    int ntx, nty, ntz;         // tiles of kTile^3 bricks
    long long ntiles;
    int tkey_bits;
};
BinGeom make_geom(gve_dims d, int B);

// The grids of one binning: one for a single grid, the volumes of a batch
// otherwise (their Gaussians, tiles and bricks numbered consecutively,
// volume by volume).  Passed to the binning kernels by value.
constexpr int kMaxBinVol = 32;
struct VolTab {
    int nvol;
    long long goff[kMaxBinVol + 1];   // first Gaussian of each volume; goff[nvol] = all
    long long toff[kMaxBinVol + 1];   // first tile
    long long boff[kMaxBinVol + 1];   // first brick
    BinGeom g[kMaxBinVol];
};
// a table of one grid with n Gaussians
VolTab single_volume(const BinGeom& g, long long n);
// the volume holding item i of a table column off[0..nvol] (the largest v
// with off[v] <= i)
__host__ __device__ __forceinline__ int vt_find(const long long* off, int nvol, long long i)
{
    int lo = 0, hi = nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the keep coefficients alone (same values as the binning's rec)
void launch_prep_rec(const float* prims, long long n, float k, float4* rec, cudaStream_t s);
// exclusive scan of counts into offsets[0..n]; the total goes to st->total
// (stage 0) or st->total1 (stage 1) and their maxima, and sets st->overflow
// when total > cap (iteration index `iter`).
void launch_offsets(const uint32_t* counts, long long n, unsigned long long* offsets, void* scanp,
                    DevState* st, unsigned long long cap, int iter, cudaStream_t s, int stage = 0);
// exclusive scan of n uint32 into out[0..n] (out[n] = total)
void launch_exscan_u32(const uint32_t* in, long long n, unsigned long long* out, void* scanp, cudaStream_t s);
// Stable LSD radix sort of (keys, vals) by key; the element count is read
// on the device (min(*n_dev, cap)); nothing runs while *stop is set.  The
// result ends in keys[out], vals[out].
int launch_sort(uint32_t* keys[2], uint32_t* vals[2], const unsigned long long* n_dev, const int* stop,
                unsigned long long cap, int key_bits, uint32_t* hist, void* scanp, cudaStream_t s);
void launch_ranges(const uint32_t* skeys, const unsigned long long* n_dev, const int* stop, unsigned long long cap,
                   uint32_t* start, uint32_t* end, cudaStream_t s);

// Scratch of one brick binning (see bin.cu): per Gaussian, per tile pair,
// per tile, per brick and per brick pair.
struct BinBufs {
    float4* rec;                  // [n][3] keep coefficients
    BinRec* br;                   // [n]
    uint32_t* tcount;             // [n] tiles of each Gaussian's brick box
    unsigned long long* toff;     // [n + 1] their exclusive scan
    void* scanp;                  // [kScanBlocks] scan partials
    uint32_t* tkeys[2];           // [cap1] tile keys (radix double buffer)
    uint32_t* tvals[2];           // [cap1] Gaussian indices
    uint32_t* hist;               // radix histograms for cap1 elements
    unsigned long long* tmask;    // [cap1] brick pass mask per sorted tile pair
    uint32_t* cbase;              // [cbase_chunks(cap1, ntiles)][64] per chunk of 32 tile-list
                                  // entries: passes of each brick by the tile's earlier entries
    unsigned long long cap1;
    uint32_t* trange;             // [2][ntiles]
    uint32_t* bcount;             // [nbricks]
    unsigned long long* boff;     // [nbricks + 1]
    uint32_t* ranges;             // [2][nbricks] start, end (0, 0 = empty)
    uint32_t* pairs;              // [cap] brick pairs in brick order
    unsigned long long cap;
    uint32_t* gcount;             // [n] brick pairs per Gaussian, or nullptr
    DevState* st;
};
// chunks of 32 tile-list entries that cap1 tile pairs over ntiles tiles can form
inline unsigned long long cbase_chunks(unsigned long long cap1, long long ntiles)
{
    return cap1 / 32 + (unsigned long long)ntiles + 2;
}
// Issues the whole binning on s without host synchronisation and returns
// the kernels launched.  Tile pairs above cap1 or brick pairs above cap set
// st->overflow (st->first_overflow_iter = iter) and skip the rest.
int launch_binning(const BinBufs& b, const float* prims, long long n, const VolTab& vt, float k, int iter,
                   cudaStream_t s);
// keys[p] = brick of pair p, from the ranges (introspection)
void launch_fill_keys(const uint32_t* ranges, long long nbricks, uint32_t* keys, cudaStream_t s);

// ---- launchers (field.cu) ------------------------------------------------
enum BrickMode { kModeEval = 0, kModeLoss = 1, kModeBwd = 2, kModeCount = 3 };
struct BrickArgs {
    BinGeom g;
    const uint32_t* start;
    const uint32_t* end;
    const uint32_t* gids;
    const float4* rec;
    const float* field;        // target V (loss) or nullptr
    const float* upstream;     // dL/dVtilde (backward mode)
    float* field_out;          // Vtilde (eval mode) or nullptr
    float* acc;                // [n][12] accumulators (loss/bwd)
    float2* part;              // per-brick {masked, unmasked} SSE (float32 within a brick)
    DevState* st;
    float T;                   // float32 keep threshold
    float rho0;
    int normalized;
    float mask_thresh;         // < 0: no mask
    float inv_m;               // 1 / (nx ny nz)
    int chunk;                 // Gaussians staged per chunk: 32 or 64 (0 = 64)
    unsigned long long* pairs;         // counting mode: kept pairs (voxel << 24 | gid), or nullptr
    unsigned long long pairs_cap;      // entries pairs can hold
};
void launch_brick(int mode, const BrickArgs& a, cudaStream_t s);

// deterministic reduction of per-brick partials; writes st->sse and, if
// trace != nullptr, trace[i] = sse_masked * inv_m with i = iter, or
// i = (*iter_dev) * trace_stride + trace_col when iter_dev is set.
void launch_sse_reduce(const float2* part, long long nbricks, DevState* st, double* trace, int iter,
                       double inv_m, cudaStream_t s, const int* iter_dev = nullptr, int trace_stride = 1,
                       int trace_col = 0);

// ---- launchers (optim.cu) ------------------------------------------------
struct AdamArgs {
    float lr, b1, b2, eps;
    float bc1, bc2;         // 1 - beta^t
    const float* bc_dev;    // if set: {bc1, bc2} read on the device (graph replay)
};
// chain rule from accumulators to raw-record gradients; either writes grad
// (grad != nullptr) or applies Adam in place (prims, m, v).  Zeroes acc.
// extra (nullable) [n][12]: a raw-record gradient added before the output or
// the Adam step (the per-Gaussian regularisers)
void launch_chain(const float* acc_in, float* acc_zero, float* prims, long long n, float* grad,
                  float* m, float* v, const AdamArgs* adam, const DevState* st, cudaStream_t s,
                  const float* extra = nullptr);

// ---- the batched persistent iteration (field.cu) ---------------------------
// Device state of one batched refinement call.
struct BatchState {
    int it;                    // iteration index within the call
    int first;                 // first iteration that overflowed, -1 if none
    float bc[2];               // Adam bias corrections of the current step
    unsigned long long next;   // bricks handed out by the work counter
    unsigned bar_count;        // grid barrier: CTAs arrived
    unsigned bar_gen;          // grid barrier: generation
    int err;                   // 1: a bounded wait ran out (GVE_E_TIMEOUT)
    unsigned done;             // CTAs past the chunk sums of the loss (the last one finishes them)
};

constexpr int kMaxBatchVol = 32;
// bricks per chunk of the batched loss reduction
constexpr int kSseChunk = 4096;
// Passed by value (a kernel parameter of about 7 KB): the per-volume tables
// sit in the constant bank, where every thread of a CTA reads the same entry.
struct BatchIterArgs {
    BrickArgs va[kMaxBatchVol];          // evaluator arguments of each volume
    long long boff[kMaxBatchVol + 1];    // first global brick of each volume
    double inv_m[kMaxBatchVol];          // 1 / voxels
    int nvol;
    long long nbricks;         // bricks of all volumes
    long long ntot;            // Gaussians of all volumes (records concatenated)
    BatchState* bs;
    float* acc;                // [ntot][12] sums of the backward, cleared after use
    float* prims;              // [ntot][12]
    float* m;                  // Adam moments [ntot][12] each, or gradient scratch
    float* v;
    float* grad;               // gradient output [ntot][12] when do_adam == 0
    int do_adam;
    AdamArgs ad;
    double* trace;             // [iters][nvol] masked mean squared errors, or nullptr
    double* sse;               // [nvol][2] {masked, unmasked} SSE of this iteration (device)
    double2* csum;             // [nchunks] per chunk of kSseChunk bricks of one volume: its partial sums
    long long coff[kMaxBatchVol + 1];    // first chunk of each volume
    long long nchunks;
    unsigned expect;           // CTAs the grid barrier waits for
    long long spin_limit;      // sleeps of ~128 ns before a wait gives up
};
// The resident grid of the persistent kernel for brick edge B and chunk CH
// (0 when it cannot be launched cooperatively).
int batch_iter_grid(int B, int CH);
// One batched iteration as one cooperative launch: every volume's bricks
// (fused forward + backward, loss mode) from a shared work counter, a bounded
// grid barrier, then each volume's loss and the chain rule + Adam (or the
// gradient) of every Gaussian.
cudaError_t launch_batch_iter(int B, int CH, const BatchIterArgs& p, unsigned grid, cudaStream_t s);

// ---- allocator (alloc.cu) ------------------------------------------------
gve_status allocate(gve_ctx* c, const float* field, gve_dims d, int64_t budget,
                    const gve_alloc_opts* o, float* prims, int64_t* feasible_max,
                    gve_alloc_info* info, cudaStream_t s);

// ---- stratified samples (alloc.cu: classes and draw) -----------------------
// voxel lists of the high (V > 0.4) and occupied mid-range (0.02 < V <= 0.4)
// classes, ascending, into c->s_hi / c->s_mid with sizes c->s_nh / c->s_nm
// (synchronises `s` to read them); the grid must have fewer than 2^32 voxels
gve_status sample_classes(gve_ctx* c, const float* V, gve_dims d, cudaStream_t s);
// sample j of iteration `iter`: (x, y, z, target) into pts[j], voxel into
// vox[j] when vox != nullptr; s_hi / s_mid = samples of the two classes
void launch_draw_samples(const float* V, gve_dims d, const uint32_t* hi, unsigned long long nh, const uint32_t* mid,
                         unsigned long long nm, long long S, long long s_hi, long long s_mid,
                         unsigned long long seed, uint32_t iter, float4* pts, long long* vox, cudaStream_t s);

// ---- full objective: smoothness partners, per-Gaussian terms (alloc.cu) ----
void launch_draw_partners(const float4* pts, long long S, gve_dims d, unsigned long long seed, uint32_t iter,
                          float radius, float4* out, cudaStream_t s);
struct RegTerms {
    float l_anc, l_aniso, l_cap;
    double ln_r, ln_lo, ln_hi;
};
// extra [n][12]: the raw-record gradient of the anchor, anisotropy and cap
// terms (a and log-scales only); terms[3..5] += the unweighted terms;
// total_a / total_b (nullable) += their weighted sum
void launch_reg(const float* prims, long long n, const float* V, gve_dims d, const RegTerms& r, float* extra,
                double* terms, double* total_a, double* total_b, cudaStream_t s);

// ---- pre-encoding structure statistics (alloc.cu) --------------------------
// out = {occupancy, top-10 % gradient-mass share, S(1), S(16), S(1)/S(16)};
// stage_ms (nullable) = {sweep 1, sweep 2 + select, whole pass (ms), kernels
// launched}; synchronises `s`
gve_status structure_stats(gve_ctx* c, const float* V, gve_dims d, double out[5], double* stage_ms,
                           cudaStream_t s);

// ---- context scratch and the evaluation pipeline (api.cu) ----------------
// streaming multiprocessors of the current device (queried once per device;
// grids of persistent and grid-stride kernels are sized from it)
int num_sms();
gve_status ensure(gve_ctx* c, Buf& b, size_t bytes, cudaStream_t s);
gve_status cuda_fail(gve_ctx* c, cudaError_t e, const char* what);
gve_status fail(gve_ctx* c, gve_status s, const char* msg);

// one call of the pipeline on one grid
struct Call {
    gve_ctx* c;
    cudaStream_t s;
    BinGeom g;
    long long n;
    VolTab vt;   // the grids the binning covers (the one grid g, or a batch's volumes)
};
DevState* dstate(gve_ctx* c);
gve_status check_common(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o);
gve_status begin(gve_ctx* c, Call& k, int64_t n, gve_dims d, const gve_eval_opts* o, void* stream);
gve_status reset_state(Call& k);
gve_status read_state(Call& k, DevState* out);
// grows the tile-pair (need1) and brick-pair (need2) buffers
gve_status grow_pairs(Call& k, unsigned long long need1, unsigned long long need2);
// per-Gaussian/per-tile/per-brick scratch for k.vt + sizing pass (synchronises k.s)
gve_status size_pairs(Call& k, const float* prims, const gve_eval_opts* o);
// the whole binning (stream-ordered, no host sync); gcount (nullable):
// brick pairs per Gaussian
gve_status bin_all(Call& k, const float* prims, const gve_eval_opts* o, int iter, uint32_t* gcount = nullptr);
BrickArgs brick_args(Call& k, const gve_eval_opts* o);

}  // namespace gve
