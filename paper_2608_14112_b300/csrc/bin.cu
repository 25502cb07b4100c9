// bin.cu -- per-iteration preparation and the brick binner.
//
//   prep    one thread per Gaussian: activation of the Eq. 2 parameters,
//           float32 keep-test coefficients, the conservative brick cover and
//           the number of tiles (kTile^3 bricks) its brick box touches.
//   stage 1 the (tile, Gaussian) pairs, Gaussian-major (exclusive scan of the
//           tile counts, one warp per 32 Gaussians over their flattened tile
//           boxes), stably sorted by tile key: every tile lists its Gaussians
//           in ascending order.
//   stage 2 one CTA per tile: the brick cover test on the bricks of each
//           listed Gaussian's box inside the tile (a 64-bit pass mask per
//           listed Gaussian, per-brick counts); the counts' exclusive scan
//           over all bricks in key order gives each brick its [start, end);
//           a second pass ranks every listed Gaussian within every brick it
//           passes (earlier listed Gaussians that pass it) and writes the
//           pair -- Gaussian index and sub-brick cover -- at start + rank.
//   The result is the (brick, Gaussian) list sorted by brick key and, within
//   a brick, by Gaussian index: what a stable sort of all brick pairs gives,
//   without sorting them.
//   sort    stable LSD radix sort, 8-bit digits, reduce-then-scan with a
//           per-warp match_any ranking in the scatter (stage 1, and the ray
//           marcher's cell pairs).
//
// Bit-exactness: the keep-test coefficients and the brick cover are computed
// with explicitly rounded float32 operations (__fmul_rn & co., no
// contraction) in the same order as the oracle's definition, so both sides
// list exactly the same pairs.
#include <climits>

#include "gve_int.cuh"

namespace gve {

BinGeom make_geom(gve_dims d, int B)
{
    BinGeom g;
    g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.B = B;
    g.nbx = (d.nx + B - 1) / B; g.nby = (d.ny + B - 1) / B; g.nbz = (d.nz + B - 1) / B;
    g.nbricks = (long long)g.nbx * g.nby * g.nbz;
    int bits = 1;
    while ((1ll << bits) < g.nbricks) ++bits;
    g.key_bits = bits;
    g.ntx = (g.nbx + kTile - 1) / kTile; g.nty = (g.nby + kTile - 1) / kTile; g.ntz = (g.nbz + kTile - 1) / kTile;
    g.ntiles = (long long)g.ntx * g.nty * g.ntz;
    bits = 1;
    while ((1ll << bits) < g.ntiles) ++bits;
    g.tkey_bits = bits;
    return g;
}

VolTab single_volume(const BinGeom& g, long long n)
{
    VolTab vt{};
    vt.nvol = 1;
    vt.goff[1] = n;
    vt.toff[1] = g.ntiles;
    vt.boff[1] = g.nbricks;
    vt.g[0] = g;
    return vt;
}

// ------------------------------------------------------------------------
// prep
// ------------------------------------------------------------------------
// BIN = false: the keep coefficients only (the sampled path has no bricks)
template <bool BIN>
__global__ void __launch_bounds__(128) k_prep(const float* __restrict__ prims, long long n, VolTab vt,
                                              float k, float4* __restrict__ rec, BinRec* __restrict__ br,
                                              uint32_t* __restrict__ tcount)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BinGeom g = vt.g[BIN ? vt_find(vt.goff, vt.nvol, i) : 0];
    const float4* p4 = reinterpret_cast<const float4*>(prims) + 3 * i;
    float4 a0 = p4[0], a1 = p4[1], a2 = p4[2];
    float pf[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
    BinRec b;
    for (int j = 0; j < 9; ++j) b.L[j] = 0.f;
    b.e[0] = b.e[1] = b.e[2] = 0.f;
    b.K2 = -1.f;
    for (int j = 0; j < 3; ++j) { b.blo[j] = 0; b.bhi[j] = -1; }
    b.nonempty = 0;
    KeepCoef kc;
    keep_coefficients(pf, kc);
    const float4 r0 = kc.r0, r1 = kc.r1, r2 = kc.r2;
    if (!BIN) {
        float4* o = rec + 3 * i;
        o[0] = r0; o[1] = r1; o[2] = r2;
        return;
    }
    // the conservative brick cover, in float32 from the keep test's own
    // scales and rotation (the CPU reference runs the same operations)
    if (kc.ok) {
        const float* sv = kc.s;
        const float smin = fminf(sv[0], fminf(sv[1], sv[2])), smax = fmaxf(sv[0], fmaxf(sv[1], sv[2]));
        const float ratio = __fdiv_rn(smax, smin);
        const float cond = __fmul_rn(ratio, ratio);
        const float kb = __fmul_rn(k, __fadd_rn(1.0001f, __fmul_rn(1e-5f, cond)));
        bool box_ok = isfinite(kb);
        for (int j = 0; j < 3 && box_ok; ++j) {
            const float var = __fadd_rn(
                __fadd_rn(__fmul_rn(__fmul_rn(kc.R[j][0], kc.R[j][0]), __fmul_rn(sv[0], sv[0])),
                          __fmul_rn(__fmul_rn(kc.R[j][1], kc.R[j][1]), __fmul_rn(sv[1], sv[1]))),
                __fmul_rn(__fmul_rn(kc.R[j][2], kc.R[j][2]), __fmul_rn(sv[2], sv[2])));
            const float r = __fadd_rn(__fmul_rn(kb, __fsqrt_rn(var)), 0.01f);
            float l = ceilf(__fsub_rn(pf[j], r)), h = floorf(__fadd_rn(pf[j], r));
            const int nj = j == 0 ? g.nx : (j == 1 ? g.ny : g.nz);
            if (!(l <= h) || !isfinite(l) || !isfinite(h)) { box_ok = false; break; }
            if (l < 0.0f) l = 0.0f;
            if (h > (float)(nj - 1)) h = (float)(nj - 1);
            if (l > h) { box_ok = false; break; }
            b.blo[j] = (int)l / g.B;
            b.bhi[j] = (int)h / g.B;
        }
        if (box_ok) {
            for (int j = 0; j < 3; ++j)
                for (int i2 = 0; i2 < 3; ++i2) b.L[j * 3 + i2] = __fdiv_rn(kc.R[i2][j], sv[j]);
            const float hB = __fadd_rn(0.5f * (float)(g.B - 1), 0.01f);
            for (int j = 0; j < 3; ++j) {
                const float sabs =
                    __fadd_rn(__fadd_rn(fabsf(b.L[j * 3 + 0]), fabsf(b.L[j * 3 + 1])), fabsf(b.L[j * 3 + 2]));
                b.e[j] = __fmul_rn(hB, sabs);
            }
            b.K2 = __fadd_rn(__fmul_rn(__fmul_rn(kb, kb), 1.0001f), 1e-4f);
            b.nonempty = 1;
        } else {
            for (int j = 0; j < 3; ++j) { b.blo[j] = 0; b.bhi[j] = -1; }
        }
    }
    float4* o = rec + 3 * i;
    o[0] = r0; o[1] = r1; o[2] = r2;
    if (BIN) {
        br[i] = b;
        uint32_t nt = 0;
        if (b.nonempty)
            nt = (uint32_t)(b.bhi[0] / kTile - b.blo[0] / kTile + 1) * (uint32_t)(b.bhi[1] / kTile - b.blo[1] / kTile + 1) *
                 (uint32_t)(b.bhi[2] / kTile - b.blo[2] / kTile + 1);
        tcount[i] = nt;
    }
}


void launch_prep_rec(const float* prims, long long n, float k, float4* rec, cudaStream_t s)
{
    if (n <= 0) return;
    VolTab vt{};
    vt.nvol = 1;
    k_prep<false><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(prims, n, vt, k, rec, nullptr, nullptr);
}


// The float32 cover test of two neighbouring bricks (bx, bx + 1) at once.
// Per brick, with c its centre (brick origin + (B - 1) / 2) and in the
// oracle's operation order: y_j = L_j2 dz + (L_j1 dy + L_j0 dx) with d =
// c - mu, a_j = max(|y_j| - e_j, 0), pass iff a_0^2 + (a_1^2 + a_2^2) <= K2,
// every operation correctly rounded (packed f32x2 multiplies and FMAs are
// two IEEE operations lane by lane).  Bit 0: brick bx passes; bit 1: bx + 1.
template <int B>
__device__ __forceinline__ uint32_t brick_test2(const BinRec& b, float mux, float muy, float muz, int bx, int by,
                                                int bz)
{
    const float half = 0.5f * (float)(B - 1);
    const float2 cx = make_float2(__fadd_rn((float)(bx * B), half), __fadd_rn((float)((bx + 1) * B), half));
    const float cy = __fadd_rn((float)(by * B), half), cz = __fadd_rn((float)(bz * B), half);
    const float2 dcx = __fadd2_rn(cx, make_float2(-mux, -mux));   // cx - mu_x
    const float dcy = __fsub_rn(cy, muy), dcz = __fsub_rn(cz, muz);
    float2 acc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float l0 = b.L[j * 3 + 0], l1 = b.L[j * 3 + 1], l2 = b.L[j * 3 + 2];
        const float2 t0 = __fmul2_rn(make_float2(l0, l0), dcx);
        const float2 y = __ffma2_rn(make_float2(l2, l2), make_float2(dcz, dcz),
                                    __ffma2_rn(make_float2(l1, l1), make_float2(dcy, dcy), t0));
        const float ax = __fsub_rn(fabsf(y.x), b.e[j]), ay = __fsub_rn(fabsf(y.y), b.e[j]);
        acc[j] = make_float2(ax > 0.0f ? ax : 0.0f, ay > 0.0f ? ay : 0.0f);
    }
    const float2 a22 = __fmul2_rn(acc[2], acc[2]);
    const float2 sq = __ffma2_rn(acc[0], acc[0], __ffma2_rn(acc[1], acc[1], a22));
    return (sq.x <= b.K2 ? 1u : 0u) | (sq.y <= b.K2 ? 2u : 0u);
}

// Gram matrix of the whitened voxel axes l_i (l_i[j] = L[j][i]), shared by
// every brick of a Gaussian: the sub-brick centres are the brick centre plus
// multiples of l_1 and l_2, so their dot products and squared lengths follow
// from the brick centre's by a few FMAs (float rounding far inside the 1e-3
// margin of the test).
struct AxisGram {
    float g01, g02, g11, g12, g22;
};

__device__ __forceinline__ AxisGram axis_gram(const float* L)
{
    AxisGram G{0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float l0 = L[j * 3 + 0], l1 = L[j * 3 + 1], l2 = L[j * 3 + 2];
        G.g01 = fmaf(l0, l1, G.g01);
        G.g02 = fmaf(l0, l2, G.g02);
        G.g11 = fmaf(l1, l1, G.g11);
        G.g12 = fmaf(l1, l2, G.g12);
        G.g22 = fmaf(l2, l2, G.g22);
    }
    return G;
}

// Sub-brick cover of a listed brick (an acceleration structure of the
// evaluator, not part of the binning definition): bit s is set when the
// B x B/2 x B/4 sub-brick s = (y half, z quarter) may hold a kept pair.  In
// whitened coordinates the sub-brick's voxel centres (half sizes
// h = ((B-1)/2, (B/2-1)/2, (B/4-1)/2) + 0.01) lie in the parallelepiped
// P = {y + sum_i s_i l_i : |s_i| <= h_i} (y its centre, l_i the images of the
// voxel axes).  Along n = y / |y| every point of P has n . p >= |y| -
// sum_i h_i |n . l_i|; when that separating distance is positive and its
// square exceeds the brick's K2 (with a 1e-3 relative margin covering the
// float32 rounding) no voxel centre of the sub-brick can be kept.  (The
// axis-aligned whitened bound of the brick test adds almost nothing here.)
// Sub-bricks outside the grid get no bit.  Conservative: it never drops a
// pair the keep test keeps.
__device__ __forceinline__ uint32_t subbrick_mask(const float* L, float K2, const AxisGram& G, float mux, float muy,
                                                  float muz, int B, int bx, int by, int bz, int ny, int nz)
{
    const float hb = 0.5f * (float)(B - 1);
    const float cx = (float)(bx * B) + hb, cy = (float)(by * B) + hb, cz = (float)(bz * B) + hb;
    const float dcx = cx - mux, dcy = cy - muy, dcz = cz - muz;
    const float h0 = hb + 0.01f, h1 = 0.5f * (float)(B / 2 - 1) + 0.01f, h2 = 0.5f * (float)(B / 4 - 1) + 0.01f;
    // brick centre yc = L (c - mu): its dot products with the axes and |yc|^2
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, yy = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float yc = fmaf(L[j * 3 + 2], dcz, fmaf(L[j * 3 + 1], dcy, L[j * 3 + 0] * dcx));
        c0 = fmaf(yc, L[j * 3 + 0], c0);
        c1 = fmaf(yc, L[j * 3 + 1], c1);
        c2 = fmaf(yc, L[j * 3 + 2], c2);
        yy = fmaf(yc, yc, yy);
    }
    // sub-brick centres y = yc + oy l_1 + oz l_2 with oy = +-B/4 and
    // oz = +-B/8, +-3B/8: the dot products with the axes are c + oy (g01,
    // g11, g12) + oz (g02, g12, g22) and |y|^2 = yy + 2 oy c1 + oy^2 g11 +
    // 2 oz (c2 + oy g12) + oz^2 g22; the +- pairs share their products
    const float oy = 0.25f * (float)B, o1 = 0.125f * (float)B, o3 = 0.375f * (float)B;
    const float ax = oy * G.g01, ay = oy * G.g11, az = oy * G.g12;
    const float A0 = fmaf(oy * oy, G.g11, yy), A1 = 2.f * oy * c1;
    const float b1x = o1 * G.g02, b1y = o1 * G.g12, b1z = o1 * G.g22;
    const float b3x = o3 * G.g02, b3y = o3 * G.g12, b3z = o3 * G.g22;
    const float q1 = o1 * o1 * G.g22, q3 = o3 * o3 * G.g22;
    const float K2m = K2 * 1.001f;
    const bool inside = (by + 1) * B <= ny && (bz + 1) * B <= nz;
    uint32_t m = 0;
#pragma unroll
    for (int yh = 0; yh < 2; ++yh) {
        const float px = yh ? c0 + ax : c0 - ax, py = yh ? c1 + ay : c1 - ay, pz = yh ? c2 + az : c2 - az;
        const float Ay = yh ? A0 + A1 : A0 - A1;
        const float s1 = 2.f * o1 * pz, s3 = 2.f * o3 * pz;
        const float Y1 = Ay + q1, Y3 = Ay + q3;
#pragma unroll
        for (int zq = 0; zq < 4; ++zq) {
            // zq = 0..3: oz = -3B/8, -B/8, +B/8, +3B/8
            const bool far = zq == 0 || zq == 3, pos = zq >= 2;
            const float bx_ = far ? b3x : b1x, by_ = far ? b3y : b1y, bz_ = far ? b3z : b1z;
            const float ylx = pos ? px + bx_ : px - bx_;
            const float yly = pos ? py + by_ : py - by_;
            const float ylz = pos ? pz + bz_ : pz - bz_;
            const float y2 = far ? (pos ? Y3 + s3 : Y3 - s3) : (pos ? Y1 + s1 : Y1 - s1);
            // |y|^2 - sum_i h_i |y . l_i| > sqrt(K2) |y|  =>  no kept voxel
            const float D = y2 - fmaf(h0, fabsf(ylx), fmaf(h1, fabsf(yly), h2 * fabsf(ylz)));
            const bool dead = D > 0.f && D * D > K2m * y2;
            const bool ingrid = inside || (by * B + (B / 2) * yh < ny && bz * B + (B / 4) * zq < nz);
            if (!dead && ingrid) m |= 1u << (yh + 2 * zq);
        }
    }
    return m;
}

// ------------------------------------------------------------------------
// device-wide exclusive scan (reduce, scan of block sums, downsweep)
// ------------------------------------------------------------------------
struct LenSpec {
    const unsigned long long* dn;  // if set: len = ceil(min(*dn, cap) / kSortTile) * 256
    unsigned long long cap;
    unsigned long long fixed;
    __device__ __forceinline__ unsigned long long get() const
    {
        if (!dn) return fixed;
        unsigned long long m = *dn < cap ? *dn : cap;
        return ((m + kSortTile - 1) / kSortTile) * 256ull;
    }
};

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// inclusive scan across the block; *total receives the block sum
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T* smem /* 32 */, T* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_incl_scan(v);
    if (lane == 31) smem[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T t = lane < nw ? smem[lane] : T(0);
        t = warp_incl_scan(t);
        if (lane < nw) smem[lane] = t;
    }
    __syncthreads();
    T add = wid > 0 ? smem[wid - 1] : T(0);
    *total = smem[nw - 1];
    __syncthreads();
    return v + add;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const TI* __restrict__ in, LenSpec L,
                                                              TO* __restrict__ part, const int* stop)
{
    if (stop && *stop) return;
    __shared__ TO sm[32];
    unsigned long long len = L.get();
    unsigned long long chunk = (len + gridDim.x - 1) / gridDim.x;
    unsigned long long b0 = (unsigned long long)blockIdx.x * chunk;
    unsigned long long b1 = b0 + chunk < len ? b0 + chunk : len;
    TO sum = 0;
    for (unsigned long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) sum += (TO)in[i];
    TO tot;
    block_incl_scan<TO>(sum, sm, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_top(TO* __restrict__ part, int nb, TO* total_out,
                                                           const int* stop)
{
    if (stop && *stop) return;
    __shared__ TO sm[32];
    TO v = threadIdx.x < nb ? part[threadIdx.x] : TO(0);
    TO tot;
    TO incl = block_incl_scan<TO>(v, sm, &tot);
    if (threadIdx.x < nb) part[threadIdx.x] = incl - v;
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const TI* in, TO* out, LenSpec L,
                                                            const TO* __restrict__ part, const int* stop)
{
    if (stop && *stop) return;
    __shared__ TO sm[32];
    unsigned long long len = L.get();
    unsigned long long chunk = (len + gridDim.x - 1) / gridDim.x;
    unsigned long long b0 = (unsigned long long)blockIdx.x * chunk;
    unsigned long long b1 = b0 + chunk < len ? b0 + chunk : len;
    TO carry = part[blockIdx.x];
    for (unsigned long long base = b0; base < b1; base += blockDim.x) {
        unsigned long long i = base + threadIdx.x;
        TO v = i < b1 ? (TO)in[i] : TO(0);
        TO tot;
        TO incl = block_incl_scan<TO>(v, sm, &tot);
        if (i < b1) out[i] = carry + incl - v;
        carry += tot;
    }
}

// pair total of a binning stage (0: brick pairs -> total, 1: tile pairs ->
// total1) against its capacity; the first iteration to exceed it is kept
__global__ void k_check_cap(DevState* st, const unsigned long long* total, unsigned long long cap, int iter, int stage)
{
    const unsigned long long t = *total;
    unsigned long long& tot = stage ? st->total1 : st->total;
    unsigned long long& mx = stage ? st->max_total1 : st->max_total;
    tot = t;
    if (t > mx) mx = t;
    if (t > cap && !st->overflow) {
        st->overflow = 1;
        st->first_overflow_iter = iter;
    }
}

void launch_offsets(const uint32_t* counts, long long n, unsigned long long* offsets, void* scanp, DevState* st,
                    unsigned long long cap, int iter, cudaStream_t s, int stage)
{
    LenSpec L{nullptr, 0, (unsigned long long)n};
    auto* part = reinterpret_cast<unsigned long long*>(scanp);
    k_scan_reduce<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(counts, L, part, nullptr);
    k_scan_top<unsigned long long><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, offsets + n, nullptr);
    k_scan_down<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(counts, offsets, L, part, nullptr);
    k_check_cap<<<1, 1, 0, s>>>(st, offsets + n, cap, iter, stage);
}

void launch_exscan_u32(const uint32_t* in, long long n, unsigned long long* out, void* scanp, cudaStream_t s)
{
    LenSpec L{nullptr, 0, (unsigned long long)n};
    auto* part = reinterpret_cast<unsigned long long*>(scanp);
    k_scan_reduce<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(in, L, part, nullptr);
    k_scan_top<unsigned long long><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, out + n, nullptr);
    k_scan_down<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(in, out, L, part, nullptr);
}

// ------------------------------------------------------------------------
// stable LSD radix sort
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long sort_len(const unsigned long long* n_dev, unsigned long long cap)
{
    const unsigned long long t = *n_dev;
    return t < cap ? t : cap;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t* __restrict__ keys, const unsigned long long* n_dev,
                                                          const int* stop,
                                                          unsigned long long cap, int shift,
                                                          uint32_t* __restrict__ hist)
{
    if (*stop) return;
    __shared__ uint32_t h[256];
    unsigned long long n = sort_len(n_dev, cap);
    unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long base = tile * kSortTile;
        // all of the thread's keys in flight at once: kSortItems / 4 vector
        // loads (the tile start is 16 KB aligned), element loads in the last
        // partial tile
        constexpr int V = kSortItems / 4;
        uint4 kv[V];
        const bool full = base + kSortTile <= n;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const unsigned long long e = base + 4ull * ((unsigned long long)k * kSortThreads + threadIdx.x);
            if (full) {
                kv[k] = *reinterpret_cast<const uint4*>(keys + e);
            } else {
                kv[k].x = e < n ? keys[e] : 0xffffffffu;
                kv[k].y = e + 1 < n ? keys[e + 1] : 0xffffffffu;
                kv[k].z = e + 2 < n ? keys[e + 2] : 0xffffffffu;
                kv[k].w = e + 3 < n ? keys[e + 3] : 0xffffffffu;
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const unsigned long long e = base + 4ull * ((unsigned long long)k * kSortThreads + threadIdx.x);
            if (e < n) atomicAdd(&h[(kv[k].x >> shift) & 255u], 1u);
            if (e + 1 < n) atomicAdd(&h[(kv[k].y >> shift) & 255u], 1u);
            if (e + 2 < n) atomicAdd(&h[(kv[k].z >> shift) & 255u], 1u);
            if (e + 3 < n) atomicAdd(&h[(kv[k].w >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(unsigned long long)threadIdx.x * ntiles + tile] = h[threadIdx.x];
        __syncthreads();
    }
}

// Stable scatter of one 8-bit digit.  Each CTA ranks its tile of kSortTile
// elements (per-warp match_any ranking, warps in element order), places the
// tile in shared memory sorted by digit, then writes every digit's run to its
// global offset with consecutive threads on consecutive addresses.
__global__ void __launch_bounds__(kSortThreads, 3) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin,
                                                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                             const unsigned long long* n_dev, const int* stop,
                                                             unsigned long long cap, int shift,
                                                             const uint32_t* __restrict__ hist)
{
    if (*stop) return;
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t wcnt[W][256];     // per-warp digit counts, then per-warp local offsets
    __shared__ uint32_t dstart[256];      // tile-local start of each digit
    __shared__ uint32_t gbase[256];       // global start of each digit for this tile
    __shared__ uint32_t sk[kSortTile], sv[kSortTile];
    __shared__ uint32_t wsum[W];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long n = sort_len(n_dev, cap);
    unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
        __syncwarp();
        const unsigned long long tbase = tile * kSortTile;
        const int tn = (int)(n - tbase < (unsigned long long)kSortTile ? n - tbase : (unsigned long long)kSortTile);
        const int wbase = w * (32 * kSortItems);
        uint32_t kk[kSortItems], vv[kSortItems];
        uint16_t rk[kSortItems];
        // issue every load of the thread before ranking
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int li = wbase + r * 32 + lane;
            kk[r] = li < tn ? kin[tbase + li] : 0xffffffffu;
            vv[r] = li < tn ? vin[tbase + li] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int li = wbase + r * 32 + lane;
            const bool valid = li < tn;
            const uint32_t key = kk[r];
            const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            const uint32_t prior = valid ? wcnt[w][d] : 0u;
            __syncwarp();
            if (valid && lane == leader) wcnt[w][d] = prior + __popc(peers);
            __syncwarp();
            rk[r] = (uint16_t)(prior + __popc(peers & lt));
        }
        __syncthreads();
        {
            // thread d: per-warp offsets within digit d, tile count of d
            const int d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) {
                const uint32_t c = wcnt[ww][d];
                wcnt[ww][d] = run;
                run += c;
            }
            // exclusive scan of the tile counts over digits (block-wide)
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane == 31) wsum[w] = incl;
            __syncthreads();
            uint32_t add = 0;
            for (int ww = 0; ww < w; ++ww) add += wsum[ww];
            const uint32_t ex = add + incl - run;
            dstart[d] = ex;
            gbase[d] = hist[(unsigned long long)d * ntiles + tile];
#pragma unroll
            for (int ww = 0; ww < W; ++ww) wcnt[ww][d] += ex;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int li = wbase + r * 32 + lane;
            if (li < tn) {
                const uint32_t d = (kk[r] >> shift) & 255u;
                const uint32_t p = wcnt[w][d] + rk[r];
                sk[p] = kk[r];
                sv[p] = vv[r];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < tn; i += kSortThreads) {
            const uint32_t key = sk[i];
            const uint32_t d = (key >> shift) & 255u;
            const uint32_t pos = gbase[d] + (uint32_t)i - dstart[d];
            kout[pos] = key;
            vout[pos] = sv[i];
        }
        __syncthreads();
    }
}

int launch_sort(uint32_t* keys[2], uint32_t* vals[2], const unsigned long long* n_dev, const int* stop,
                unsigned long long cap, int key_bits, uint32_t* hist, void* scanp, cudaStream_t s)
{
    static_assert(kSortThreads == 256, "one thread per digit in the scatter");
    int passes = (key_bits + 7) / 8;
    unsigned long long max_tiles = (cap + kSortTile - 1) / kSortTile;
    const unsigned long long gcap = 8ull * num_sms();
    int grid = (int)(max_tiles < gcap ? max_tiles : gcap);
    if (grid < 1) grid = 1;
    int cur = 0;
    auto* part = reinterpret_cast<uint32_t*>(scanp);
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<grid, kSortThreads, 0, s>>>(keys[cur], n_dev, stop, cap, shift, hist);
        LenSpec L{n_dev, cap, 0};
        k_scan_reduce<uint32_t, uint32_t><<<kScanBlocks, kScanThreads, 0, s>>>(hist, L, part, stop);
        k_scan_top<uint32_t><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, nullptr, stop);
        k_scan_down<uint32_t, uint32_t><<<kScanBlocks, kScanThreads, 0, s>>>(hist, hist, L, part, stop);
        k_rs_scatter<<<grid, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_dev, stop, cap,
                                                   shift, hist);
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------------------------
// ranges
// ------------------------------------------------------------------------
// Per-brick [start, end) of the sorted keys: each thread takes four
// consecutive keys (one vector load; the key buffer is 256-byte aligned) and
// compares them with their neighbours.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ sk, const unsigned long long* n_dev,
                                                const int* stop,
                                                unsigned long long cap, uint32_t* __restrict__ start,
                                                uint32_t* __restrict__ end)
{
    if (*stop) return;
    const unsigned long long n = sort_len(n_dev, cap);
    const unsigned long long ng = (n + 3) / 4;
    for (unsigned long long gi = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; gi < ng;
         gi += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long i0 = 4 * gi;
        uint32_t k[4];
        if (i0 + 4 <= n) {
            const uint4 v = *reinterpret_cast<const uint4*>(sk + i0);
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? sk[i0 + j] : 0u;
        }
        const uint32_t prev = i0 > 0 ? sk[i0 - 1] : 0u;
        const uint32_t next = i0 + 4 < n ? sk[i0 + 4] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned long long i = i0 + j;
            if (i >= n) break;
            const uint32_t kp = j > 0 ? k[j - 1] : prev, kn = j < 3 ? k[j + 1] : next;
            if (i == 0 || kp != k[j]) start[k[j]] = (uint32_t)i;
            if (i + 1 == n || kn != k[j]) end[k[j]] = (uint32_t)(i + 1);
        }
    }
}

void launch_ranges(const uint32_t* skeys, const unsigned long long* n_dev, const int* stop, unsigned long long cap,
                   uint32_t* start, uint32_t* end, cudaStream_t s)
{
    k_ranges<<<16 * num_sms(), 256, 0, s>>>(skeys, n_dev, stop, cap, start, end);
}


// ------------------------------------------------------------------------
// two-level binning: stage 1 (tiles) and stage 2 (bricks)
// ------------------------------------------------------------------------
// Owner of flattened item `it` among a warp's 32 entries: the first j whose
// inclusive item count exceeds it (incl is non-decreasing, it < incl[31]).
__device__ __forceinline__ int flat_owner(const uint32_t* incl, uint32_t it)
{
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (incl[j + step - 1] <= it) j += step;
    return j;
}

// Stage 1 emission: warp = 32 consecutive Gaussians; their tile boxes are
// flattened (box-major, z-major inside a box) and handed out 32 items at a
// time, so small and large boxes keep every lane busy.  The group's pairs
// start at the scanned offset of its first Gaussian.
__global__ void __launch_bounds__(256) k_temit(const BinRec* __restrict__ br, const uint32_t* __restrict__ tcount,
                                               const unsigned long long* __restrict__ toff, long long n, VolTab vt,
                                               uint32_t* __restrict__ tkeys, uint32_t* __restrict__ tvals,
                                               const DevState* __restrict__ st)
{
    if (st->overflow) return;
    __shared__ uint32_t s_incl[8][32];
    __shared__ int4 s_box[8][32];      // first tile (x, y, z) and x extent of each box
    __shared__ uint32_t s_exy[8][32];  // x extent * y extent
    __shared__ int4 s_tg[8][32];       // the volume's tile grid (x, y) and first global tile
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long ngroups = (n + 31) >> 5;
    for (long long grp = (long long)blockIdx.x * 8 + w; grp < ngroups; grp += (long long)gridDim.x * 8) {
        const long long i = (grp << 5) + lane;
        uint32_t cnt = 0, exy = 1;
        int4 box = make_int4(0, 0, 0, 1);
        int4 tg = make_int4(1, 1, 0, 0);   // tile grid x, y and first tile (low, high word) of the volume
        if (i < n) {
            cnt = tcount[i];
            if (cnt) {
                const BinRec& b = br[i];
                const int x0 = b.blo[0] / kTile, y0 = b.blo[1] / kTile, z0 = b.blo[2] / kTile;
                const int ex = b.bhi[0] / kTile - x0 + 1, ey = b.bhi[1] / kTile - y0 + 1;
                box = make_int4(x0, y0, z0, ex);
                exy = (uint32_t)ex * (uint32_t)ey;
                const int v = vt_find(vt.goff, vt.nvol, i);
                const unsigned long long t0 = (unsigned long long)vt.toff[v];
                tg = make_int4(vt.g[v].ntx, vt.g[v].nty, (int)(uint32_t)t0, (int)(uint32_t)(t0 >> 32));
            }
        }
        const uint32_t incl = warp_incl_scan(cnt);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        s_incl[w][lane] = incl;
        s_box[w][lane] = box;
        s_exy[w][lane] = exy;
        s_tg[w][lane] = tg;
        __syncwarp();
        const unsigned long long base = total ? toff[grp << 5] : 0ull;
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
            const uint32_t it = t0 + lane;
            if (it < total) {
                const int j = flat_owner(s_incl[w], it);
                const uint32_t t = it - (j ? s_incl[w][j - 1] : 0u);
                const int4 bx = s_box[w][j];
                const uint32_t e2 = s_exy[w][j];
                const uint32_t tz = t / e2, r = t - tz * e2;
                const uint32_t ty = r / (uint32_t)bx.w, tx = r - ty * (uint32_t)bx.w;
                const int4 tgj = s_tg[w][j];
                const unsigned long long t0 = (unsigned long long)(uint32_t)tgj.z | ((unsigned long long)(uint32_t)tgj.w << 32);
                tkeys[base + it] = (uint32_t)(t0 + (unsigned long long)(((long long)(bx.z + (int)tz) * tgj.y +
                                                                          (bx.y + (int)ty)) * tgj.x + (bx.x + (int)tx)));
                tvals[base + it] = (uint32_t)((grp << 5) + j);
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void tile_origin(const BinGeom& g, long long tile, int& ox, int& oy, int& oz)
{
    ox = (int)(tile % g.ntx) * kTile;
    oy = (int)((tile / g.ntx) % g.nty) * kTile;
    oz = (int)(tile / ((long long)g.ntx * g.nty)) * kTile;
}

// 32 x 32 bit transpose across a warp: lane i holds row x (bit j = column
// j); afterwards lane j holds column j (bit i = bit j of lane i's row), i.e.
// the ballot of bit j.  Five rounds of exchanging the off-diagonal blocks.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x)
{
    const int lane = threadIdx.x & 31;
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sh = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y >> sh) & m)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

// floor(t / d) for t < 64 and 1 <= d <= 64 as (t * ceil(2^16 / d)) >> 16:
// the rounding of the reciprocal adds less than t / 2^16 < 1/1024 < 1/d to
// t / d, whose fraction is at most (d - 1) / d, so the floor is exact.
__device__ __forceinline__ uint32_t small_div(uint32_t t, uint32_t magic) { return (t * magic) >> 16; }
__device__ __forceinline__ uint32_t small_magic(uint32_t d) { return (65536u + d - 1u) / d; }

// chunk index of chunk c (32 list entries) of the tile whose list starts at
// ts: (ts >> 5) + tile + c -- distinct over all tiles, below
// cap1 / 32 + ntiles + 1
__device__ __forceinline__ unsigned long long chunk_id(uint32_t ts, long long tile, uint32_t c)
{
    return (unsigned long long)(ts >> 5) + (unsigned long long)tile + c;
}

// Stage 2, first pass (one 256-thread CTA per tile; rounds of 256 list
// entries, warp w holding chunk 8 r + w = entries 32 w .. 32 w + 31 of round
// r).  The cover test runs on the bricks of each listed Gaussian's box
// inside the tile: the box's rows of bricks along x (up to four) are
// flattened per warp as in stage 1, and each lane tests one row, two bricks
// at a time.  Writes the 64-bit pass
// mask of every entry (bit = (z * 4 + y) * 4 + x of the brick inside the
// tile), per chunk and brick the passes of all earlier entries of the tile
// (the chunk's base), the pair count of each brick of the tile, and, when
// gcount is set, adds each Gaussian's passes to gcount (introspection).
template <int B>
__global__ void __launch_bounds__(256, 6) k_bcount(const BinRec* __restrict__ br, const float4* __restrict__ rec,
                                                const uint32_t* __restrict__ tgid, const uint32_t* __restrict__ trange,
                                                VolTab vt, unsigned long long* __restrict__ tmask,
                                                uint32_t* __restrict__ cbase, uint32_t* __restrict__ bcount,
                                                uint32_t* __restrict__ gcount, const DevState* __restrict__ st)
{
    if (st->overflow) return;
    const long long tile = blockIdx.x;
    const int vol = vt_find(vt.toff, vt.nvol, tile);
    const BinGeom g = vt.g[vol];
    const long long ntiles = vt.toff[vt.nvol], bbase = vt.boff[vol];
    __shared__ BinRec s_br[256];
    __shared__ float4 s_mu[256];
    __shared__ uint32_t s_m[256][2];
    __shared__ uint32_t s_wc[8][64];   // per-warp passes of each brick, then the chunk's base
    __shared__ uint32_t s_run[64];     // passes of each brick by the tile's earlier rounds
    __shared__ uint32_t s_incl[8][32];
    __shared__ int4 s_box[8][32];      // first brick (x, y, z) inside the tile, x extent
    __shared__ uint2 s_div[8][32];     // reciprocal of the y extent, y extent
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int ox, oy, oz;
    tile_origin(g, tile - vt.toff[vol], ox, oy, oz);
    if (tid < 64) s_run[tid] = 0u;
    const uint32_t ts = trange[tile], te = trange[ntiles + tile];
    for (uint32_t r0 = ts; r0 < te; r0 += 256) {
        const uint32_t e = r0 + tid;
        uint32_t cnt = 0, gid = 0;
        int4 box = make_int4(0, 0, 0, 1);
        uint2 dv = make_uint2(65536u, 1u);
        s_m[tid][0] = 0u;
        s_m[tid][1] = 0u;
        if (e < te) {
            gid = tgid[e];
            const BinRec b = br[gid];
            s_br[tid] = b;
            s_mu[tid] = rec[3 * (size_t)gid];
            const int lx = max(b.blo[0], ox) - ox, hx = min(b.bhi[0], ox + kTile - 1) - ox;
            const int ly = max(b.blo[1], oy) - oy, hy = min(b.bhi[1], oy + kTile - 1) - oy;
            const int lz = max(b.blo[2], oz) - oz, hz = min(b.bhi[2], oz + kTile - 1) - oz;
            if (lx <= hx && ly <= hy && lz <= hz) {
                const uint32_t ey = (uint32_t)(hy - ly + 1);
                box = make_int4(lx, ly, lz, hx - lx + 1);
                dv = make_uint2(small_magic(ey), ey);
                cnt = ey * (uint32_t)(hz - lz + 1);   // rows of bricks along x
            }
        }
        const uint32_t incl = warp_incl_scan(cnt);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        s_incl[w][lane] = incl;
        s_box[w][lane] = box;
        s_div[w][lane] = dv;
        __syncwarp();
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
            const uint32_t it = t0 + lane;
            if (it < total) {
                const int j = flat_owner(s_incl[w], it);
                const uint32_t t = it - (j ? s_incl[w][j - 1] : 0u);
                const int4 bx = s_box[w][j];
                const uint2 d = s_div[w][j];
                const uint32_t cz = small_div(t, d.x), cy = t - cz * d.y;
                const int ly = bx.y + (int)cy, lz = bx.z + (int)cz;
                const int slot = (w << 5) + j;
                const float4 mu = s_mu[slot];
                // the row's bricks share one word of the mask (4 | 32)
                const int lb0 = (lz * kTile + ly) * kTile + bx.x;
                uint32_t bits = 0;
                for (int cx = 0; cx < bx.w; cx += 2) {
                    const uint32_t two = brick_test2<B>(s_br[slot], mu.x, mu.y, mu.z, ox + bx.x + cx, oy + ly, oz + lz);
                    bits |= (cx + 1 < bx.w ? two : (two & 1u)) << cx;
                }
                if (bits) atomicOr(&s_m[slot][lb0 >> 5], bits << (lb0 & 31));
            }
        }
        __syncwarp();
        const uint32_t m0 = s_m[tid][0], m1 = s_m[tid][1];
        if (e < te) {
            tmask[e] = ((unsigned long long)m1 << 32) | m0;
            if (gcount) atomicAdd(&gcount[gid], (uint32_t)(__popc(m0) + __popc(m1)));
        }
        // lane j: passes of bricks j and 32 + j by this warp's entries
        s_wc[w][lane] = __popc(warp_transpose32(m0));
        s_wc[w][32 + lane] = __popc(warp_transpose32(m1));
        __syncthreads();
        if (tid < 64) {
            uint32_t run = s_run[tid];
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) {
                const uint32_t c = s_wc[ww][tid];
                s_wc[ww][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        const uint32_t c0 = r0 - ts + (uint32_t)(w << 5);   // first entry of the chunk, within the tile
        if (ts + c0 < te) {
            uint32_t* cb = cbase + 64ull * chunk_id(ts, tile, c0 >> 5);
            cb[lane] = s_wc[w][lane];
            cb[32 + lane] = s_wc[w][32 + lane];
        }
        __syncthreads();
    }
    if (tid < 64) {
        const int bx = ox + (tid & 3), by = oy + ((tid >> 2) & 3), bz = oz + (tid >> 4);
        if (bx < g.nbx && by < g.nby && bz < g.nbz)
            bcount[bbase + ((long long)bz * g.nby + by) * g.nbx + bx] = s_run[tid];
    }
}

// Stage 2 ranges from the scanned brick counts: [start, end) per brick, 0,0
// for an empty brick; the total is checked against the pair capacity.
__global__ void __launch_bounds__(256) k_brick_ranges(const uint32_t* __restrict__ bcount,
                                                      const unsigned long long* __restrict__ boff, long long nbricks,
                                                      uint32_t* __restrict__ start, uint32_t* __restrict__ end,
                                                      DevState* st, unsigned long long cap, int iter)
{
    if (st->overflow) return;  // an earlier stage overflowed: the counts are stale
    const unsigned long long total = boff[nbricks];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->total = total;
        if (total > st->max_total) st->max_total = total;
        if (total > cap) {
            st->overflow = 1;
            st->first_overflow_iter = iter;
        }
    }
    if (total > cap) return;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nbricks;
         b += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = bcount[b];
        const uint32_t s0 = c ? (uint32_t)boff[b] : 0u;
        start[b] = s0;
        end[b] = c ? s0 + c : 0u;
    }
}

// what the second pass needs of a listed Gaussian (19 words: an odd stride,
// so consecutive slots fall in distinct banks)
struct SubRec {
    float L[9];
    float K2;
    float mx, my, mz;
    AxisGram G;
    uint32_t gid;
};

// Stage 2, second pass (one 256-thread CTA per tile; warps take the tile's
// chunks of 32 list entries independently, no block barrier after the
// start).  Per chunk: the 64 per-brick ballots of the entries' masks come
// from one bit transpose; the chunk's (entry, brick) pairs are laid out
// brick-major in shared memory (slot = passes of lower bricks in the chunk
// + passes of earlier entries in the brick), half of the bricks at a time;
// then every lane takes one pair, computes its sub-brick cover and writes it
// at brick start + chunk base + rank, so a brick's pairs of one chunk land
// on consecutive addresses.
template <int B>
__global__ void __launch_bounds__(256) k_bemit(const BinRec* __restrict__ br, const float4* __restrict__ rec,
                                               const uint32_t* __restrict__ tgid, const uint32_t* __restrict__ trange,
                                               const unsigned long long* __restrict__ tmask,
                                               const uint32_t* __restrict__ cbase,
                                               const unsigned long long* __restrict__ boff, VolTab vt,
                                               uint32_t* __restrict__ pairs, const DevState* __restrict__ st)
{
    if (st->overflow) return;
    const long long tile = blockIdx.x;
    const uint32_t ts = trange[tile], te = trange[vt.toff[vt.nvol] + tile];
    if (ts >= te) return;
    const int vol = vt_find(vt.toff, vt.nvol, tile);
    const BinGeom g = vt.g[vol];
    const long long bbase = vt.boff[vol];
    __shared__ SubRec s_r[256];
    __shared__ uint32_t s_start[64];
    __shared__ uint32_t s_col[8][64];    // per brick: ballot of the chunk's entries passing it
    __shared__ uint32_t s_pos[8][64];    // per brick: global position of the chunk's first pair in it
    __shared__ uint32_t s_pre[8][64];    // per brick: pairs of lower bricks of the same half in the chunk
    __shared__ uint16_t s_list[8][1024]; // (entry << 6 | brick), brick-major
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int ox, oy, oz;
    tile_origin(g, tile - vt.toff[vol], ox, oy, oz);
    if (tid < 64) {
        const int bx = ox + (tid & 3), by = oy + ((tid >> 2) & 3), bz = oz + (tid >> 4);
        s_start[tid] = (bx < g.nbx && by < g.nby && bz < g.nbz)
                           ? (uint32_t)boff[bbase + ((long long)bz * g.nby + by) * g.nbx + bx]
                           : 0u;
    }
    __syncthreads();
    const uint32_t nchunks = (te - ts + 31) >> 5;
    for (uint32_t c = (uint32_t)w; c < nchunks; c += 8) {
        const uint32_t e = ts + (c << 5) + lane;
        uint32_t m0 = 0u, m1 = 0u;
        if (e < te) {
            const unsigned long long m = tmask[e];
            m0 = (uint32_t)m;
            m1 = (uint32_t)(m >> 32);
            if (m) {
                const uint32_t gid = tgid[e];
                const BinRec b = br[gid];
                const float4 mu = rec[3 * (size_t)gid];
                SubRec& q = s_r[tid];
#pragma unroll
                for (int j = 0; j < 9; ++j) q.L[j] = b.L[j];
                q.K2 = b.K2;
                q.mx = mu.x;
                q.my = mu.y;
                q.mz = mu.z;
                q.G = axis_gram(b.L);
                q.gid = gid;
            }
        }
        const uint32_t* cb = cbase + 64ull * chunk_id(ts, tile, c);
        const uint32_t col0 = warp_transpose32(m0), col1 = warp_transpose32(m1);
        const uint32_t n0 = __popc(col0), n1 = __popc(col1);
        const uint32_t p0 = warp_incl_scan(n0) - n0, p1 = warp_incl_scan(n1) - n1;
        const uint32_t tot0 = __shfl_sync(0xffffffffu, p0 + n0, 31), tot1 = __shfl_sync(0xffffffffu, p1 + n1, 31);
        s_col[w][lane] = col0;
        s_col[w][32 + lane] = col1;
        s_pre[w][lane] = p0;
        s_pre[w][32 + lane] = p1;
        s_pos[w][lane] = s_start[lane] + cb[lane];
        s_pos[w][32 + lane] = s_start[32 + lane] + cb[32 + lane];
        __syncwarp();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const uint32_t tot = half ? tot1 : tot0;
            if (tot == 0) continue;
            for (uint32_t mm = half ? m1 : m0; mm; mm &= mm - 1) {
                const int b = (__ffs(mm) - 1) + 32 * half;
                s_list[w][s_pre[w][b] + __popc(s_col[w][b] & lt)] = (uint16_t)((lane << 6) | b);
            }
            __syncwarp();
            for (uint32_t k0 = 0; k0 < tot; k0 += 32) {
                const uint32_t k = k0 + lane;
                if (k < tot) {
                    const uint32_t jb = s_list[w][k];
                    const uint32_t j = jb >> 6;
                    const int lb = (int)(jb & 63u);
                    const SubRec& q = s_r[(w << 5) + j];
                    const uint32_t mask = subbrick_mask(q.L, q.K2, q.G, q.mx, q.my, q.mz, B, ox + (lb & 3),
                                                        oy + ((lb >> 2) & 3), oz + (lb >> 4), g.ny, g.nz);
                    const uint32_t rank = __popc(s_col[w][lb] & ((1u << j) - 1u));
                    pairs[s_pos[w][lb] + rank] = q.gid | (mask << kGidBits);
                }
            }
            __syncwarp();
        }
    }
}

// fills keys[start, end) with the brick key of every non-empty brick
// (introspection: the sorted key column of the pair list)
__global__ void k_fill_keys(const uint32_t* __restrict__ start, const uint32_t* __restrict__ end, long long nbricks,
                            uint32_t* __restrict__ keys)
{
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nbricks;
         b += (long long)gridDim.x * blockDim.x)
        for (uint32_t p = start[b]; p < end[b]; ++p) keys[p] = (uint32_t)b;
}

void launch_fill_keys(const uint32_t* ranges, long long nbricks, uint32_t* keys, cudaStream_t s)
{
    k_fill_keys<<<4 * num_sms(), 256, 0, s>>>(ranges, ranges + nbricks, nbricks, keys);
}

int launch_binning(const BinBufs& b, const float* prims, long long n, const VolTab& vt, float k, int iter,
                   cudaStream_t s)
{
    DevState* st = b.st;
    const long long ntiles = vt.toff[vt.nvol], nbricks = vt.boff[vt.nvol];
    int tbits = 1;
    while ((1ll << tbits) < ntiles) ++tbits;
    int launches = 0;
    if (n > 0) {
        k_prep<true><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(prims, n, vt, k, b.rec, b.br, b.tcount);
        ++launches;
    }
    launch_offsets(b.tcount, n, b.toff, b.scanp, st, b.cap1, iter, s, 1);
    launches += 4;
    if (n > 0) {
        long long blocks = ((n + 31) / 32 + 7) / 8;
        if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
        k_temit<<<(unsigned)blocks, 256, 0, s>>>(b.br, b.tcount, b.toff, n, vt, b.tkeys[0], b.tvals[0], st);
        ++launches;
    }
    uint32_t* kk[2] = {b.tkeys[0], b.tkeys[1]};
    uint32_t* vv[2] = {b.tvals[0], b.tvals[1]};
    const int cur = launch_sort(kk, vv, &st->total1, &st->overflow, b.cap1, tbits, b.hist, b.scanp, s);
    launches += 5 * ((tbits + 7) / 8);
    cudaMemsetAsync(b.trange, 0, sizeof(uint32_t) * 2 * (size_t)ntiles, s);
    launch_ranges(kk[cur], &st->total1, &st->overflow, b.cap1, b.trange, b.trange + ntiles, s);
    ++launches;
    if (b.gcount && n > 0) cudaMemsetAsync(b.gcount, 0, sizeof(uint32_t) * (size_t)n, s);
    const int B = vt.g[0].B;   // one brick edge for every volume
    if (B == 4)
        k_bcount<4><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, vt, b.tmask, b.cbase, b.bcount,
                                                      b.gcount, st);
    else if (B == 16)
        k_bcount<16><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, vt, b.tmask, b.cbase,
                                                       b.bcount, b.gcount, st);
    else
        k_bcount<8><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, vt, b.tmask, b.cbase, b.bcount,
                                                      b.gcount, st);
    launch_exscan_u32(b.bcount, nbricks, b.boff, b.scanp, s);
    long long rb = (nbricks + 255) / 256;
    if (rb > 8LL * num_sms()) rb = 8LL * num_sms();
    k_brick_ranges<<<(unsigned)rb, 256, 0, s>>>(b.bcount, b.boff, nbricks, b.ranges, b.ranges + nbricks, st, b.cap,
                                                iter);
    if (B == 4)
        k_bemit<4><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, b.tmask, b.cbase, b.boff, vt,
                                                     b.pairs, st);
    else if (B == 16)
        k_bemit<16><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, b.tmask, b.cbase, b.boff, vt,
                                                      b.pairs, st);
    else
        k_bemit<8><<<(unsigned)ntiles, 256, 0, s>>>(b.br, b.rec, vv[cur], b.trange, b.tmask, b.cbase, b.boff, vt,
                                                     b.pairs, st);
    launches += 6;
    return launches;
}

}  // namespace gve
