// bin.cu -- per-iteration preparation and the brick binner.
//
//   prep    one thread per Gaussian: activation of the Eq. 2 parameters,
//           float32 keep-test coefficients, and the conservative brick cover.
//   count   one warp per Gaussian: bricks of its box that pass the cover test.
//   offsets exclusive scan of the counts (total checked against capacity).
//   emit    one warp per Gaussian: (brick key, gid) pairs, Gaussian-major,
//           bricks ascending (ballot + popc keeps the order).
//   sort    stable LSD radix sort, 8-bit digits, reduce-then-scan with a
//           per-warp match_any ranking in the scatter.
//   ranges  per-brick [start, end) by adjacent difference.
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
    return g;
}

// ------------------------------------------------------------------------
// prep
// ------------------------------------------------------------------------
// BIN = false: the keep coefficients only (the sampled path has no bricks)
template <bool BIN>
__global__ void __launch_bounds__(128) k_prep(const float* __restrict__ prims, long long n, BinGeom g,
                                              float k, float4* __restrict__ rec, BinRec* __restrict__ br)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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
            const float hB = __fadd_rn((float)(0.5 * (double)(g.B - 1)), 0.01f);
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
    if (BIN) br[i] = b;
}

void launch_prep(const float* prims, long long n, const BinGeom& g, float k, float4* rec, BinRec* br,
                 cudaStream_t s)
{
    if (n <= 0) return;
    k_prep<true><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(prims, n, g, k, rec, br);
}

void launch_prep_rec(const float* prims, long long n, float k, float4* rec, cudaStream_t s)
{
    if (n <= 0) return;
    BinGeom g{};
    k_prep<false><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(prims, n, g, k, rec, nullptr);
}

// float32 cover test of one brick (same operation order as the oracle)
__device__ __forceinline__ bool brick_test(const BinRec& b, float mux, float muy, float muz, int B, int bx,
                                           int by, int bz)
{
    float half = (float)(0.5 * (double)(B - 1));
    float cx = __fadd_rn((float)(bx * B), half);
    float cy = __fadd_rn((float)(by * B), half);
    float cz = __fadd_rn((float)(bz * B), half);
    float dcx = __fsub_rn(cx, mux), dcy = __fsub_rn(cy, muy), dcz = __fsub_rn(cz, muz);
    float acc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float t0 = __fmul_rn(b.L[j * 3 + 0], dcx);
        float y = __fmaf_rn(b.L[j * 3 + 2], dcz, __fmaf_rn(b.L[j * 3 + 1], dcy, t0));
        float a = __fsub_rn(fabsf(y), b.e[j]);
        acc[j] = a > 0.0f ? a : 0.0f;
    }
    float a22 = __fmul_rn(acc[2], acc[2]);
    float sq = __fmaf_rn(acc[0], acc[0], __fmaf_rn(acc[1], acc[1], a22));
    return sq <= b.K2;
}

// Gram matrix of the whitened voxel axes l_i (l_i[j] = L[j][i]), shared by
// every brick of a Gaussian: the sub-brick centres are the brick centre plus
// multiples of l_1 and l_2, so their dot products and squared lengths follow
// from the brick centre's by a few FMAs (float rounding far inside the 1e-3
// margin of the test).
struct AxisGram {
    float g01, g02, g11, g12, g22;
};

__device__ __forceinline__ AxisGram axis_gram(const BinRec& b)
{
    AxisGram G{0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float l0 = b.L[j * 3 + 0], l1 = b.L[j * 3 + 1], l2 = b.L[j * 3 + 2];
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
__device__ __forceinline__ uint32_t subbrick_mask(const BinRec& b, const AxisGram& G, float mux, float muy,
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
        const float yc = fmaf(b.L[j * 3 + 2], dcz, fmaf(b.L[j * 3 + 1], dcy, b.L[j * 3 + 0] * dcx));
        c0 = fmaf(yc, b.L[j * 3 + 0], c0);
        c1 = fmaf(yc, b.L[j * 3 + 1], c1);
        c2 = fmaf(yc, b.L[j * 3 + 2], c2);
        yy = fmaf(yc, yc, yy);
    }
    const float oyv = 0.25f * (float)B, ozv = 0.125f * (float)B;
    const float K2m = b.K2 * 1.001f;
    uint32_t m = 0;
#pragma unroll
    for (int yh = 0; yh < 2; ++yh) {
        if (by * B + (B / 2) * yh >= ny) continue;
        const float oy = yh ? oyv : -oyv;
        // y = yc + oy l_1 + oz l_2
        const float px = fmaf(oy, G.g01, c0), py = fmaf(oy, G.g11, c1), pz = fmaf(oy, G.g12, c2);
        const float A = fmaf(oy, fmaf(oy, G.g11, 2.f * c1), yy);
        const float Bz = 2.f * pz;
#pragma unroll
        for (int zq = 0; zq < 4; ++zq) {
            if (bz * B + (B / 4) * zq >= nz) continue;
            const float oz = (float)(2 * zq - 3) * ozv;
            const float ylx = fmaf(oz, G.g02, px), yly = fmaf(oz, G.g12, py), ylz = fmaf(oz, G.g22, pz);
            const float y2 = fmaf(oz, fmaf(oz, G.g22, Bz), A);
            // |y|^2 - sum_i h_i |y . l_i| > sqrt(K2) |y|  =>  no kept voxel
            const float D = y2 - fmaf(h0, fabsf(ylx), fmaf(h1, fabsf(yly), h2 * fabsf(ylz)));
            if (D > 0.f && D * D > K2m * y2) continue;
            m |= 1u << (yh + 2 * zq);
        }
    }
    return m;
}

// ------------------------------------------------------------------------
// count / emit (one warp per Gaussian)
// ------------------------------------------------------------------------
// Bricks of a Gaussian's box in z-major order; the box has fewer than 2^31
// bricks, so 32-bit index arithmetic suffices.  The pass/fail ballots of the
// first kMaskChunks x 32 bricks are kept for the emission pass.
// Division by the box extents: for boxes of fewer than 2^24 bricks a float
// reciprocal gives the quotient to within one (relative error below 2^-23 on
// quotients below 2^23; divisor 1 is exact), and one exact integer step
// corrects it; larger boxes use integer division.
struct BoxIdx {
    uint32_t ex, exy;
    float iex, iexy;
    bool fast;
};

__device__ __forceinline__ BoxIdx box_idx(uint32_t ex, uint32_t exy, uint32_t tot)
{
    BoxIdx d;
    d.ex = ex;
    d.exy = exy;
    d.iex = 1.f / (float)ex;
    d.iexy = 1.f / (float)exy;
    d.fast = tot < (1u << 24);
    return d;
}

__device__ __forceinline__ uint32_t udiv_small(uint32_t t, uint32_t d, float id)
{
    int q = (int)__fmul_rn((float)t, id);
    const int r = (int)t - q * (int)d;
    if (r < 0) --q;
    else if (r >= (int)d) ++q;
    return (uint32_t)q;
}

__device__ __forceinline__ void box_brick(const BinRec& b, uint32_t t, const BoxIdx& d, int& bx, int& by, int& bz)
{
    uint32_t zq, yq;
    if (d.fast) {
        zq = udiv_small(t, d.exy, d.iexy);
        yq = udiv_small(t - zq * d.exy, d.ex, d.iex);
    } else {
        zq = t / d.exy;
        yq = (t - zq * d.exy) / d.ex;
    }
    const uint32_t r = t - zq * d.exy;
    bx = b.blo[0] + (int)(r - yq * d.ex);
    by = b.blo[1] + (int)yq;
    bz = b.blo[2] + (int)zq;
}

__global__ void __launch_bounds__(256) k_count(const BinRec* __restrict__ br, const float4* __restrict__ rec,
                                               long long n, BinGeom g, uint32_t* __restrict__ counts,
                                               uint32_t* __restrict__ bmask)
{
    const int lane = threadIdx.x & 31;
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wid; i < n; i += nw) {
        const BinRec b = br[i];
        uint32_t cnt = 0;
        if (b.nonempty) {
            const float4 r0 = rec[3 * i];
            const uint32_t ex = b.bhi[0] - b.blo[0] + 1, ey = b.bhi[1] - b.blo[1] + 1, ez = b.bhi[2] - b.blo[2] + 1;
            const uint32_t exy = ex * ey, tot = exy * ez;
        const BoxIdx D = box_idx(ex, exy, tot);
            for (uint32_t t0 = 0, c = 0; t0 < tot; t0 += 32, ++c) {
                const uint32_t t = t0 + lane;
                bool pass = false;
                if (t < tot) {
                    int bx, by, bz;
                    box_brick(b, t, D, bx, by, bz);
                    pass = brick_test(b, r0.x, r0.y, r0.z, g.B, bx, by, bz);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                cnt += __popc(bal);
                if (c < kMaskChunks && lane == 0) bmask[kMaskChunks * i + c] = bal;
            }
        }
        if (lane == 0) counts[i] = cnt;
    }
}

// One warp per Gaussian.  The listed bricks of its box are queued in box
// order in shared memory and processed 32 at a time, so that every lane
// computes a sub-brick cover (the costly part) instead of only the lanes
// whose brick passed; pair i of the Gaussian goes to offsets[g] + i.
__global__ void __launch_bounds__(256) k_emit(const BinRec* __restrict__ br, const float4* __restrict__ rec,
                                              const unsigned long long* __restrict__ offsets, long long n,
                                              BinGeom g, const uint32_t* __restrict__ bmask,
                                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                              const DevState* __restrict__ st)
{
    if (st->overflow) return;
    __shared__ uint32_t s_q[8][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* q = s_q[w];
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wid; i < n; i += nw) {
        const BinRec b = br[i];
        if (!b.nonempty) continue;
        const float4 r0 = rec[3 * i];
        const AxisGram G = axis_gram(b);
        unsigned long long base = offsets[i];
        const uint32_t ex = b.bhi[0] - b.blo[0] + 1, ey = b.bhi[1] - b.blo[1] + 1, ez = b.bhi[2] - b.blo[2] + 1;
        const uint32_t exy = ex * ey, tot = exy * ez;
        const BoxIdx D = box_idx(ex, exy, tot);
        // write the first m queued bricks (m <= 32) as pairs base .. base + m - 1
        auto flush = [&](uint32_t m) {
            if ((uint32_t)lane < m) {
                int bx, by, bz;
                box_brick(b, q[lane], D, bx, by, bz);
                const uint32_t key = (uint32_t)(((long long)bz * g.nby + by) * g.nbx + bx);
                const uint32_t mask = subbrick_mask(b, G, r0.x, r0.y, r0.z, g.B, bx, by, bz, g.ny, g.nz);
                keys[base + lane] = key;
                vals[base + lane] = (uint32_t)i | (mask << kGidBits);
            }
            base += m;
        };
        uint32_t qn = 0;
        for (uint32_t t0 = 0, c = 0; t0 < tot; t0 += 32, ++c) {
            const uint32_t t = t0 + lane;
            unsigned bal;
            if (c < kMaskChunks) {
                bal = bmask[kMaskChunks * i + c];
            } else {
                bool p = false;
                if (t < tot) {
                    int bx, by, bz;
                    box_brick(b, t, D, bx, by, bz);
                    p = brick_test(b, r0.x, r0.y, r0.z, g.B, bx, by, bz);
                }
                bal = __ballot_sync(0xffffffffu, p);
            }
            if ((bal >> lane) & 1u) q[qn + __popc(bal & lt)] = t;
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {
                flush(32);
                __syncwarp();
                if ((uint32_t)lane < qn - 32) q[lane] = q[32 + lane];
                qn -= 32;
                __syncwarp();
            }
        }
        flush(qn);
        __syncwarp();
    }
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
                                                              TO* __restrict__ part, const DevState* st)
{
    if (st && st->overflow) return;
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
                                                           const DevState* st)
{
    if (st && st->overflow) return;
    __shared__ TO sm[32];
    TO v = threadIdx.x < nb ? part[threadIdx.x] : TO(0);
    TO tot;
    TO incl = block_incl_scan<TO>(v, sm, &tot);
    if (threadIdx.x < nb) part[threadIdx.x] = incl - v;
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const TI* in, TO* out, LenSpec L,
                                                            const TO* __restrict__ part, const DevState* st)
{
    if (st && st->overflow) return;
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

__global__ void k_check_cap(DevState* st, const unsigned long long* total, unsigned long long cap, int iter)
{
    unsigned long long t = *total;
    st->total = t;
    if (t > st->max_total) st->max_total = t;
    if (t > cap && !st->overflow) {
        st->overflow = 1;
        st->first_overflow_iter = iter;
    }
}

void launch_offsets(const uint32_t* counts, long long n, unsigned long long* offsets, void* scanp, DevState* st,
                    unsigned long long cap, int iter, cudaStream_t s)
{
    LenSpec L{nullptr, 0, (unsigned long long)n};
    auto* part = reinterpret_cast<unsigned long long*>(scanp);
    k_scan_reduce<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(counts, L, part, nullptr);
    k_scan_top<unsigned long long><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, offsets + n, nullptr);
    k_scan_down<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(counts, offsets, L, part, nullptr);
    k_check_cap<<<1, 1, 0, s>>>(st, offsets + n, cap, iter);
}

void launch_exscan_u32(const uint32_t* in, long long n, unsigned long long* out, void* scanp, cudaStream_t s)
{
    LenSpec L{nullptr, 0, (unsigned long long)n};
    auto* part = reinterpret_cast<unsigned long long*>(scanp);
    k_scan_reduce<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(in, L, part, nullptr);
    k_scan_top<unsigned long long><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, out + n, nullptr);
    k_scan_down<uint32_t, unsigned long long><<<kScanBlocks, kScanThreads, 0, s>>>(in, out, L, part, nullptr);
}

static int emit_blocks(long long n)
{
    long long warps = n;
    long long blocks = (warps * 32 + 255) / 256;
    if (blocks > 64LL * num_sms()) blocks = 64LL * num_sms();
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

void launch_count(const BinRec* br, const float4* rec, long long n, const BinGeom& g, uint32_t* counts,
                  uint32_t* bmask, cudaStream_t s)
{
    if (n <= 0) return;
    k_count<<<emit_blocks(n), 256, 0, s>>>(br, rec, n, g, counts, bmask);
}

void launch_emit(const BinRec* br, const float4* rec, const unsigned long long* offsets, long long n,
                 const BinGeom& g, const uint32_t* bmask, uint32_t* keys, uint32_t* vals, const DevState* st,
                 cudaStream_t s)
{
    if (n <= 0) return;
    k_emit<<<emit_blocks(n), 256, 0, s>>>(br, rec, offsets, n, g, bmask, keys, vals, st);
}

// ------------------------------------------------------------------------
// stable LSD radix sort
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long sort_len(const DevState* st, unsigned long long cap)
{
    unsigned long long t = st->total;
    return t < cap ? t : cap;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t* __restrict__ keys, const DevState* st,
                                                          unsigned long long cap, int shift,
                                                          uint32_t* __restrict__ hist)
{
    if (st->overflow) return;
    __shared__ uint32_t h[256];
    unsigned long long n = sort_len(st, cap);
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
                                                             const DevState* st, unsigned long long cap, int shift,
                                                             const uint32_t* __restrict__ hist)
{
    if (st->overflow) return;
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t wcnt[W][256];     // per-warp digit counts, then per-warp local offsets
    __shared__ uint32_t dstart[256];      // tile-local start of each digit
    __shared__ uint32_t gbase[256];       // global start of each digit for this tile
    __shared__ uint32_t sk[kSortTile], sv[kSortTile];
    __shared__ uint32_t wsum[W];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long n = sort_len(st, cap);
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

int launch_sort(uint32_t* keys[2], uint32_t* vals[2], const DevState* st, unsigned long long cap, int key_bits,
                uint32_t* hist, void* scanp, cudaStream_t s)
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
        k_rs_hist<<<grid, kSortThreads, 0, s>>>(keys[cur], st, cap, shift, hist);
        LenSpec L{&st->total, cap, 0};
        k_scan_reduce<uint32_t, uint32_t><<<kScanBlocks, kScanThreads, 0, s>>>(hist, L, part, st);
        k_scan_top<uint32_t><<<1, kScanThreads, 0, s>>>(part, kScanBlocks, nullptr, st);
        k_scan_down<uint32_t, uint32_t><<<kScanBlocks, kScanThreads, 0, s>>>(hist, hist, L, part, st);
        k_rs_scatter<<<grid, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], st, cap,
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
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ sk, const DevState* st,
                                                unsigned long long cap, uint32_t* __restrict__ start,
                                                uint32_t* __restrict__ end)
{
    if (st->overflow) return;
    const unsigned long long n = sort_len(st, cap);
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

void launch_ranges(const uint32_t* skeys, const DevState* st, unsigned long long cap, uint32_t* start,
                   uint32_t* end, cudaStream_t s)
{
    k_ranges<<<16 * num_sms(), 256, 0, s>>>(skeys, st, cap, start, end);
}

}  // namespace gve
