// field.cu -- the brick evaluator: Eq. 3 forward, residual and SSE, and the
// backward of the loss, fused per brick of 8^3 voxels.
//
// Written for a brick edge B in {4, 8, 16} (8 by default): one CTA of
// max(B^2, 32) threads per brick, one lane per row of B voxels.  The brick's
// Gaussian list is staged in shared memory in chunks of CH (32 or 64)
// prepared records (3 x float4), each with the 8-bit sub-brick mask the
// binner attached: bit s says that the B x B/2 x B/4 sub-brick s (y half =
// s & 1, z quarter = s >> 1) may hold a kept pair.  For B = 8 this is a
// 64-thread CTA and 8x4x2 sub-bricks.
//
// Phase 1 (forward): each lane owns one row of B voxels along x.  Each warp
// takes the listed Gaussians with a live sub-brick among its rows (a ballot
// over the staged chunk), two at a time for independent work, in list
// order.  The keep exponent t is evaluated by the fixed float32 chain
//     dy = y - mu_y, dz = z - mu_z, dx = x - mu_x,
//     b = fma(qxy2, dy, qxz2*dz), c = fma(dy, fma(qyy, dy, qyz2*dz), dz*(qzz*dz)),
//     t = fma(dx, fma(qxx, dx, b), c)
// (q.. = -0.5 log2(e) Sigma^-1; voxel pairs go through the packed f32x2
// FMA, lane-wise identical to the scalar chain), the pair is kept iff t > T,
// and G = 2^t on the SFU (ex2.approx).  num += w a G, den += w G;
// Vtilde = num / max(den, rho0) (Eq. 3), residual and per-brick SSE
// (float32 within the CTA, FP64 across CTAs, in the reduction kernel:
// B300's FP64 rate is a small fraction of its FP32 rate).  The row's target
// values (or, in the backward mode, its upstream gradient) are copied to
// shared memory with cp.async when the brick starts, so that their HBM
// latency passes during the forward work.  The upstream gradient gives per
// voxel gn = dL/dnum = up / max(den, rho0) and gd = dL/dden = -Vtilde gn
// (when den >= rho0), kept in shared memory sub-brick by sub-brick.
//
// Phase 2 (backward): the (Gaussian, live sub-brick) tasks are compacted
// (sub-brick-major) and spread over all threads; a task recomputes G by the
// same chain on its B^3/8 voxels and accumulates
//     A = sum G gn,  H = sum h,  S1 = sum h d,  S2 = sum h d d^T,
//     h = G (a gn + gd)
// (dL/da = w A, dL/dw = H, and the chain rule scales S1, S2 by -w/2), with
// the y- and z-dependence factored per row and per slice and the
// x-moments taken against the brick-local offset X (constants of the
// unrolled loop), shifted to dx once per task, in packed f32x2
// arithmetic.  Task sums meet in shared memory (float atomics); one thread
// per Gaussian then issues three 16-byte vector atomics into its global
// accumulator.  Nothing per pair or per voxel goes to HBM.
#include "chain.cuh"
#include "gve_int.cuh"

namespace gve {

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// asynchronous global -> shared copies (each thread waits for its own)
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kAccStride = 13;  // padded per-Gaussian stride of the shared sums

// CTA geometry for brick edge B: one lane per row of B voxels along x (B^2
// rows; B = 4 uses one warp with 16 row lanes), sub-bricks of B x B/2 x B/4.
template <int B>
struct BrickShape {
    static constexpr int ROWS = B * B;
    static constexpr int THREADS = ROWS < 32 ? 32 : ROWS;
    static constexpr int NW = THREADS / 32;
    static constexpr int HALF = B / 2;  // voxel pairs per row
    static constexpr int SY = B / 2;    // sub-brick extent in y
    static constexpr int SZ = B / 4;    // sub-brick extent in z
    static constexpr int MINB = B == 16 ? 3 : (B == 8 ? 14 : 16);
};

// Stages the chunk's records: each thread takes whole Gaussians and issues
// all of its list and record loads before any store, so a chunk costs two
// dependent trips to L2 whatever the list length.
template <int NT, int CH>
__device__ __forceinline__ void stage_chunk(const BrickArgs& a, uint32_t s0, int c0, int cnt, float4* s_rec,
                                            uint32_t* s_msk, int tid)
{
    constexpr int PER = (CH + NT - 1) / NT;
    uint32_t v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int j = tid + k * NT;
        v[k] = j < cnt ? a.gids[s0 + c0 + j] : 0u;
    }
    float4 r[PER][3];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int j = tid + k * NT;
        if (j < cnt) {
            const float4* p = a.rec + 3 * (size_t)(v[k] & kGidMask);
            r[k][0] = p[0]; r[k][1] = p[1]; r[k][2] = p[2];
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int j = tid + k * NT;
        if (j < cnt) {
            s_rec[3 * j] = r[k][0]; s_rec[3 * j + 1] = r[k][1]; s_rec[3 * j + 2] = r[k][2];
            s_msk[j] = v[k] >> kGidBits;
        }
    }
}

// One backward task: the sums of Gaussian j (staged record) over slices
// zs0 .. zs0 + NZ - 1 of sub-brick sbt, added to its shared sums.  Whole
// tasks take all SZ slices; the tail of a round may be split into halves.
template <int B, int NZ>
__device__ __forceinline__ void task_sums(const float4* s_rec, const float4* s_g, float* s_acc, int j, int sbt,
                                          int zs0, int by, int bz, float fxb, float T)
{
    using S = BrickShape<B>;
    constexpr int HALF = S::HALF, SY = S::SY, SZ = S::SZ;
    constexpr int GBLK = SY * SZ * HALF + 1;
    const float4 r0 = s_rec[3 * j], r1 = s_rec[3 * j + 1], r2 = s_rec[3 * j + 2];
    const float2 nmu = f2(-r0.x);
    float2 dx[HALF];
#pragma unroll
    for (int q = 0; q < HALF; ++q)
        dx[q] = __fadd2_rn(make_float2(fxb + (float)(2 * q), fxb + (float)(2 * q + 1)), nmu);
    const int yb = SY * (sbt & 1), zb = SZ * (sbt >> 1);
    const float2 qxx = f2(r0.w), amp = f2(r2.w);
    // h = G (a gn + gd); x-moments against the brick-local X = x - x0,
    // shifted to dx = X + (x0 - mu_x) once per task below.  Per-voxel
    // sums are packed; the per-row and per-slice sums are scalar, so
    // they run beside the packed pipe instead of on it.
    float2 A = make_float2(0.f, 0.f), R2 = A;
    float S0 = 0.f, S1x = 0.f, S1y = 0.f, S1z = 0.f, Syy = 0.f, Szz = 0.f, Sxy = 0.f, Sxz = 0.f, Syz = 0.f;
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        const int zs = zs0 + i;
        const float dz = __fsub_rn((float)(bz * B + zb + zs), r0.z);
        const float e_ = __fmul_rn(r1.w, dz), f_ = __fmul_rn(r2.x, dz);
        const float dzh = __fmul_rn(dz, __fmul_rn(r1.y, dz));
        float T0 = 0.f, T1 = 0.f, Ty = 0.f;
#pragma unroll
        for (int yr = 0; yr < SY; ++yr) {
            const float dy = __fsub_rn((float)(by * B + yb + yr), r0.y);
            const float bb = __fmaf_rn(r1.z, dy, e_);
            const float cc = __fmaf_rn(dy, __fmaf_rn(r1.x, dy, f_), dzh);
            const float2 b2 = f2(bb), c2 = f2(cc);
            const float4* gp = s_g + sbt * GBLK + (yr + SY * zs) * HALF;
            float2 R0 = make_float2(0.f, 0.f), R1 = R0;
#pragma unroll
            for (int q = 0; q < HALF; ++q) {
                const float4 gv = gp[q];
                const float2 t = __ffma2_rn(dx[q], __ffma2_rn(qxx, dx[q], b2), c2);
                float2 G;
                G.x = t.x > T ? ex2_approx(t.x) : 0.f;
                G.y = t.y > T ? ex2_approx(t.y) : 0.f;
                const float2 gn = make_float2(gv.x, gv.y);
                const float2 h = __fmul2_rn(G, __ffma2_rn(amp, gn, make_float2(gv.z, gv.w)));
                A = __ffma2_rn(G, gn, A);
                R0 = __fadd2_rn(R0, h);
                const float X0 = (float)(2 * q), X1 = (float)(2 * q + 1);
                R1 = __ffma2_rn(h, make_float2(X0, X1), R1);
                R2 = __ffma2_rn(h, make_float2(X0 * X0, X1 * X1), R2);
            }
            const float r0s = R0.x + R0.y, r1s = R1.x + R1.y;
            const float dyr0 = dy * r0s;
            S1y = fmaf(dy, r0s, S1y);
            Sxy = fmaf(dy, r1s, Sxy);
            Syy = fmaf(dy, dyr0, Syy);
            T0 += r0s;
            T1 += r1s;
            Ty += dyr0;
        }
        S0 += T0;
        S1x += T1;
        S1z = fmaf(dz, T0, S1z);
        Sxz = fmaf(dz, T1, Sxz);
        Syz = fmaf(dz, Ty, Syz);
        Szz = fmaf(dz * dz, T0, Szz);
    }
    const float del = __fsub_rn(fxb, r0.x);
    float* sa = s_acc + j * kAccStride;
    atomicAdd(sa + 0, A.x + A.y);
    atomicAdd(sa + 1, S0);
    atomicAdd(sa + 2, fmaf(del, S0, S1x));
    atomicAdd(sa + 3, S1y);
    atomicAdd(sa + 4, S1z);
    atomicAdd(sa + 5, fmaf(del, fmaf(del, S0, 2.f * S1x), R2.x + R2.y));
    atomicAdd(sa + 6, Syy);
    atomicAdd(sa + 7, Szz);
    atomicAdd(sa + 8, fmaf(del, S1y, Sxy));
    atomicAdd(sa + 9, fmaf(del, S1z, Sxz));
    atomicAdd(sa + 10, Syz);
}

// The fused evaluation of one brick (all threads of the CTA take part; the
// shared arrays are the CTA's).  Launched one CTA per brick by k_brick, and
// in a loop over the bricks of many volumes by the batched kernel.
template <int MODE, int B, int CH>
__device__ __forceinline__ void brick_body(const BrickArgs& a, const unsigned brick)
{
    using S = BrickShape<B>;
    constexpr int NT = S::THREADS, NW = S::NW, HALF = S::HALF, SY = S::SY, SZ = S::SZ;
    constexpr int CPT = 8 * CH / NT;  // compaction candidates per thread
    static_assert(CPT >= 1 && CPT <= 32, "candidates per thread");
    if (a.st->overflow) return;
    __shared__ float4 s_rec[CH * 3];
    __shared__ uint32_t s_msk[CH];
    // per row: HALF x (gn[x], gn[x+1], gd[x], gd[x+1]), stored sub-brick by
    // sub-brick in blocks of GBLK float4 (one of padding), so that lanes
    // reading the same position in different sub-bricks hit different banks
    constexpr int GBLK = SY * SZ * HALF + 1;
    __shared__ float4 s_g[8 * GBLK];
    __shared__ float s_acc[CH * kAccStride];
    __shared__ uint16_t s_task[CH * 8];
    __shared__ int s_scan[NW];
    __shared__ float s_red[2][NW];
    __shared__ unsigned long long s_cnt[3][NW];
    __shared__ __align__(16) float s_v[(MODE == kModeLoss || MODE == kModeBwd) ? S::ROWS * B : 4];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BinGeom& g = a.g;
    const int bx = (int)(brick % g.nbx);
    const int by = (int)((brick / g.nbx) % g.nby);
    const int bz = (int)(brick / ((long long)g.nbx * g.nby));
    const uint32_t s0 = a.start[brick];
    const int L = (int)(a.end[brick] - s0);
    const float T = a.T;

    // ---------------- phase 1: lane = row of B voxels ----------------
    const bool has_row = tid < S::ROWS;
    const int row = has_row ? tid : 0;
    const int ly = row % B, lz = row / B;
    const int gy = by * B + ly, gz = bz * B + lz, gx0 = bx * B;
    const bool rowin = has_row && gy < g.ny && gz < g.nz;
    const int nxin = rowin ? min(B, g.nx - gx0) : 0;  // in-grid voxels of the row
    const float fy = (float)gy, fz = (float)gz;
    if (MODE == kModeLoss || MODE == kModeBwd) {
        // the row's target (loss) or upstream (backward) values travel to
        // shared memory while the forward phase runs
        if (nxin > 0) {
            const float* src = (MODE == kModeLoss ? a.field : a.upstream) + (((size_t)gz * g.ny + gy) * g.nx + gx0);
            float* dst = s_v + row * B;
            if (nxin == B && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
#pragma unroll
                for (int x = 0; x < B; x += 4) cp_async16(dst + x, src + x);
            } else {
                for (int x = 0; x < nxin; ++x) cp_async4(dst + x, src + x);
            }
        }
    }
    // sub-brick bits (bit = y half + 2 * z quarter) covering this warp's rows
    uint32_t wmask = 0;
    {
        const int z0 = (32 * warp) / B, z1 = min(B - 1, (32 * warp + 31) / B);
        for (int q = z0 / SZ; q <= z1 / SZ; ++q) wmask |= 3u << (2 * q);
    }
    float2 num[HALF], den[HALF];
#pragma unroll
    for (int q = 0; q < HALF; ++q) { num[q] = make_float2(0.f, 0.f); den[q] = num[q]; }
    unsigned long long kept = 0, live = 0;
    const int nchunks = (L + CH - 1) / CH;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int c0 = ch * CH;
        const int cnt = min(CH, L - c0);
        if (ch > 0) __syncthreads();
        stage_chunk<NT, CH>(a, s0, c0, cnt, s_rec, s_msk, tid);
        __syncthreads();
        // the warp's live Gaussians of this chunk, two at a time (list order kept)
        for (int base = 0; base < cnt; base += 32) {
            const int jl = base + lane;
            uint32_t bal = __ballot_sync(0xffffffffu, jl < cnt && (s_msk[jl] & wmask));
            while (bal) {
                const int j1 = base + __ffs(bal) - 1;
                bal &= bal - 1;
                const bool two = bal != 0;
                const int j2 = two ? base + __ffs(bal) - 1 : j1;
                if (two) bal &= bal - 1;
                const float4 r0 = s_rec[3 * j1], r1 = s_rec[3 * j1 + 1], r2 = s_rec[3 * j1 + 2];
                const float4 u0 = s_rec[3 * j2], u1 = s_rec[3 * j2 + 1], u2 = s_rec[3 * j2 + 2];
                const float dy = __fsub_rn(fy, r0.y), dz = __fsub_rn(fz, r0.z);
                const float b = __fmaf_rn(r1.z, dy, __fmul_rn(r1.w, dz));
                const float c = __fmaf_rn(dy, __fmaf_rn(r1.x, dy, __fmul_rn(r2.x, dz)), __fmul_rn(dz, __fmul_rn(r1.y, dz)));
                const float ey = __fsub_rn(fy, u0.y), ez = __fsub_rn(fz, u0.z);
                const float bu = __fmaf_rn(u1.z, ey, __fmul_rn(u1.w, ez));
                const float cu = __fmaf_rn(ey, __fmaf_rn(u1.x, ey, __fmul_rn(u2.x, ez)), __fmul_rn(ez, __fmul_rn(u1.y, ez)));
                const float2 nmu = f2(-r0.x), qxx = f2(r0.w), b2 = f2(b), c2 = f2(c), al = f2(r2.y), be = f2(r2.z);
                const float2 nmv = f2(-u0.x), qxv = f2(u0.w), bv = f2(bu), cv = f2(cu);
                const float2 alv = f2(two ? u2.y : 0.f), bev = f2(two ? u2.z : 0.f);
#pragma unroll
                for (int q = 0; q < HALF; ++q) {
                    const float2 xq = make_float2((float)(gx0 + 2 * q), (float)(gx0 + 2 * q + 1));
                    const float2 dx = __fadd2_rn(xq, nmu);
                    const float2 t = __ffma2_rn(dx, __ffma2_rn(qxx, dx, b2), c2);
                    const float2 dv = __fadd2_rn(xq, nmv);
                    const float2 tv = __ffma2_rn(dv, __ffma2_rn(qxv, dv, bv), cv);
                    float2 G, H;
                    G.x = t.x > T ? ex2_approx(t.x) : 0.f;
                    G.y = t.y > T ? ex2_approx(t.y) : 0.f;
                    H.x = tv.x > T ? ex2_approx(tv.x) : 0.f;
                    H.y = tv.y > T ? ex2_approx(tv.y) : 0.f;
                    if (MODE == kModeCount) {
                        kept += (unsigned)((t.x > T) && (2 * q < nxin)) + (unsigned)((t.y > T) && (2 * q + 1 < nxin));
                        if (two)
                            kept += (unsigned)((tv.x > T) && (2 * q < nxin)) + (unsigned)((tv.y > T) && (2 * q + 1 < nxin));
                        if (a.pairs) {  // the kept pairs themselves: (voxel << 24) | Gaussian
                            const unsigned long long v0 = ((unsigned long long)gz * g.ny + gy) * g.nx + gx0 + 2 * q;
                            const unsigned long long i1 = a.gids[s0 + c0 + j1] & kGidMask;
                            const unsigned long long i2 = a.gids[s0 + c0 + j2] & kGidMask;
                            const bool kk[4] = {t.x > T && 2 * q < nxin, t.y > T && 2 * q + 1 < nxin,
                                                two && tv.x > T && 2 * q < nxin, two && tv.y > T && 2 * q + 1 < nxin};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if (!kk[e]) continue;
                                const unsigned long long pos = atomicAdd(&a.st->listed, 1ull);
                                if (pos < a.pairs_cap)
                                    a.pairs[pos] = ((v0 + (e & 1)) << kGidBits) | (e < 2 ? i1 : i2);
                            }
                        }
                    }
                    num[q] = __ffma2_rn(al, G, num[q]);
                    den[q] = __ffma2_rn(be, G, den[q]);
                    num[q] = __ffma2_rn(alv, H, num[q]);
                    den[q] = __ffma2_rn(bev, H, den[q]);
                }
                if (MODE == kModeCount) live += (unsigned long long)nxin * (two ? 2u : 1u);
            }
        }
    }

    if (MODE == kModeCount) {
        // backward candidates: in-grid voxels of every live sub-brick
        unsigned long long cand2 = 0;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int c0 = ch * CH;
            const int cnt = min(CH, L - c0);
            for (int j = tid; j < cnt; j += NT) {
                const uint32_t m = a.gids[s0 + c0 + j] >> kGidBits;
                for (int sb = 0; sb < 8; ++sb) {
                    if (!((m >> sb) & 1u)) continue;
                    const int y0 = by * B + SY * (sb & 1), z0 = bz * B + SZ * (sb >> 1);
                    const long long vx = min(B, g.nx - gx0), vy = max(0, min(SY, g.ny - y0)),
                                    vz = max(0, min(SZ, g.nz - z0));
                    cand2 += (unsigned long long)(vx * vy * vz);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kept += __shfl_xor_sync(0xffffffffu, kept, o);
            live += __shfl_xor_sync(0xffffffffu, live, o);
            cand2 += __shfl_xor_sync(0xffffffffu, cand2, o);
        }
        if (lane == 0) { s_cnt[0][warp] = kept; s_cnt[1][warp] = live; s_cnt[2][warp] = cand2; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long k = 0, c = 0;
            for (int w = 0; w < NW; ++w) { k += s_cnt[0][w]; c += s_cnt[1][w] + s_cnt[2][w]; }
            atomicAdd(&a.st->kept, k);
            atomicAdd(&a.st->cand, c);
        }
        return;
    }

    const float rho0 = a.rho0;
    const size_t vrow = ((size_t)gz * g.ny + gy) * g.nx + gx0;
    float up[B], vt[B], inv[B];
    if (MODE == kModeEval) {
        // the field handed to the caller: Eq. 3 with a correctly rounded division
#pragma unroll
        for (int q = 0; q < HALF; ++q) {
            vt[2 * q] = a.normalized ? num[q].x / fmaxf(den[q].x, rho0) : num[q].x;
            vt[2 * q + 1] = a.normalized ? num[q].y / fmaxf(den[q].y, rho0) : num[q].y;
        }
#pragma unroll
        for (int x = 0; x < B; ++x)
            if (x < nxin) a.field_out[vrow + x] = vt[x];
        return;
    }
    // loss and backward: one reciprocal of max(den, rho0) per voxel serves
    // Vtilde = num / den' and gn = up / den' (rcp.approx: within 1 ulp)
#pragma unroll
    for (int q = 0; q < HALF; ++q) {
        inv[2 * q] = a.normalized ? rcp_approx(fmaxf(den[q].x, rho0)) : 1.f;
        inv[2 * q + 1] = a.normalized ? rcp_approx(fmaxf(den[q].y, rho0)) : 1.f;
        vt[2 * q] = num[q].x * inv[2 * q];
        vt[2 * q + 1] = num[q].y * inv[2 * q + 1];
    }
    cp_async_wait_all();
    const float* sv = s_v + (MODE == kModeLoss || MODE == kModeBwd ? row * B : 0);
    if (MODE == kModeLoss) {
        float ef = 0.f, el = 0.f;
#pragma unroll
        for (int x = 0; x < B; ++x) {
            const float V = x < nxin ? sv[x] : 0.f;
            const float r = x < nxin ? vt[x] - V : 0.f;
            const float rl = (a.mask_thresh < 0.f || V > a.mask_thresh) ? r : 0.f;
            ef = fmaf(r, r, ef);
            el = fmaf(rl, rl, el);
            up[x] = 2.f * rl * a.inv_m;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ef += __shfl_xor_sync(0xffffffffu, ef, o);
            el += __shfl_xor_sync(0xffffffffu, el, o);
        }
        if (lane == 0) { s_red[0][warp] = el; s_red[1][warp] = ef; }
    } else {  // kModeBwd
#pragma unroll
        for (int x = 0; x < B; ++x) up[x] = x < nxin ? sv[x] : 0.f;
    }
    // the upstream terms of the backward, only when the gradient is wanted
    // (a forward-only loss evaluation has no sums to fill)
    if (has_row && a.acc != nullptr && L > 0) {
#pragma unroll
        for (int q = 0; q < HALF; ++q) {
            float gn0, gd0, gn1, gd1;
            gn0 = up[2 * q] * inv[2 * q];
            gn1 = up[2 * q + 1] * inv[2 * q + 1];
            if (a.normalized) {
                gd0 = den[q].x >= rho0 ? -vt[2 * q] * gn0 : 0.f;
                gd1 = den[q].y >= rho0 ? -vt[2 * q + 1] * gn1 : 0.f;
            } else {
                gd0 = 0.f; gd1 = 0.f;
            }
            s_g[(ly / SY + 2 * (lz / SZ)) * GBLK + (ly % SY + SY * (lz % SZ)) * HALF + q] =
                make_float4(gn0, gn1, gd0, gd1);
        }
    }
    __syncthreads();
    if (MODE == kModeLoss && tid == 0) {
        float el = 0.f, ef = 0.f;
        for (int w = 0; w < NW; ++w) { el += s_red[0][w]; ef += s_red[1][w]; }
        a.part[brick] = make_float2(el, ef);
    }
    if (a.acc == nullptr || L == 0) return;

    // ---------------- phase 2: compacted (Gaussian, sub-brick) tasks ----------------
    const float fxb = (float)gx0;
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        const int c0 = ch * CH;
        const int cnt = min(CH, L - c0);
        if (ch != nchunks - 1) {
            __syncthreads();
            stage_chunk<NT, CH>(a, s0, c0, cnt, s_rec, s_msk, tid);
            __syncthreads();
        }
        // candidates c = sub-brick * CH + j: tasks come out sub-brick-major,
        // Gaussian-ascending
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = tid * CPT + k;
            const int sb = c / CH, j = c % CH;
            if (j < cnt && ((s_msk[j] >> sb) & 1u)) bits |= 1u << k;
        }
        const int mine = __popc(bits);
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_scan[warp] = incl;
        for (int j = tid; j < cnt * kAccStride; j += NT) s_acc[j] = 0.f;
        __syncthreads();
        int ntask = 0, woff = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            woff += w < warp ? s_scan[w] : 0;
            ntask += s_scan[w];
        }
        int pos = woff + incl - mine;
        while (bits) {
            const int k = __ffs(bits) - 1;
            bits &= bits - 1;
            const int c = tid * CPT + k;
            s_task[pos++] = (uint16_t)((c % CH) | ((c / CH) << 8));
        }
        __syncthreads();

        // whole tasks in rounds of NT; a last round of at most 16 tasks is
        // taken by one warp as twice as many half tasks (SZ / 2 slices each)
        const int full = ntask - ntask % NT, rem = ntask - full;
        const bool split = SZ >= 2 && rem > 0 && 2 * rem <= 32;
        const bool split2x = SZ >= 2 && NT >= 64 && rem > 16 && rem <= 32;
        for (int tk = tid; tk < (split || split2x ? full : ntask); tk += NT) {
            const int task = s_task[tk];
            task_sums<B, SZ>(s_rec, s_g, s_acc, task & 255, task >> 8, 0, by, bz, fxb, T);
        }
        // a last round of 17 to 32 tasks: each of two warps takes one half of
        // every task
        const bool split2 = SZ >= 2 && NT >= 64 && rem > 16 && rem <= 32;
        const bool half = (split && tid < 2 * rem) || (split2 && tid < 64 && (tid & 31) < rem);
        if (SZ >= 2 && half) {
            const int k = split ? tid % rem : (tid & 31), h = split ? tid / rem : (tid >> 5);
            const int task = s_task[full + k];
            task_sums<B, (SZ >= 2 ? SZ / 2 : 1)>(s_rec, s_g, s_acc, task & 255, task >> 8, h * (SZ / 2), by, bz, fxb,
                                                  T);
        }
        __syncthreads();
        for (int j = tid; j < cnt; j += NT) {
            if (s_msk[j] == 0) continue;
            const float* sa = s_acc + j * kAccStride;
            const uint32_t gid = a.gids[s0 + c0 + j] & kGidMask;
            float* dst = a.acc + 12 * (size_t)gid;
            red_add_v4(dst, sa[0], sa[1], sa[2], sa[3]);
            red_add_v4(dst + 4, sa[4], sa[5], sa[6], sa[7]);
            red_add_v4(dst + 8, sa[8], sa[9], sa[10], 0.f);
        }
    }
}

template <int MODE, int B, int CH>
__global__ void __launch_bounds__(BrickShape<B>::THREADS, BrickShape<B>::MINB) k_brick(const BrickArgs a)
{
    brick_body<MODE, B, CH>(a, blockIdx.x);
}

template <int B, int CH>
static void launch_brick_bc(int mode, const BrickArgs& a, cudaStream_t s)
{
    const unsigned grid = (unsigned)a.g.nbricks;
    constexpr int NT = BrickShape<B>::THREADS;
    switch (mode) {
        case kModeEval: k_brick<kModeEval, B, CH><<<grid, NT, 0, s>>>(a); break;
        case kModeLoss: k_brick<kModeLoss, B, CH><<<grid, NT, 0, s>>>(a); break;
        case kModeBwd: k_brick<kModeBwd, B, CH><<<grid, NT, 0, s>>>(a); break;
        default: k_brick<kModeCount, B, CH><<<grid, NT, 0, s>>>(a); break;
    }
}

void launch_brick(int mode, const BrickArgs& a, cudaStream_t s)
{
    const int B = a.g.B;
    const bool c32 = a.chunk == 32;
    if (B == 4) {
        if (c32) launch_brick_bc<4, 32>(mode, a, s); else launch_brick_bc<4, 64>(mode, a, s);
    } else if (B == 16) {
        if (c32) launch_brick_bc<16, 32>(mode, a, s); else launch_brick_bc<16, 64>(mode, a, s);
    } else {
        if (c32) launch_brick_bc<8, 32>(mode, a, s); else launch_brick_bc<8, 64>(mode, a, s);
    }
}

// ------------------------------------------------------------------------
// batched persistent iteration
// ------------------------------------------------------------------------
// Grid barrier of a cooperative launch with a bounded wait: thread 0 of each
// CTA arrives on a counter; the last arrival resets it and advances the
// generation, the others sleep until the generation moves or `limit` sleeps
// pass, in which case the error flag is set.  Returns false (for the whole
// CTA) when the wait ran out.
__device__ __forceinline__ bool grid_barrier(BatchState* bs, unsigned expect, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &bs->bar_gen;
        const unsigned g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&bs->bar_count, 1u) + 1u == expect) {
            atomicExch(&bs->bar_count, 0u);
            __threadfence();
            atomicAdd(&bs->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > limit) {
                    ok = 0;
                    atomicExch(&bs->err, 1);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// the chain rule out of line: its register needs stay out of the brick body's
__device__ __noinline__ void chain_one_call(const long long i, const BatchIterArgs& p)
{
    chain_one(i, p.acc, p.acc, p.prims, p.grad, p.m, p.v, p.ad, p.do_adam, nullptr);
}

template <int B, int CH>
__global__ void __launch_bounds__(BrickShape<B>::THREADS, BrickShape<B>::MINB) k_batch_iter(const BatchIterArgs p)
{
    constexpr int NT = BrickShape<B>::THREADS;
    __shared__ unsigned long long s_gb;
    __shared__ double s_red[2][NT / 32 > 0 ? NT / 32 : 1];
    BatchState* bs = p.bs;
    // an earlier wait ran out, or the pairs overflowed: nothing runs
    if (*(volatile int*)&bs->err || p.va[0].st->overflow) return;

    // phase 1: the bricks of every volume from one work counter
    for (;;) {
        if (threadIdx.x == 0) s_gb = atomicAdd(&bs->next, 1ull);
        __syncthreads();
        const unsigned long long gb = s_gb;
        if (gb >= (unsigned long long)p.nbricks) break;
        int lo = 0, hi = p.nvol - 1;   // the volume holding global brick gb
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.boff[mid] <= (long long)gb) lo = mid; else hi = mid - 1;
        }
        brick_body<kModeLoss, B, CH>(p.va[lo], (unsigned)(gb - (unsigned long long)p.boff[lo]));
        __syncthreads();
    }
    if (!grid_barrier(bs, p.expect, p.spin_limit)) return;

    // phase 2a: each volume's SSE in a fixed order: every chunk of kSseChunk
    // bricks is summed by one CTA; the last CTA past its chunks adds each
    // volume's chunk sums in chunk order
    __shared__ int s_last;
    for (long long ch = blockIdx.x; ch < p.nchunks; ch += gridDim.x) {
        int v = 0, hi = p.nvol - 1;
        while (v < hi) {
            const int mid = (v + hi + 1) >> 1;
            if (p.coff[mid] <= ch) v = mid; else hi = mid - 1;
        }
        const long long nb = p.boff[v + 1] - p.boff[v];
        const long long b0 = (ch - p.coff[v]) * kSseChunk;
        const long long b1 = b0 + kSseChunk < nb ? b0 + kSseChunk : nb;
        const float2* part = p.va[v].part;
        double x = 0.0, y = 0.0;
        for (long long i = b0 + threadIdx.x; i < b1; i += NT) {
            const float2 q = part[i];
            x += (double)q.x;
            y += (double)q.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = x; s_red[1][threadIdx.x >> 5] = y; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, c = 0.0;
            for (int w = 0; w < NT / 32; ++w) { a += s_red[0][w]; c += s_red[1][w]; }
            p.csum[ch] = make_double2(a, c);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&bs->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int v = threadIdx.x; v < p.nvol; v += NT) {
            double a = 0.0, c = 0.0;
            for (long long ch = p.coff[v]; ch < p.coff[v + 1]; ++ch) {
                const volatile double* q = reinterpret_cast<const volatile double*>(p.csum + ch);
                a += q[0];
                c += q[1];
            }
            p.sse[2 * v] = a;
            p.sse[2 * v + 1] = c;
            if (p.trace) p.trace[(size_t)bs->it * p.nvol + v] = a * p.inv_m[v];
        }
        if (threadIdx.x == 0) bs->done = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bs->next = 0;   // every CTA is past phase 1
    // phase 2b: chain rule and Adam (or the gradient) of every Gaussian
    const long long stride = (long long)gridDim.x * NT;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < p.ntot; i += stride) chain_one_call(i, p);
}

template <int B, int CH>
static int batch_grid_bc()
{
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_iter<B, CH>, BrickShape<B>::THREADS, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * num_sms();
}

int batch_iter_grid(int B, int CH)
{
    const bool c32 = CH == 32;
    if (B == 4) return c32 ? batch_grid_bc<4, 32>() : batch_grid_bc<4, 64>();
    if (B == 16) return c32 ? batch_grid_bc<16, 32>() : batch_grid_bc<16, 64>();
    return c32 ? batch_grid_bc<8, 32>() : batch_grid_bc<8, 64>();
}

template <int B, int CH>
static cudaError_t launch_batch_bc(const BatchIterArgs& p, unsigned grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BrickShape<B>::THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_iter<B, CH>, p);
}

cudaError_t launch_batch_iter(int B, int CH, const BatchIterArgs& p, unsigned grid, cudaStream_t s)
{
    const bool c32 = CH == 32;
    if (B == 4) return c32 ? launch_batch_bc<4, 32>(p, grid, s) : launch_batch_bc<4, 64>(p, grid, s);
    if (B == 16) return c32 ? launch_batch_bc<16, 32>(p, grid, s) : launch_batch_bc<16, 64>(p, grid, s);
    return c32 ? launch_batch_bc<8, 32>(p, grid, s) : launch_batch_bc<8, 64>(p, grid, s);
}

// ------------------------------------------------------------------------
// deterministic SSE reduction: contiguous chunks per block, then one block
// ------------------------------------------------------------------------
constexpr int kRedBlocks = 592;

__global__ void __launch_bounds__(256) k_sse_partial(const float2* __restrict__ part, long long nb,
                                                     double2* __restrict__ out, const DevState* st)
{
    if (st->overflow) return;
    __shared__ double sm[2][8];
    long long chunk = (nb + gridDim.x - 1) / gridDim.x;
    long long b0 = (long long)blockIdx.x * chunk, b1 = min(nb, b0 + chunk);
    double x = 0.0, y = 0.0;
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const float2 p = part[i];
        x += (double)p.x;
        y += (double)p.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = x; sm[1][threadIdx.x >> 5] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += sm[0][w]; b += sm[1][w]; }
        out[blockIdx.x] = make_double2(a, b);
    }
}

__global__ void __launch_bounds__(1024) k_sse_final(const double2* __restrict__ in, int nin, DevState* st,
                                                    double* trace, int iter, double inv_m, const int* iter_dev,
                                                    int trace_stride, int trace_col)
{
    if (st->overflow) return;
    __shared__ double sm[2][32];
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < nin; i += blockDim.x) { x += in[i].x; y += in[i].y; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = x; sm[1][threadIdx.x >> 5] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 32; ++w) { a += sm[0][w]; b += sm[1][w]; }
        st->sse[0] = a;
        st->sse[1] = b;
        if (trace) trace[iter_dev ? (size_t)(*iter_dev) * trace_stride + trace_col : (size_t)iter] = a * inv_m;
    }
}

void launch_sse_reduce(const float2* part, long long nbricks, DevState* st, double* trace, int iter,
                       double inv_m, cudaStream_t s, const int* iter_dev, int trace_stride, int trace_col)
{
    // the partial buffer past the bricks' sums (16-byte aligned) is scratch
    // for the block sums
    const uintptr_t end = reinterpret_cast<uintptr_t>(part + nbricks);
    double2* tmp = reinterpret_cast<double2*>((end + 15) & ~static_cast<uintptr_t>(15));
    k_sse_partial<<<kRedBlocks, 256, 0, s>>>(part, nbricks, tmp, st);
    k_sse_final<<<1, 1024, 0, s>>>(tmp, kRedBlocks, st, trace, iter, inv_m, iter_dev, trace_stride, trace_col);
}

}  // namespace gve
