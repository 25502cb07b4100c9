// field.cu -- the brick evaluator: Eq. 3 forward, residual and SSE, and the
// backward of the mean squared error, fused per brick of 8^3 voxels.
//
// One CTA (256 threads) per brick.  The brick's Gaussian list is staged in
// shared memory in chunks of kChunk prepared records (3 x float4 each).
//
// Phase 1 (forward, one thread per voxel pair along x): for every listed
// Gaussian, the keep exponent t is evaluated by the fixed float32 chain
//     dy = y - mu_y, dz = z - mu_z, dx = x - mu_x,
//     b = fma(qxy2, dy, qxz2*dz), c = fma(dy, fma(qyy, dy, qyz2*dz), dz*(qzz*dz)),
//     t = fma(dx, fma(qxx, dx, b), c)
// (q.. = -0.5 log2(e) Sigma^-1), the pair is kept iff t > T, and G = 2^t on
// the SFU (ex2.approx).  num += w a G, den += w G; Vtilde = num/max(den,rho0)
// (Eq. 3).  Residual r = Vtilde - V, SSE partial per brick in FP64.  The
// upstream gradient of the loss gives per voxel
//     gn = dL/dnum = up / max(den, rho0),   gd = dL/dden = -Vtilde gn (den >= rho0)
// stored in shared memory.
//
// Phase 2 (backward, one 8-lane group per Gaussian, one lane per z-slice of
// the brick): each lane walks the 64 voxels of its slice, recomputes G by the
// same chain, and accumulates
//     A = sum G gn,  Bs = sum G gd,  S1 = sum h d,  S2 = sum h d d^T,
//     h = G (alpha gn + beta gd)        (S1, S2 scaled by -1/2 later)
// with the per-row factorisation of the x-dependence; the 8 lanes reduce by
// shuffles and one lane issues three 16-byte vector atomics into the
// Gaussian's accumulator.  Nothing per pair or per voxel goes to HBM.
#include "gve_int.cuh"

namespace gve {

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(kBrickThreads, 3) k_brick(const BrickArgs a)
{
    if (a.st->overflow) return;
    __shared__ float4 s_rec[kChunk * 3];
    __shared__ float4 s_g[8 * 33];
    __shared__ double s_red[2][8];
    __shared__ unsigned s_cnt[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BinGeom& g = a.g;
    const long long brick = blockIdx.x;
    const int bx = (int)(brick % g.nbx);
    const int by = (int)((brick / g.nbx) % g.nby);
    const int bz = (int)(brick / ((long long)g.nbx * g.nby));
    const uint32_t s0 = a.start[brick];
    const int L = (int)(a.end[brick] - s0);
    const float T = a.T;

    // ---------------- phase 1: forward over (x, x+1), y, z ----------------
    const int xp = tid & 3, ly = (tid >> 2) & 7, lz = tid >> 5;
    const int gx = bx * 8 + 2 * xp, gy = by * 8 + ly, gz = bz * 8 + lz;
    const bool rowin = gy < g.ny && gz < g.nz;
    const bool in0 = rowin && gx < g.nx, in1 = rowin && gx + 1 < g.nx;
    const float fx0 = (float)gx, fx1 = (float)(gx + 1), fy = (float)gy, fz = (float)gz;
    float num0 = 0.f, den0 = 0.f, num1 = 0.f, den1 = 0.f;
    unsigned kept = 0;
    const int nchunks = (L + kChunk - 1) / kChunk;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int c0 = ch * kChunk;
        const int cnt = min(kChunk, L - c0);
        if (ch > 0) __syncthreads();
        for (int j = tid; j < cnt * 3; j += kBrickThreads) {
            const uint32_t gid = a.gids[s0 + c0 + j / 3];
            s_rec[j] = a.rec[3 * (size_t)gid + (j % 3)];
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float4 r0 = s_rec[3 * j], r1 = s_rec[3 * j + 1], r2 = s_rec[3 * j + 2];
            const float dy = __fsub_rn(fy, r0.y), dz = __fsub_rn(fz, r0.z);
            const float b = __fmaf_rn(r1.z, dy, __fmul_rn(r1.w, dz));
            const float c = __fmaf_rn(dy, __fmaf_rn(r1.x, dy, __fmul_rn(r2.x, dz)), __fmul_rn(dz, __fmul_rn(r1.y, dz)));
            const float dx0 = __fsub_rn(fx0, r0.x), dx1 = __fsub_rn(fx1, r0.x);
            const float t0 = __fmaf_rn(dx0, __fmaf_rn(r0.w, dx0, b), c);
            const float t1 = __fmaf_rn(dx1, __fmaf_rn(r0.w, dx1, b), c);
            const float G0 = t0 > T ? ex2_approx(t0) : 0.f;
            const float G1 = t1 > T ? ex2_approx(t1) : 0.f;
            if (MODE == kModeCount) kept += (unsigned)((t0 > T) && in0) + (unsigned)((t1 > T) && in1);
            num0 = fmaf(r2.y, G0, num0);
            den0 = fmaf(r2.z, G0, den0);
            num1 = fmaf(r2.y, G1, num1);
            den1 = fmaf(r2.z, G1, den1);
        }
    }

    if (MODE == kModeCount) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
        if (lane == 0) s_cnt[warp] = kept;
        __syncthreads();
        if (tid == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < 8; ++w) tot += s_cnt[w];
            long long vx = min(8, g.nx - bx * 8), vy = min(8, g.ny - by * 8), vz = min(8, g.nz - bz * 8);
            atomicAdd(&a.st->kept, tot);
            atomicAdd(&a.st->cand, (unsigned long long)L * (unsigned long long)(vx * vy * vz));
        }
        return;
    }

    const float rho0 = a.rho0;
    const float vt0 = a.normalized ? num0 / fmaxf(den0, rho0) : num0;
    const float vt1 = a.normalized ? num1 / fmaxf(den1, rho0) : num1;
    const size_t v0 = ((size_t)gz * g.ny + gy) * g.nx + gx;
    if (MODE == kModeEval) {
        if (in0) a.field_out[v0] = vt0;
        if (in1) a.field_out[v0 + 1] = vt1;
        return;
    }

    float up0 = 0.f, up1 = 0.f;
    if (MODE == kModeLoss) {
        const float V0 = in0 ? a.field[v0] : 0.f;
        const float V1 = in1 ? a.field[v0 + 1] : 0.f;
        const float r0 = in0 ? vt0 - V0 : 0.f;
        const float r1 = in1 ? vt1 - V1 : 0.f;
        const bool m0 = a.mask_thresh < 0.f || V0 > a.mask_thresh;
        const bool m1 = a.mask_thresh < 0.f || V1 > a.mask_thresh;
        const float rl0 = m0 ? r0 : 0.f, rl1 = m1 ? r1 : 0.f;
        double ef = (double)r0 * r0 + (double)r1 * r1;
        double el = (double)rl0 * rl0 + (double)rl1 * rl1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ef += __shfl_xor_sync(0xffffffffu, ef, o);
            el += __shfl_xor_sync(0xffffffffu, el, o);
        }
        if (lane == 0) { s_red[0][warp] = el; s_red[1][warp] = ef; }
        up0 = 2.f * rl0 * a.inv_m;
        up1 = 2.f * rl1 * a.inv_m;
    } else {  // kModeBwd
        up0 = in0 ? a.upstream[v0] : 0.f;
        up1 = in1 ? a.upstream[v0 + 1] : 0.f;
    }
    float gn0, gd0, gn1, gd1;
    if (a.normalized) {
        gn0 = up0 / fmaxf(den0, rho0);
        gn1 = up1 / fmaxf(den1, rho0);
        gd0 = den0 >= rho0 ? -vt0 * gn0 : 0.f;
        gd1 = den1 >= rho0 ? -vt1 * gn1 : 0.f;
    } else {
        gn0 = up0; gn1 = up1; gd0 = 0.f; gd1 = 0.f;
    }
    s_g[33 * lz + 4 * ly + xp] = make_float4(gn0, gd0, gn1, gd1);
    __syncthreads();
    if (MODE == kModeLoss && tid == 0) {
        double el = 0.0, ef = 0.0;
        for (int w = 0; w < 8; ++w) { el += s_red[0][w]; ef += s_red[1][w]; }
        a.part[brick] = make_double2(el, ef);
    }
    if (a.acc == nullptr || L == 0) return;

    // ---------------- phase 2: backward, 8-lane group per Gaussian ----------------
    const int sl = lane & 7, gs = lane >> 3;
    const unsigned gmask = 0xffu << (8 * gs);
    const float fzs = (float)(bz * 8 + sl);
    const float fyb = (float)(by * 8), fxb = (float)(bx * 8);
    // the last chunk of phase 1 is still staged; walk the chunks backwards
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        const int c0 = ch * kChunk;
        const int cnt = min(kChunk, L - c0);
        if (ch != nchunks - 1) {
            __syncthreads();
            for (int j = tid; j < cnt * 3; j += kBrickThreads) {
                const uint32_t gid = a.gids[s0 + c0 + j / 3];
                s_rec[j] = a.rec[3 * (size_t)gid + (j % 3)];
            }
            __syncthreads();
        }
        for (int jr = warp * 4 + gs; jr < cnt; jr += 32) {
            const float4 r0 = s_rec[3 * jr], r1 = s_rec[3 * jr + 1], r2 = s_rec[3 * jr + 2];
            float dxv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) dxv[k] = __fsub_rn(fxb + (float)k, r0.x);
            const float dz = __fsub_rn(fzs, r0.z);
            const float e_ = __fmul_rn(r1.w, dz), f_ = __fmul_rn(r2.x, dz);
            const float dzh = __fmul_rn(dz, __fmul_rn(r1.y, dz));
            float A = 0.f, Bs = 0.f, S1x = 0.f, S1y = 0.f, S1z = 0.f;
            float Sxx = 0.f, Syy = 0.f, Szz = 0.f, Sxy = 0.f, Sxz = 0.f, Syz = 0.f;
#pragma unroll 2
            for (int y = 0; y < 8; ++y) {
                const float dy = __fsub_rn(fyb + (float)y, r0.y);
                const float b = __fmaf_rn(r1.z, dy, e_);
                const float c = __fmaf_rn(dy, __fmaf_rn(r1.x, dy, f_), dzh);
                float R0 = 0.f, R1 = 0.f, R2 = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 gv = s_g[33 * sl + 4 * y + q];
                    {
                        const float dx = dxv[2 * q];
                        const float t = __fmaf_rn(dx, __fmaf_rn(r0.w, dx, b), c);
                        const float G = t > T ? ex2_approx(t) : 0.f;
                        const float Ggn = G * gv.x, Ggd = G * gv.y;
                        A += Ggn;
                        Bs += Ggd;
                        const float h = fmaf(r2.y, Ggn, r2.z * Ggd);
                        R0 += h;
                        const float hx = h * dx;
                        R1 += hx;
                        R2 = fmaf(hx, dx, R2);
                    }
                    {
                        const float dx = dxv[2 * q + 1];
                        const float t = __fmaf_rn(dx, __fmaf_rn(r0.w, dx, b), c);
                        const float G = t > T ? ex2_approx(t) : 0.f;
                        const float Ggn = G * gv.z, Ggd = G * gv.w;
                        A += Ggn;
                        Bs += Ggd;
                        const float h = fmaf(r2.y, Ggn, r2.z * Ggd);
                        R0 += h;
                        const float hx = h * dx;
                        R1 += hx;
                        R2 = fmaf(hx, dx, R2);
                    }
                }
                S1x += R1;
                S1y = fmaf(dy, R0, S1y);
                S1z = fmaf(dz, R0, S1z);
                Sxx += R2;
                Sxy = fmaf(dy, R1, Sxy);
                Sxz = fmaf(dz, R1, Sxz);
                const float dyR0 = dy * R0;
                Syy = fmaf(dy, dyR0, Syy);
                Syz = fmaf(dz, dyR0, Syz);
                Szz = fmaf(dz * dz, R0, Szz);
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                A += __shfl_xor_sync(gmask, A, o);
                Bs += __shfl_xor_sync(gmask, Bs, o);
                S1x += __shfl_xor_sync(gmask, S1x, o);
                S1y += __shfl_xor_sync(gmask, S1y, o);
                S1z += __shfl_xor_sync(gmask, S1z, o);
                Sxx += __shfl_xor_sync(gmask, Sxx, o);
                Syy += __shfl_xor_sync(gmask, Syy, o);
                Szz += __shfl_xor_sync(gmask, Szz, o);
                Sxy += __shfl_xor_sync(gmask, Sxy, o);
                Sxz += __shfl_xor_sync(gmask, Sxz, o);
                Syz += __shfl_xor_sync(gmask, Syz, o);
            }
            if (sl == 0) {
                const uint32_t gid = a.gids[s0 + c0 + jr];
                float* dst = a.acc + 12 * (size_t)gid;
                red_add_v4(dst, A, Bs, S1x, S1y);
                red_add_v4(dst + 4, S1z, Sxx, Syy, Szz);
                red_add_v4(dst + 8, Sxy, Sxz, Syz, 0.f);
            }
        }
    }
}

void launch_brick(int mode, const BrickArgs& a, cudaStream_t s)
{
    const unsigned grid = (unsigned)a.g.nbricks;
    switch (mode) {
        case kModeEval: k_brick<kModeEval><<<grid, kBrickThreads, 0, s>>>(a); break;
        case kModeLoss: k_brick<kModeLoss><<<grid, kBrickThreads, 0, s>>>(a); break;
        case kModeBwd: k_brick<kModeBwd><<<grid, kBrickThreads, 0, s>>>(a); break;
        default: k_brick<kModeCount><<<grid, kBrickThreads, 0, s>>>(a); break;
    }
}

// ------------------------------------------------------------------------
// deterministic SSE reduction: contiguous chunks per block, then one block
// ------------------------------------------------------------------------
constexpr int kRedBlocks = 592;

__global__ void __launch_bounds__(256) k_sse_partial(const double2* __restrict__ part, long long nb,
                                                     double2* __restrict__ out, const DevState* st)
{
    if (st->overflow) return;
    __shared__ double sm[2][8];
    long long chunk = (nb + gridDim.x - 1) / gridDim.x;
    long long b0 = (long long)blockIdx.x * chunk, b1 = min(nb, b0 + chunk);
    double x = 0.0, y = 0.0;
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double2 p = part[i];
        x += p.x;
        y += p.y;
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
                                                    double* trace, int iter, double inv_m)
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
        if (trace) trace[iter] = a * inv_m;
    }
}

void launch_sse_reduce(const double2* part, long long nbricks, DevState* st, double* trace, int iter,
                       double inv_m, cudaStream_t s)
{
    // the second half of the partial buffer is scratch for the block sums
    double2* tmp = const_cast<double2*>(part) + nbricks;
    k_sse_partial<<<kRedBlocks, 256, 0, s>>>(part, nbricks, tmp, st);
    k_sse_final<<<1, 1024, 0, s>>>(tmp, kRedBlocks, st, trace, iter, inv_m);
}

}  // namespace gve
