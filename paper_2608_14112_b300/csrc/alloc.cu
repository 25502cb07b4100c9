// alloc.cu -- analytic fixed-budget allocation on the device (Sec. III-E,
// Table I stages S1a..S1e, Eq. 4).
//
//   S1a  k_grad_occ     float32 |grad V| (central differences, one-sided at
//                       the borders), occupancy and eligibility counts.
//        gbar           lower median of |grad V| over occupied voxels: radix
//                       select on the float bits (exact).
//   S1b  draws          detail: Efraimidis-Spirakis keys -ln(u)/g, u from
//                       Philox4x32-10; coverage: raw 64-bit Philox words.  The
//                       N smallest (key, voxel) pairs are found by a radix
//                       select of the N-th key plus an order-preserving
//                       compaction, which also yields the seeds in voxel order.
//        jitter         u = (x >> 8) 2^-24 - 1/2 per axis (Eq. 4).
//   S1c  k_spacing      mean distance to the 3 nearest seeds of the same
//                       group for an evenly strided subsample of <= 4096
//                       seeds (brute force); lower median on the host.
//   S1d  k_assemble     7^3 structure tensor (FP64), cyclic Jacobi (FP64),
//   S1e                 canonical frame, quaternion (Shepperd), scales
//                       elongated along the tangent and clamped, a = trilinear
//                       V(mu), w_logit = logit(w0).
//
// This file is compiled without FMA contraction: its FP64 arithmetic follows
// the written operation order, like the CPU reference of the same steps.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "gve_int.cuh"

namespace gve {

namespace {

// ---------------- Philox4x32-10 (Salmon et al., SC'11) ----------------
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

constexpr uint32_t kCtrTag = 0x47564531u;  // 'GVE1'

__device__ __forceinline__ void draw(unsigned long long index, uint32_t stream, unsigned long long seed, uint32_t out[4])
{
    out[0] = (uint32_t)index; out[1] = (uint32_t)(index >> 32); out[2] = stream; out[3] = kCtrTag;
    philox(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ long long vid(int nx, int ny, int x, int y, int z)
{
    return ((long long)z * ny + y) * nx + x;
}

// float32 derivative along one axis, the same operations as the stencil spec
__device__ __forceinline__ float dcomp32(const float* V, int nx, int ny, int nz, int x, int y, int z, int axis)
{
    int c[3] = {x, y, z};
    int dims[3] = {nx, ny, nz};
    int n = dims[axis];
    if (n < 2) return 0.0f;
    int lo = c[axis] - 1, hi = c[axis] + 1;
    float scale = 0.5f;
    if (lo < 0) { lo = c[axis]; scale = 1.0f; }
    if (hi > n - 1) { hi = c[axis]; scale = 1.0f; }
    int a[3] = {x, y, z}, b[3] = {x, y, z};
    a[axis] = hi; b[axis] = lo;
    float diff = V[vid(nx, ny, a[0], a[1], a[2])] - V[vid(nx, ny, b[0], b[1], b[2])];
    return scale * diff;
}

// float32 |grad V|: squares summed x, y, then z, no contraction
__device__ __forceinline__ float grad_mag(const float* V, int nx, int ny, int nz, int x, int y, int z)
{
    const float gx = dcomp32(V, nx, ny, nz, x, y, z, 0);
    const float gy = dcomp32(V, nx, ny, nz, x, y, z, 1);
    const float gz = dcomp32(V, nx, ny, nz, x, y, z, 2);
    const float sx = gx * gx, sy = gy * gy, sz = gz * gz;
    float sq = sx + sy;
    sq = sq + sz;
    return sqrtf(sq);
}

__global__ void __launch_bounds__(256) k_grad_occ(const float* __restrict__ V, int nx, int ny, int nz, float thr,
                                                  float* __restrict__ g, unsigned long long* cnt)
{
    long long M = (long long)nx * ny * nz;
    unsigned occ = 0, elig = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
        int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const float gm = grad_mag(V, nx, ny, nz, x, y, z);
        g[v] = gm;
        if (V[v] > thr) { ++occ; if (gm > 0.0f) ++elig; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        occ += __shfl_xor_sync(0xffffffffu, occ, o);
        elig += __shfl_xor_sync(0xffffffffu, elig, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[0], (unsigned long long)occ);
        atomicAdd(&cnt[1], (unsigned long long)elig);
    }
}

// detail key of voxel v (Efraimidis-Spirakis with weight g > 0): -ln(u) / g
// in FP64, u = (2m + 1) 2^-53 from the voxel's Philox draw; its bits order as
// the key (positive doubles)
__device__ __forceinline__ unsigned long long detail_key(unsigned long long v, float gv, unsigned long long seed)
{
    uint32_t r[4];
    draw(v, 0u, seed, r);
    unsigned long long m = (((unsigned long long)r[0] << 32) | r[1]) >> 12;
    double u = (double)(2 * m + 1) * 0x1p-53;
    double kd = -log(u) / (double)gv;
    return (unsigned long long)__double_as_longlong(kd);
}

// float32 companion of detail_key, within a relative 2^-21 of it (the bound
// used is 2^-16): -ln(u) as -logf(u) for u <= 1/2, and as -log1pf(-(1 - u))
// above, with 1 - u formed exactly from the integer 2^53 - (2m + 1); both
// arguments are one rounding from exact, and -ln is well conditioned on
// either side (relative condition number below 1.45)
__device__ __forceinline__ uint32_t detail_key32(unsigned long long v, float gv, unsigned long long seed)
{
    uint32_t r[4];
    draw(v, 0u, seed, r);
    const unsigned long long m = (((unsigned long long)r[0] << 32) | r[1]) >> 12;
    const unsigned long long a = 2 * m + 1;
    const float L = a <= (1ull << 52) ? -logf((float)a * 0x1p-53f)
                                       : -log1pf(-((float)((1ull << 53) - a) * 0x1p-53f));
    return __float_as_uint(L / gv);
}

// keys: detail (mode 0, FP64; mode 3, float32), coverage (mode 1; mode 4, its top 32 bits), gbar (mode 2, 32-bit)
__global__ void __launch_bounds__(256) k_keys(const float* __restrict__ V, const float* __restrict__ g, long long M,
                                              float thr, unsigned long long seed, int mode,
                                              unsigned long long* __restrict__ k64, uint32_t* __restrict__ k32)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
        const bool occ = V[v] > thr;
        if (mode == 2) {
            k32[v] = occ ? __float_as_uint(g[v]) : 0xFFFFFFFFu;
            continue;
        }
        if (mode == 3) {
            const float gv = g[v];
            k32[v] = occ && gv > 0.0f ? detail_key32((unsigned long long)v, gv, seed) : 0xFFFFFFFFu;
            continue;
        }
        if (mode == 4) {  // the coverage key's top 32 bits
            uint32_t r[4];
            if (occ) draw((unsigned long long)v, 1u, seed, r);
            k32[v] = occ ? r[0] : 0xFFFFFFFFu;
            continue;
        }
        unsigned long long key = ~0ull;
        if (mode == 1) {
            if (occ) {
                uint32_t r[4];
                draw((unsigned long long)v, 1u, seed, r);
                key = ((unsigned long long)r[0] << 32) | r[1];
            }
        } else {
            const float gv = g[v];
            if (occ && gv > 0.0f) key = detail_key((unsigned long long)v, gv, seed);
        }
        k64[v] = key;
    }
}

// the full 64-bit keys (mode 0: detail, mode 1: coverage) of the candidate voxels
__global__ void __launch_bounds__(256) k_cand_keys(const float* __restrict__ V, const float* __restrict__ g, float thr,
                                                   const long long* __restrict__ cand, long long C,
                                                   unsigned long long seed, int mode,
                                                   unsigned long long* __restrict__ key)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const long long v = cand[i];
    const bool occ = V[v] > thr;
    unsigned long long k = ~0ull;
    if (mode == 0) {
        const float gv = g[v];
        if (occ && gv > 0.0f) k = detail_key((unsigned long long)v, gv, seed);
    } else if (occ) {
        uint32_t r[4];
        draw((unsigned long long)v, 1u, seed, r);
        k = ((unsigned long long)r[0] << 32) | r[1];
    }
    key[i] = k;
}

__global__ void __launch_bounds__(256) k_gather_vox(const long long* __restrict__ cand, const long long* __restrict__ pos,
                                                    long long n, long long* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cand[pos[i]];
}

template <typename K>
__global__ void __launch_bounds__(256) k_sel_hist(const K* __restrict__ keys, long long M, K prefix, K pmask, int shift,
                                                  unsigned long long* __restrict__ hist)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
        K k = keys[v];
        if ((k & pmask) == prefix) atomicAdd(&h[(unsigned)((k >> shift) & 255u)], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// order-preserving compaction: selected iff key < K or (key == K and v <= vlast)
constexpr int kCompactTiles = 32;
constexpr long long kCompactChunk = 256LL * kCompactTiles;

template <typename K>
__device__ __forceinline__ bool sel_pred(const K* keys, long long v, long long M, K thr, long long vlast, int tie_only)
{
    if (v >= M) return false;
    K k = keys[v];
    if (tie_only) return k == thr;
    return k < thr || (k == thr && v <= vlast);
}

template <typename K>
__global__ void __launch_bounds__(256) k_compact_count(const K* __restrict__ keys, long long M, K thr, long long vlast,
                                                       int tie_only, uint32_t* __restrict__ bcnt)
{
    __shared__ unsigned sw[8];
    long long base = (long long)blockIdx.x * kCompactChunk;
    unsigned c = 0;
    for (int t = 0; t < kCompactTiles; ++t) c += sel_pred(keys, base + t * 256 + threadIdx.x, M, thr, vlast, tie_only);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned s = 0;
        for (int w = 0; w < 8; ++w) s += sw[w];
        bcnt[blockIdx.x] = s;
    }
}

template <typename K>
__global__ void __launch_bounds__(256) k_compact_write(const K* __restrict__ keys, long long M, K thr, long long vlast,
                                                       int tie_only, const unsigned long long* __restrict__ boff,
                                                       long long limit, long long* __restrict__ out)
{
    __shared__ unsigned sw[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long base = (long long)blockIdx.x * kCompactChunk;
    unsigned long long run = boff[blockIdx.x];
    for (int t = 0; t < kCompactTiles; ++t) {
        long long v = base + t * 256 + threadIdx.x;
        bool p = sel_pred(keys, v, M, thr, vlast, tie_only);
        unsigned bal = __ballot_sync(0xffffffffu, p);
        if (lane == 0) sw[w] = __popc(bal);
        __syncthreads();
        unsigned before = 0, tot = 0;
        for (int ww = 0; ww < 8; ++ww) {
            if (ww < w) before += sw[ww];
            tot += sw[ww];
        }
        if (p) {
            unsigned long long pos = run + before + __popc(bal & ((1u << lane) - 1u));
            if ((long long)pos < limit) out[pos] = v;
        }
        run += tot;
        __syncthreads();
    }
}

__global__ void k_coords(const long long* __restrict__ vox, long long ng, int nx, int ny, int4* __restrict__ xyz)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    long long v = vox[i];
    xyz[i] = make_int4((int)(v % nx), (int)((v / nx) % ny), (int)(v / ((long long)nx * ny)), 0);
}

// mean distance to the 3 nearest seeds of the group, for subsample point j
__global__ void __launch_bounds__(256) k_spacing(const int4* __restrict__ xyz, long long ng, int nsub, int knn,
                                                 double* __restrict__ vals)
{
    const int j = blockIdx.x;
    const long long i = (long long)(((unsigned long long)j * (unsigned long long)ng) / (unsigned long long)nsub);
    const int4 p = xyz[i];
    unsigned long long b0 = ~0ull, b1 = ~0ull, b2 = ~0ull;
    for (long long o = threadIdx.x; o < ng; o += blockDim.x) {
        if (o == i) continue;
        const int4 q = xyz[o];
        long long dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
        if (d2 < b2) {
            if (d2 < b1) {
                b2 = b1;
                if (d2 < b0) { b1 = b0; b0 = d2; } else b1 = d2;
            } else b2 = d2;
        }
    }
    __shared__ unsigned long long cand[256 * 3];
    cand[threadIdx.x * 3] = b0; cand[threadIdx.x * 3 + 1] = b1; cand[threadIdx.x * 3 + 2] = b2;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long best[3] = {~0ull, ~0ull, ~0ull};
        for (int t = 0; t < 256 * 3; ++t) {
            unsigned long long d2 = cand[t];
            if (d2 < best[2]) {
                if (d2 < best[1]) {
                    best[2] = best[1];
                    if (d2 < best[0]) { best[1] = best[0]; best[0] = d2; } else best[1] = d2;
                } else best[2] = d2;
            }
        }
        double s = 0.0;
        for (int t = 0; t < knn; ++t) s += sqrt((double)best[t]);
        vals[j] = s / (double)knn;
    }
}

// ---------------- per-seed assembly (FP64) ----------------
__device__ void grad64(const float* V, int nx, int ny, int nz, int x, int y, int z, double gv[3])
{
    int c[3] = {x, y, z};
    int dims[3] = {nx, ny, nz};
    for (int axis = 0; axis < 3; ++axis) {
        int n = dims[axis];
        if (n < 2) { gv[axis] = 0.0; continue; }
        int lo = c[axis] - 1, hi = c[axis] + 1;
        double scale = 0.5;
        if (lo < 0) { lo = c[axis]; scale = 1.0; }
        if (hi > n - 1) { hi = c[axis]; scale = 1.0; }
        int a[3] = {x, y, z}, b[3] = {x, y, z};
        a[axis] = hi; b[axis] = lo;
        gv[axis] = scale * ((double)V[vid(nx, ny, a[0], a[1], a[2])] - (double)V[vid(nx, ny, b[0], b[1], b[2])]);
    }
}

__device__ void jacobi3(const double J6[6], double evals[3], double ev9[9])
{
    double a[3][3] = {{J6[0], J6[3], J6[4]}, {J6[3], J6[1], J6[5]}, {J6[4], J6[5], J6[2]}};
    double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double fro = off * 2 + a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-30 * fro || off == 0.0) break;
        for (int r = 0; r < 3; ++r) {
            int p = PQ[r][0], q = PQ[r][1];
            if (a[p][q] == 0.0) continue;
            double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            for (int k = 0; k < 3; ++k) {
                double akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - s * akq;
                a[k][q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                double apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - s * aqk;
                a[q][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    int idx[3] = {0, 1, 2};
    double lam[3] = {a[0][0], a[1][1], a[2][2]};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[idx[j]] < lam[idx[i]] || (lam[idx[j]] == lam[idx[i]] && idx[j] < idx[i])) {
                int t = idx[i]; idx[i] = idx[j]; idx[j] = t;
            }
    for (int c = 0; c < 3; ++c) {
        evals[c] = lam[idx[c]];
        for (int r = 0; r < 3; ++r) ev9[r * 3 + c] = v[r][idx[c]];
    }
}

__device__ void frame_quat(const double ev9[9], double q[4])
{
    double e[2][3];
    for (int c = 0; c < 2; ++c) {
        int best = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(ev9[r * 3 + c]) > fabs(ev9[best * 3 + c])) best = r;
        double sgn = ev9[best * 3 + c] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) e[c][r] = sgn * ev9[r * 3 + c];
    }
    double e3[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                    e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    double R[3][3];
    for (int r = 0; r < 3; ++r) { R[r][0] = e[0][r]; R[r][1] = e[1][r]; R[r][2] = e3[r]; }
    double tr = R[0][0] + R[1][1] + R[2][2];
    double w, x, y, z;
    if (tr > 0.0) {
        double S = sqrt(tr + 1.0) * 2.0;
        w = 0.25 * S; x = (R[2][1] - R[1][2]) / S; y = (R[0][2] - R[2][0]) / S; z = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double S = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2.0;
        w = (R[2][1] - R[1][2]) / S; x = 0.25 * S; y = (R[0][1] + R[1][0]) / S; z = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        double S = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2.0;
        w = (R[0][2] - R[2][0]) / S; x = (R[0][1] + R[1][0]) / S; y = 0.25 * S; z = (R[1][2] + R[2][1]) / S;
    } else {
        double S = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2.0;
        w = (R[1][0] - R[0][1]) / S; x = (R[0][2] + R[2][0]) / S; y = (R[1][2] + R[2][1]) / S; z = 0.25 * S;
    }
    if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
    q[0] = w; q[1] = x; q[2] = y; q[3] = z;
}

__device__ double trilinear(const float* V, int nx, int ny, int nz, double px, double py, double pz)
{
    double p[3] = {px, py, pz};
    int dims[3] = {nx, ny, nz};
    int i0[3], i1[3];
    double f[3];
    for (int j = 0; j < 3; ++j) {
        double c = p[j];
        if (c < 0.0) c = 0.0;
        if (c > dims[j] - 1) c = dims[j] - 1;
        double fl = floor(c);
        i0[j] = (int)fl;
        i1[j] = i0[j] + 1 < dims[j] ? i0[j] + 1 : i0[j];
        f[j] = c - fl;
    }
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double wgt = (cx ? f[0] : 1 - f[0]) * (cy ? f[1] : 1 - f[1]) * (cz ? f[2] : 1 - f[2]);
                acc += wgt * (double)V[vid(nx, ny, cx ? i1[0] : i0[0], cy ? i1[1] : i0[1], cz ? i1[2] : i0[2])];
            }
    return acc;
}

struct AssembleArgs {
    const float* V;
    const float* g;
    const long long* vd;
    const long long* vc;
    long long Nd, N;
    int nx, ny, nz;
    unsigned long long seed;
    double hd, hc, gbar, smax_cap, smin_cap, wl;
    float* prims;
};

__global__ void __launch_bounds__(128) k_assemble(const AssembleArgs a)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int grp = i < a.Nd ? 0 : 1;
    const long long gi = grp == 0 ? i : i - a.Nd;
    const long long v = grp == 0 ? a.vd[gi] : a.vc[gi];
    const int cx = (int)(v % a.nx), cy = (int)((v / a.nx) % a.ny), cz = (int)(v / ((long long)a.nx * a.ny));
    uint32_t r[4];
    draw((unsigned long long)gi, 2u + (uint32_t)grp, a.seed, r);
    float u[3];
    for (int j = 0; j < 3; ++j) u[j] = (float)(r[j] >> 8) * 0x1p-24f - 0.5f;
    double mu[3] = {cx + (double)u[0], cy + (double)u[1], cz + (double)u[2]};
    // 7^3 structure tensor, window clipped at the borders
    double J[6] = {0, 0, 0, 0, 0, 0};
    for (int z = cz - 3; z <= cz + 3; ++z) {
        if (z < 0 || z >= a.nz) continue;
        for (int y = cy - 3; y <= cy + 3; ++y) {
            if (y < 0 || y >= a.ny) continue;
            for (int x = cx - 3; x <= cx + 3; ++x) {
                if (x < 0 || x >= a.nx) continue;
                double gv[3];
                grad64(a.V, a.nx, a.ny, a.nz, x, y, z, gv);
                J[0] += gv[0] * gv[0]; J[1] += gv[1] * gv[1]; J[2] += gv[2] * gv[2];
                J[3] += gv[0] * gv[1]; J[4] += gv[0] * gv[2]; J[5] += gv[1] * gv[2];
            }
        }
    }
    double ev[3], evec[9], q[4];
    jacobi3(J, ev, evec);
    frame_quat(evec, q);
    double sg = 0.5 * (grp == 0 ? a.hd : a.hc);
    double ratio = a.gbar > 0.0 ? 1.0 + (double)a.g[v] / a.gbar : 1.0;
    if (ratio < 1.0) ratio = 1.0;
    if (ratio > 3.0) ratio = 3.0;
    double s[3] = {sg * ratio, sg, sg};
    float out[12];
    out[0] = (float)mu[0]; out[1] = (float)mu[1]; out[2] = (float)mu[2];
    for (int j = 0; j < 3; ++j) {
        if (s[j] > a.smax_cap) s[j] = a.smax_cap;
        if (s[j] < a.smin_cap) s[j] = a.smin_cap;
        out[3 + j] = (float)log(s[j]);
    }
    out[6] = (float)q[0]; out[7] = (float)q[1]; out[8] = (float)q[2]; out[9] = (float)q[3];
    out[10] = (float)trilinear(a.V, a.nx, a.ny, a.nz, mu[0], mu[1], mu[2]);
    out[11] = (float)a.wl;
    float4* o = reinterpret_cast<float4*>(a.prims) + 3 * i;
    o[0] = make_float4(out[0], out[1], out[2], out[3]);
    o[1] = make_float4(out[4], out[5], out[6], out[7]);
    o[2] = make_float4(out[8], out[9], out[10], out[11]);
}

int grid_for(long long M)
{
    long long b = (M + 255) / 256;
    if (b > 32LL * num_sms()) b = 32LL * num_sms();
    return (int)(b < 1 ? 1 : b);
}

// k-th smallest key (0-based rank) by radix select; host-driven passes of
// 8-bit digits from the top.  When every key shares its top `known` bits
// (those of `prefix0`), the passes start below them; a last pass that
// would reach below bit 0 is taken at bit 0 (its top digit bits are fixed).
template <typename K>
gve_status radix_select(gve_ctx* c, const K* keys, long long M, unsigned long long rank, K* out, cudaStream_t s,
                        K prefix0 = 0, int known = 0)
{
    const int bits = (int)sizeof(K) * 8;
    gve_status st = ensure(c, c->a_tmp, 256 * sizeof(unsigned long long), s);
    if (st != GVE_OK) return st;
    unsigned long long* dh = (unsigned long long*)c->a_tmp.p;
    std::vector<unsigned long long> h(256);
    K pmask = known > 0 ? (K)(~(K)0 << (bits - known)) : (K)0;
    K prefix = prefix0 & pmask;
    const int first = bits - known - 8 > 0 ? bits - known - 8 : 0;
    for (int shift = first;; shift = shift > 8 ? shift - 8 : 0) {
        cudaError_t e = cudaMemsetAsync(dh, 0, 256 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset select hist");
        k_sel_hist<K><<<grid_for(M), 256, 0, s>>>(keys, M, prefix, pmask, shift, dh);
        e = cudaMemcpyAsync(h.data(), dh, 256 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "select hist");
        unsigned long long acc = 0;
        int d = 0;
        for (; d < 256; ++d) {
            if (acc + h[d] > rank) break;
            acc += h[d];
        }
        if (d == 256) { c->err = "radix select rank beyond key count"; return GVE_E_INTERNAL; }
        rank -= acc;
        prefix |= (K)d << shift;
        pmask |= (K)255 << shift;
        if (shift == 0) break;
    }
    *out = prefix;
    return GVE_OK;
}

// seeds of one draw: the `count` smallest (key, voxel) pairs, in voxel order
gve_status draw_set(gve_ctx* c, const unsigned long long* keys, long long M, long long count, long long* out,
                    cudaStream_t s)
{
    if (count <= 0) return GVE_OK;
    unsigned long long K;
    gve_status st = radix_select<unsigned long long>(c, keys, M, (unsigned long long)(count - 1), &K, s);
    if (st != GVE_OK) return st;
    long long nblk = (M + kCompactChunk - 1) / kCompactChunk;
    st = ensure(c, c->a_cnt, sizeof(uint32_t) * nblk + sizeof(unsigned long long) * (nblk + 1) + 64, s);
    if (st != GVE_OK) return st;
    uint32_t* bcnt = (uint32_t*)c->a_cnt.p;
    unsigned long long* boff = (unsigned long long*)((char*)c->a_cnt.p + ((sizeof(uint32_t) * nblk + 15) / 16) * 16);
    std::vector<unsigned long long> tail(1);
    // number strictly below K
    k_compact_count<unsigned long long><<<(unsigned)nblk, 256, 0, s>>>(keys, M, K, -1, 0, bcnt);
    launch_exscan_u32(bcnt, nblk, boff, c->scanp.p, s);
    unsigned long long less = 0;
    cudaError_t e = cudaMemcpyAsync(&less, boff + nblk, sizeof(less), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "draw count");
    long long need = count - (long long)less;  // ties at K taken in voxel order
    long long vlast = -1;
    if (need > 0) {
        // voxel index of the need-th tie
        k_compact_count<unsigned long long><<<(unsigned)nblk, 256, 0, s>>>(keys, M, K, 0, 1, bcnt);
        launch_exscan_u32(bcnt, nblk, boff, c->scanp.p, s);
        k_compact_write<unsigned long long><<<(unsigned)nblk, 256, 0, s>>>(keys, M, K, 0, 1, boff, need, out);
        e = cudaMemcpyAsync(&vlast, out + need - 1, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "draw ties");
    }
    k_compact_count<unsigned long long><<<(unsigned)nblk, 256, 0, s>>>(keys, M, K, vlast, 0, bcnt);
    launch_exscan_u32(bcnt, nblk, boff, c->scanp.p, s);
    k_compact_write<unsigned long long><<<(unsigned)nblk, 256, 0, s>>>(keys, M, K, vlast, 0, boff, count, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "draw compaction");
    return GVE_OK;
}

// One draw (mode 0: detail, FP64 keys; mode 1: coverage, 64-bit integer
// keys) in two levels: the same seeds as draw_set over every voxel's key,
// with the full key computed only where it can decide.  A 32-bit surrogate
// of each key is selected first: for the coverage keys their top 32 bits (a
// monotone map, so the n-th smallest surrogate t is the surrogate of the
// n-th smallest key, and every voxel whose key is at most that key has a
// surrogate <= t); for the detail keys a float32 key within a relative
// e = 2^-16 of the FP64 one (at least n FP64 keys are <= t / (1 - e), and
// every voxel whose FP64 key is at most the n-th smallest has a float key
// <= t (1 + e) / (1 - e)).  The candidates under that bound (in voxel order)
// get their full keys, and draw_set over them picks the same voxels, ties
// included, in the same order.  Falls back to full keys everywhere when the
// candidates would not fit beside the surrogates (or t is not finite).
gve_status draw_two_level(gve_ctx* c, const float* V, const float* g, long long M, float thr, unsigned long long seed,
                          int mode, long long n, long long* out, cudaStream_t s)
{
    if (n <= 0) return GVE_OK;
    unsigned long long* k64 = (unsigned long long*)c->a_keys.p;
    uint32_t* k32 = (uint32_t*)c->a_keys.p;
    bool fast = getenv("GVE_TEST_DRAW_FULL") == nullptr;
    long long C = 0;
    uint32_t bb = 0;
    const long long nblk = (M + kCompactChunk - 1) / kCompactChunk;
    gve_status st = ensure(c, c->a_cnt, sizeof(uint32_t) * nblk + sizeof(unsigned long long) * (nblk + 1) + 64, s);
    if (st != GVE_OK) return st;
    uint32_t* bcnt = (uint32_t*)c->a_cnt.p;
    unsigned long long* boff = (unsigned long long*)((char*)c->a_cnt.p + ((sizeof(uint32_t) * nblk + 15) / 16) * 16);
    if (fast) {
        k_keys<<<grid_for(M), 256, 0, s>>>(V, g, M, thr, seed, mode == 0 ? 3 : 4, nullptr, k32);
        uint32_t tb = 0;
        if ((st = radix_select<uint32_t>(c, k32, M, (unsigned long long)(n - 1), &tb, s)) != GVE_OK) return st;
        if (mode == 0) {
            float t;
            memcpy(&t, &tb, sizeof(t));
            fast = std::isfinite(t);
            const double e = 0x1p-16;
            const double bd = (double)t * (1.0 + e) / (1.0 - e);
            float bf = (float)bd;
            if ((double)bf < bd) bf = std::nextafter(bf, INFINITY);
            memcpy(&bb, &bf, sizeof(bb));
        } else {
            bb = tb;
        }
        if (fast) {
            k_compact_count<uint32_t><<<(unsigned)nblk, 256, 0, s>>>(k32, M, bb, M, 0, bcnt);
            launch_exscan_u32(bcnt, nblk, boff, c->scanp.p, s);
            unsigned long long hcnt = 0;
            cudaError_t e2 = cudaMemcpyAsync(&hcnt, boff + nblk, sizeof(hcnt), cudaMemcpyDeviceToHost, s);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "draw candidates");
            C = (long long)hcnt;
            // candidates, their full keys and the picked positions beside the surrogates
            fast = C >= n && 16 * C + 8 * n + 64 <= 4 * M;
        }
    }
    if (!fast) {
        k_keys<<<grid_for(M), 256, 0, s>>>(V, g, M, thr, seed, mode, k64, nullptr);
        return draw_set(c, k64, M, n, out, s);
    }
    const size_t base = ((size_t)4 * M + 15) / 16 * 16;
    long long* cand = (long long*)((char*)c->a_keys.p + base);
    unsigned long long* kc = (unsigned long long*)(cand + C);
    long long* pos = (long long*)(kc + C);
    k_compact_write<uint32_t><<<(unsigned)nblk, 256, 0, s>>>(k32, M, bb, M, 0, boff, C, cand);
    k_cand_keys<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(V, g, thr, cand, C, seed, mode, kc);
    if ((st = draw_set(c, kc, C, n, pos, s)) != GVE_OK) return st;
    k_gather_vox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cand, pos, n, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "two-level draw");
    return GVE_OK;
}

gve_status group_spacing(gve_ctx* c, const long long* vox, long long ng, gve_dims d, long long n_occ, long long N,
                         double* h, cudaStream_t s)
{
    if (ng < 2) {
        *h = std::cbrt((double)(n_occ > 0 ? n_occ : 1) / (double)(N > 0 ? N : 1));
        return GVE_OK;
    }
    int nsub = ng < 4096 ? (int)ng : 4096;
    int knn = ng - 1 < 3 ? (int)(ng - 1) : 3;
    gve_status st = ensure(c, c->a_tmp, sizeof(int4) * ng + sizeof(double) * 4096 + 64, s);
    if (st != GVE_OK) return st;
    int4* xyz = (int4*)c->a_tmp.p;
    double* vals = (double*)((char*)c->a_tmp.p + sizeof(int4) * ng);
    k_coords<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(vox, ng, d.nx, d.ny, xyz);
    k_spacing<<<nsub, 256, 0, s>>>(xyz, ng, nsub, knn, vals);
    std::vector<double> hv(nsub);
    cudaError_t e = cudaMemcpyAsync(hv.data(), vals, sizeof(double) * nsub, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "spacing");
    std::sort(hv.begin(), hv.end());
    *h = hv[(nsub - 1) / 2];
    return GVE_OK;
}

long long nd_of(long long N, double frac) { return (long long)std::floor(frac * (double)N + 0.5); }

long long feasible_max(long long N, double frac, long long n_elig, long long n_occ)
{
    long long lo = 0, hi = N;
    while (lo < hi) {
        long long mid = lo + (hi - lo + 1) / 2;
        long long nd = nd_of(mid, frac), nc = mid - nd;
        if (nd <= n_elig && nc <= n_occ) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

gve_status allocate(gve_ctx* c, const float* V, gve_dims d, int64_t N, const gve_alloc_opts* o, float* prims,
                    int64_t* feasible_out, gve_alloc_info* info, cudaStream_t s)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    gve_status st;
    if ((st = ensure(c, c->a_g, sizeof(float) * M, s)) != GVE_OK) return st;
    if ((st = ensure(c, c->a_keys, sizeof(unsigned long long) * M, s)) != GVE_OK) return st;
    if ((st = ensure(c, c->scanp, sizeof(unsigned long long) * kScanBlocks, s)) != GVE_OK) return st;
    if ((st = ensure(c, c->a_sel, sizeof(long long) * (N > 0 ? N : 1) + 64, s)) != GVE_OK) return st;
    if ((st = ensure(c, c->state, sizeof(DevState), s)) != GVE_OK) return st;
    float* g = (float*)c->a_g.p;
    unsigned long long* cnt = (unsigned long long*)c->state.p;  // scratch use of the state block
    cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset counts");
    const float thr = o->occ_thresh;
    k_grad_occ<<<grid_for(M), 256, 0, s>>>(V, d.nx, d.ny, d.nz, thr, g, cnt);
    unsigned long long hc[2] = {0, 0};
    e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy counts");
    const long long n_occ = (long long)hc[0], n_elig = (long long)hc[1];
    const long long Nd = nd_of(N, o->detail_frac), Nc = N - Nd;
    if (info) {
        info->n_occupied = n_occ; info->n_eligible = n_elig; info->n_detail = Nd; info->n_coverage = Nc;
        info->gbar = 0; info->h_detail = 0; info->h_coverage = 0;
    }
    if (Nd > n_elig || Nc > n_occ) {
        if (feasible_out) *feasible_out = feasible_max(N, o->detail_frac, n_elig, n_occ);
        c->err = "budget exceeds the distinct positions the field supports";
        return GVE_E_BUDGET;
    }
    if (feasible_out) *feasible_out = N;
    if (N == 0) return GVE_OK;
    // gbar: lower median of g over occupied voxels
    uint32_t* k32 = (uint32_t*)c->a_keys.p;
    k_keys<<<grid_for(M), 256, 0, s>>>(V, g, M, thr, o->seed, 2, nullptr, k32);
    uint32_t gbits = 0;
    if ((st = radix_select<uint32_t>(c, k32, M, (unsigned long long)((n_occ - 1) / 2), &gbits, s)) != GVE_OK) return st;
    float gbar_f;
    memcpy(&gbar_f, &gbits, sizeof(float));
    const double gbar = (double)gbar_f;
    // draws
    long long* vd = (long long*)c->a_sel.p;
    long long* vc = vd + Nd;
    if ((st = draw_two_level(c, V, g, M, thr, o->seed, 0, Nd, vd, s)) != GVE_OK) return st;
    if ((st = draw_two_level(c, V, g, M, thr, o->seed, 1, Nc, vc, s)) != GVE_OK) return st;
    // group spacing
    double hd = 0, hcv = 0;
    if ((st = group_spacing(c, vd, Nd, d, n_occ, N, &hd, s)) != GVE_OK) return st;
    if ((st = group_spacing(c, vc, Nc, d, n_occ, N, &hcv, s)) != GVE_OK) return st;
    AssembleArgs a;
    a.V = V; a.g = g; a.vd = vd; a.vc = vc; a.Nd = Nd; a.N = N;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz; a.seed = o->seed;
    a.hd = hd; a.hc = hcv; a.gbar = gbar;
    int mx = d.nx > d.ny ? (d.nx > d.nz ? d.nx : d.nz) : (d.ny > d.nz ? d.ny : d.nz);
    a.smax_cap = (double)mx / 16.0;
    a.smin_cap = 0.3;
    a.wl = std::log((double)o->w0 / (1.0 - (double)o->w0));
    a.prims = prims;
    k_assemble<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "assemble");
    if (info) { info->gbar = gbar; info->h_detail = hd; info->h_coverage = hcv; }
    return GVE_OK;
}

// ------------------------------------------------------------------------
// Stratified samples (Sec. III-F; Table III: 3,072 per iteration, 35 / 40 /
// 25 %): value-class lists and the per-iteration draw.  Compiled without
// FMA contraction, so the FP64 trilinear targets follow the written order.
// ------------------------------------------------------------------------
namespace {

constexpr int kClsChunk = 4096;          // voxels per block of the class passes
constexpr uint32_t kSampleStream = 4u;   // Philox stream of the sample draw

__device__ __forceinline__ bool cls_hi(float x) { return x > 0.4f; }
__device__ __forceinline__ bool cls_mid(float x) { return x > 0.02f && !(x > 0.4f); }

__global__ void __launch_bounds__(256) k_cls_count(const float* __restrict__ V, long long M,
                                                   uint32_t* __restrict__ cnt_hi, uint32_t* __restrict__ cnt_mid)
{
    __shared__ uint32_t sh[8], sm[8];
    const long long b0 = (long long)blockIdx.x * kClsChunk;
    uint32_t h = 0, m = 0;
    for (int k = threadIdx.x; k < kClsChunk; k += 256) {
        const long long v = b0 + k;
        if (v < M) {
            const float x = V[v];
            h += cls_hi(x);
            m += cls_mid(x);
        }
    }
    h = __reduce_add_sync(0xffffffffu, h);
    m = __reduce_add_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = h; sm[threadIdx.x >> 5] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t th = 0, tm = 0;
        for (int w = 0; w < 8; ++w) { th += sh[w]; tm += sm[w]; }
        cnt_hi[blockIdx.x] = th;
        cnt_mid[blockIdx.x] = tm;
    }
}

// members of each block's chunk, ascending, at the block's offsets
__global__ void __launch_bounds__(256) k_cls_write(const float* __restrict__ V, long long M,
                                                   const unsigned long long* __restrict__ off_hi,
                                                   const unsigned long long* __restrict__ off_mid,
                                                   uint32_t* __restrict__ hi, uint32_t* __restrict__ mid)
{
    __shared__ uint32_t wh[8], wm[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long oh = off_hi[blockIdx.x], om = off_mid[blockIdx.x];
    const long long b0 = (long long)blockIdx.x * kClsChunk;
    for (int it = 0; it < kClsChunk / 256; ++it) {
        const long long v = b0 + (long long)it * 256 + threadIdx.x;
        const float x = v < M ? V[v] : 0.f;
        const bool fh = v < M && cls_hi(x), fm = v < M && cls_mid(x);
        const unsigned bh = __ballot_sync(0xffffffffu, fh), bm = __ballot_sync(0xffffffffu, fm);
        if (lane == 0) { wh[w] = __popc(bh); wm[w] = __popc(bm); }
        __syncthreads();
        uint32_t ph = 0, pm = 0, th = 0, tm = 0;
        for (int k = 0; k < 8; ++k) {
            if (k < w) { ph += wh[k]; pm += wm[k]; }
            th += wh[k];
            tm += wm[k];
        }
        if (fh) hi[oh + ph + __popc(bh & lt)] = (uint32_t)v;
        if (fm) mid[om + pm + __popc(bm & lt)] = (uint32_t)v;
        oh += th;
        om += tm;
        __syncthreads();
    }
}

struct SampleDraw {
    const float* V;
    int nx, ny, nz;
    const uint32_t* hi;
    const uint32_t* mid;
    unsigned long long nh, nm;
    long long S, s_hi, s_mid;
    unsigned long long seed;
    uint32_t iter;
    float4* pts;
    long long* vox;
};

// sample j: Philox words x0..x3 of counter (j, iter, 4, 'GVE1'); the voxel
// is the floor(x0 count / 2^32)-th of its class (a class without voxels
// hands its samples to the uniform draw over the grid), the point c + u with
// u_k = (x_{k+1} >> 8) 2^-24 - 1/2, the target the FP64 trilinear V(p)
__global__ void __launch_bounds__(128) k_draw_samples(SampleDraw a)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.S) return;
    uint32_t r[4];
    draw(((unsigned long long)a.iter << 32) | (unsigned long long)(uint32_t)j, kSampleStream, a.seed, r);
    const uint32_t* list = nullptr;
    unsigned long long count = (unsigned long long)a.nx * a.ny * a.nz;
    if (j < a.s_hi && a.nh > 0) {
        list = a.hi;
        count = a.nh;
    } else if (j >= a.s_hi && j < a.s_hi + a.s_mid && a.nm > 0) {
        list = a.mid;
        count = a.nm;
    }
    const unsigned long long k = ((unsigned long long)r[0] * count) >> 32;
    const long long v = list ? (long long)list[k] : (long long)k;
    const int c[3] = {(int)(v % a.nx), (int)((v / a.nx) % a.ny), (int)(v / ((long long)a.nx * a.ny))};
    float p[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float u = (float)(r[q + 1] >> 8) * 0x1p-24f - 0.5f;
        p[q] = (float)c[q] + u;
    }
    const float val = (float)trilinear(a.V, a.nx, a.ny, a.nz, (double)p[0], (double)p[1], (double)p[2]);
    a.pts[j] = make_float4(p[0], p[1], p[2], val);
    if (a.vox) a.vox[j] = v;
}

}  // namespace

gve_status sample_classes(gve_ctx* c, const float* V, gve_dims d, cudaStream_t s)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    if (M >= (1ll << 32)) return fail(c, GVE_E_INVALID, "sampled refinement needs fewer than 2^32 voxels");
    const long long nb = (M + kClsChunk - 1) / kClsChunk;
    gve_status st;
    if ((st = ensure(c, c->s_cnt, sizeof(uint32_t) * 2 * nb, s)) != GVE_OK) return st;
    if ((st = ensure(c, c->s_off, sizeof(unsigned long long) * 2 * (nb + 1), s)) != GVE_OK) return st;
    if ((st = ensure(c, c->scanp, sizeof(unsigned long long) * kScanBlocks, s)) != GVE_OK) return st;
    uint32_t* ch = (uint32_t*)c->s_cnt.p;
    uint32_t* cm = ch + nb;
    unsigned long long* oh = (unsigned long long*)c->s_off.p;
    unsigned long long* om = oh + nb + 1;
    k_cls_count<<<(unsigned)nb, 256, 0, s>>>(V, M, ch, cm);
    launch_exscan_u32(ch, nb, oh, c->scanp.p, s);
    launch_exscan_u32(cm, nb, om, c->scanp.p, s);
    unsigned long long tot[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&tot[0], oh + nb, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[1], om + nb, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "class counts");
    if ((st = ensure(c, c->s_hi, sizeof(uint32_t) * (tot[0] > 0 ? tot[0] : 1), s)) != GVE_OK) return st;
    if ((st = ensure(c, c->s_mid, sizeof(uint32_t) * (tot[1] > 0 ? tot[1] : 1), s)) != GVE_OK) return st;
    k_cls_write<<<(unsigned)nb, 256, 0, s>>>(V, M, oh, om, (uint32_t*)c->s_hi.p, (uint32_t*)c->s_mid.p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "class lists");
    c->s_nh = tot[0];
    c->s_nm = tot[1];
    c->launches += 8;
    return GVE_OK;
}

void launch_draw_samples(const float* V, gve_dims d, const uint32_t* hi, unsigned long long nh, const uint32_t* mid,
                         unsigned long long nm, long long S, long long s_hi, long long s_mid,
                         unsigned long long seed, uint32_t iter, float4* pts, long long* vox, cudaStream_t s)
{
    if (S <= 0) return;
    SampleDraw a{V, d.nx, d.ny, d.nz, hi, mid, nh, nm, S, s_hi, s_mid, seed, iter, pts, vox};
    k_draw_samples<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(a);
}

// ------------------------------------------------------------------------
// The full objective (Sec. III-F): smoothness partners and the per-Gaussian
// regularisers (anchor, anisotropy, scale cap).  The paper gives the terms
// in words; the forms here are the readings:
//   partner of sample j of iteration t: u = (x >> 8) 2^-24 - 1/2 per axis
//     from Philox4x32-10 stream 5, counter (j, t), p' = clamp(p + 2 r u,
//     0, n - 1) in float32;
//   L_anc   = (1/N) sum (a_i - V(mu_i))^2, V trilinear (float32 here, the
//             oracle's in FP64: 1e-7 apart), gradient into a_i only;
//   L_aniso = (1/N) sum_i sum_{j<k} relu(|l_ij - l_ik| - ln r_max)^2 over
//             the log-scales l;
//   L_cap   = (1/N) sum_i sum_j relu(l_ij - ln s_hi)^2 + relu(ln s_lo - l_ij)^2.
// ------------------------------------------------------------------------
namespace {

constexpr uint32_t kPartnerStream = 5u;

__global__ void __launch_bounds__(128) k_draw_partners(const float4* __restrict__ pts, long long S, int nx, int ny,
                                                       int nz, unsigned long long seed, uint32_t iter, float radius,
                                                       float4* __restrict__ out)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    uint32_t r[4];
    draw(((unsigned long long)iter << 32) | (unsigned long long)(uint32_t)j, kPartnerStream, seed, r);
    const float span = 2.0f * radius;
    const float4 p = pts[j];
    const float q[3] = {p.x, p.y, p.z};
    const int dims[3] = {nx, ny, nz};
    float o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = (float)(r[a] >> 8) * 0x1p-24f - 0.5f;
        float v = q[a] + u * span;
        const float hi = (float)(dims[a] - 1);
        v = v < 0.0f ? 0.0f : (v > hi ? hi : v);
        o[a] = v;
    }
    out[j] = make_float4(o[0], o[1], o[2], -1.0f);  // no target: outside the value and density terms
}

// float32 trilinear V(p), edge-clamped (the anchor's target; the FP64
// version above serves the allocator and the sample draw)
__device__ __forceinline__ float trilinear32(const float* V, int nx, int ny, int nz, float px, float py, float pz)
{
    const float p[3] = {px, py, pz};
    const int dims[3] = {nx, ny, nz};
    int i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float c = p[j];
        c = c < 0.f ? 0.f : (c > (float)(dims[j] - 1) ? (float)(dims[j] - 1) : c);
        const float fl = floorf(c);
        i0[j] = (int)fl;
        i1[j] = i0[j] + 1 < dims[j] ? i0[j] + 1 : i0[j];
        f[j] = c - fl;
    }
    float acc = 0.f;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const float wgt = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
                acc += wgt * V[vid(nx, ny, cx ? i1[0] : i0[0], cy ? i1[1] : i0[1], cz ? i1[2] : i0[2])];
            }
    return acc;
}

// Per-Gaussian terms in float32 (B300's FP64 rate would make them the
// slowest pass of an iteration); partial sums compensated, folded in FP64
// per warp.
__global__ void __launch_bounds__(256) k_reg(const float* __restrict__ prims, long long n, const float* __restrict__ V,
                                             int nx, int ny, int nz, RegTerms rt, double invN,
                                             float* __restrict__ extra, double* __restrict__ terms,
                                             double* total_a, double* total_b)
{
    float sa = 0.f, ca = 0.f, sn = 0.f, cn = 0.f, sc = 0.f, cc = 0.f;  // Kahan pairs
    auto kadd = [](float& s, float& c, float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    };
    const float fN = (float)invN;
    const float ln_r = (float)rt.ln_r, ln_lo = (float)rt.ln_lo, ln_hi = (float)rt.ln_hi;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float4* p4 = reinterpret_cast<const float4*>(prims) + 3 * i;
        const float4 p0 = p4[0], p1 = p4[1], p2 = p4[2];
        const float p[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
        bool ok = true;
        for (int j = 0; j < 12; ++j) ok = ok && isfinite(p[j]);
        ok = ok && (p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]) > 0.f;
        float g[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
            if (rt.l_anc != 0.f && V) {
                const float r = p[10] - trilinear32(V, nx, ny, nz, p[0], p[1], p[2]);
                kadd(sa, ca, r * r);
                g[10] = rt.l_anc * 2.f * r * fN;
            }
            for (int j = 0; j < 3; ++j)
                for (int m = j + 1; m < 3; ++m) {
                    const float dlt = p[3 + j] - p[3 + m];
                    const float u = fabsf(dlt) - ln_r;
                    if (u > 0.f) {
                        kadd(sn, cn, u * u);
                        const float gg = rt.l_aniso * 2.f * u * fN * (dlt > 0.f ? 1.f : -1.f);
                        g[3 + j] += gg;
                        g[3 + m] -= gg;
                    }
                }
            for (int j = 0; j < 3; ++j) {
                const float u = p[3 + j] - ln_hi, w2 = ln_lo - p[3 + j];
                if (u > 0.f) { kadd(sc, cc, u * u); g[3 + j] += rt.l_cap * 2.f * u * fN; }
                if (w2 > 0.f) { kadd(sc, cc, w2 * w2); g[3 + j] -= rt.l_cap * 2.f * w2 * fN; }
            }
        }
        float4* e4 = reinterpret_cast<float4*>(extra) + 3 * i;
        e4[0] = make_float4(g[0], g[1], g[2], g[3]);
        e4[1] = make_float4(g[4], g[5], g[6], g[7]);
        e4[2] = make_float4(g[8], g[9], g[10], g[11]);
    }
    // compensated pairs (value s - c) merged across the warp in float32 with
    // an exact TwoSum of the heads; FP64 once per warp
    auto wmerge = [](float& s0, float& c0) {
        for (int o = 16; o > 0; o >>= 1) {
            const float s1 = __shfl_xor_sync(0xffffffffu, s0, o), c1 = __shfl_xor_sync(0xffffffffu, c0, o);
            const float t = s0 + s1;
            const float bp = t - s0;
            const float e = (s0 - (t - bp)) + (s1 - bp);
            s0 = t;
            c0 = (c0 + c1) - e;
        }
    };
    wmerge(sa, ca);
    wmerge(sn, cn);
    wmerge(sc, cc);
    // then across the CTA's warps, so one set of FP64 atomics leaves per CTA
    // (per-warp atomics on five addresses serialised in L2)
    __shared__ float red[8][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp][0] = sa; red[warp][1] = ca; red[warp][2] = sn;
        red[warp][3] = cn; red[warp][4] = sc; red[warp][5] = cc;
    }
    __syncthreads();
    if (warp != 0) return;
    const bool in = lane < (int)(blockDim.x >> 5);
    sa = in ? red[lane][0] : 0.f; ca = in ? red[lane][1] : 0.f;
    sn = in ? red[lane][2] : 0.f; cn = in ? red[lane][3] : 0.f;
    sc = in ? red[lane][4] : 0.f; cc = in ? red[lane][5] : 0.f;
    wmerge(sa, ca);
    wmerge(sn, cn);
    wmerge(sc, cc);
    if (lane == 0) {
        const double da = (double)sa - (double)ca, dn = (double)sn - (double)cn, dc = (double)sc - (double)cc;
        atomicAdd(terms + 3, da * invN);
        atomicAdd(terms + 4, dn * invN);
        atomicAdd(terms + 5, dc * invN);
        const double t = ((double)rt.l_anc * da + (double)rt.l_aniso * dn + (double)rt.l_cap * dc) * invN;
        if (total_a) atomicAdd(total_a, t);
        if (total_b) atomicAdd(total_b, t);
    }
}

}  // namespace

void launch_draw_partners(const float4* pts, long long S, gve_dims d, unsigned long long seed, uint32_t iter,
                          float radius, float4* out, cudaStream_t s)
{
    if (S <= 0) return;
    k_draw_partners<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(pts, S, d.nx, d.ny, d.nz, seed, iter, radius, out);
}

void launch_reg(const float* prims, long long n, const float* V, gve_dims d, const RegTerms& r, float* extra,
                double* terms, double* total_a, double* total_b, cudaStream_t s)
{
    if (n <= 0) return;
    const long long b = (n + 255) / 256;
    const long long cap = 16LL * num_sms();
    const unsigned grid = (unsigned)(b < cap ? b : cap);
    k_reg<<<grid, 256, 0, s>>>(prims, n, V, d.nx, d.ny, d.nz, r, 1.0 / (double)n, extra, terms, total_a, total_b);
}

// ------------------------------------------------------------------------
// Pre-encoding structure statistics (Sec. V-F, Table VI): occupancy, the
// share of the occupied voxels' gradient-magnitude mass held by the largest
// K = ceil(n_occ / 10), and S(1) / S(16) of the second-order structure
// function S(l) = mean over the axes longer than l of the mean
// (V(x + l e) - V(x))^2.
//
// One stencil sweep of the field, then one streaming sweep of 4 bytes per
// voxel.  Sweep 1 takes the occupancy, the gradient mass, the
// structure-function sums and a 4096-bin histogram of the gradient bits
// (sign 0, 8 exponent and 4 mantissa bits: float order), and writes each
// voxel's gradient bits (all ones where it is not occupied).  The host walks
// the histogram down to the bin b* that holds the K-th largest.  Sweep 2
// reads those bits, sums the mass of the bins above b* and compacts the bits
// of bin b*; an exact radix select over those candidates and one sum finish
// the top-K mass.
// ------------------------------------------------------------------------
namespace {

constexpr int kStatShift = 19;
constexpr int kStatBins = 4096;
constexpr int kStatTileRows = 256;
// scratch: doubles [0] gradient mass, [1..3] S(1) per axis, [4..6] S(16) per
// axis, [7] mass above b*, [8] candidate mass above the select threshold;
// counts [0] occupied, [1] candidates, [2] candidates above the threshold;
// then the 4096-bin histogram
constexpr int kStatDoubles = 10;
constexpr int kStatCounts = 4;

// compensated float32 sum (Kahan); the file is compiled without contraction
// or reassociation, so the compensation survives
struct KSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ unsigned stat_bin(float gm)
{
    return min(__float_as_uint(gm) >> kStatShift, (unsigned)(kStatBins - 1));
}

__device__ __forceinline__ double warp_sum_d(double a)
{
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Sweep order: the grid is cut into tiles of whole x rows and `ty` y rows;
// each tile is walked slab by slab in z, one x row per warp at a time in
// 32-voxel chunks.  The resident warps then cover a few consecutive slabs of
// one tile, so the z +- 1 and z + 16 neighbours are still in L2.
struct StatGrid {
    const float* V;
    int nx, ny, nz, ty;
    long long rows_tile, nrows;
};

// one x row: its start and the row-uniform border facts
struct Row {
    long long base;
    int y, z;
    bool ylo, yhi, zlo, zhi, y16, z16;
};

__device__ __forceinline__ bool decode_row(const StatGrid& g, long long row, Row& r)
{
    const long long t = row / g.rows_tile;
    const long long rr = row - t * g.rows_tile;
    r.z = (int)(rr / g.ty);
    r.y = (int)(t * g.ty) + (int)(rr - (long long)r.z * g.ty);
    if (r.y >= g.ny) return false;
    r.base = ((long long)r.z * g.ny + r.y) * g.nx;
    r.ylo = r.y > 0; r.yhi = r.y + 1 < g.ny; r.y16 = r.y + 16 < g.ny;
    r.zlo = r.z > 0; r.zhi = r.z + 1 < g.nz; r.z16 = r.z + 16 < g.nz;
    return true;
}

// One 32-voxel chunk of a row: the lane's value, its neighbours and (with
// S16) the values 16 voxels further along each axis.  All loads of a batch
// of chunks are issued before any is used, so a warp keeps several DRAM
// lines in flight.
template <bool S16>
struct Vals {
    float c, xm, xp, ym, yp, zm, zp, x16, y16, z16;
};

template <bool S16>
__device__ __forceinline__ void load_chunk(const StatGrid& g, const Row& r, int x, int lane, Vals<S16>& q)
{
    const float* V = g.V;
    const bool ok = x < g.nx;
    const long long v = r.base + x;
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    q.c = ok ? V[v] : 0.0f;
    q.xm = (ok && lane == 0 && x > 0) ? V[v - 1] : 0.0f;
    q.xp = (ok && lane == 31 && x + 1 < g.nx) ? V[v + 1] : 0.0f;
    q.ym = (ok && r.ylo) ? V[v - sy] : 0.0f;
    q.yp = (ok && r.yhi) ? V[v + sy] : 0.0f;
    q.zm = (ok && r.zlo) ? V[v - sz] : 0.0f;
    q.zp = (ok && r.zhi) ? V[v + sz] : 0.0f;
    if (S16) {
        q.x16 = (ok && x + 16 < g.nx) ? V[v + 16] : 0.0f;
        q.y16 = (ok && r.y16) ? V[v + 16 * sy] : 0.0f;
        q.z16 = (ok && r.z16) ? V[v + 16 * sz] : 0.0f;
    }
}

// float32 |grad V| of the chunk voxel (all lanes call: shuffles), the same
// operations as grad_mag: one-sided differences at the borders, squares
// summed x, y, then z.  Leaves xp, yp, zp holding the +1 neighbours where
// they exist.
// float32 |grad V| of one voxel from its six neighbours, the same operations
// as grad_mag: one-sided differences at the borders, squares summed x, y,
// then z (both sweep layouts call this, so the gradient bits agree)
__device__ __forceinline__ float voxel_grad(const StatGrid& g, const Row& r, float c, float xm, float xp, bool xlo,
                                            bool xhi, float ym, float yp, float zm, float zp)
{
    const float lx = xlo ? xm : c, hx = xhi ? xp : c;
    const float ly = r.ylo ? ym : c, hy = r.yhi ? yp : c;
    const float lz = r.zlo ? zm : c, hz = r.zhi ? zp : c;
    const float gx = g.nx < 2 ? 0.0f : ((xlo && xhi) ? 0.5f : 1.0f) * (hx - lx);
    const float gy = g.ny < 2 ? 0.0f : ((r.ylo && r.yhi) ? 0.5f : 1.0f) * (hy - ly);
    const float gz = g.nz < 2 ? 0.0f : ((r.zlo && r.zhi) ? 0.5f : 1.0f) * (hz - lz);
    const float sx = gx * gx, s2 = gy * gy, s3 = gz * gz;
    float sq = sx + s2;
    sq = sq + s3;
    return sqrtf(sq);
}

template <bool S16>
__device__ __forceinline__ float chunk_grad(const StatGrid& g, const Row& r, int x, int lane, Vals<S16>& q)
{
    const float c = q.c;
    const float um = __shfl_up_sync(0xffffffffu, c, 1);
    const float dn = __shfl_down_sync(0xffffffffu, c, 1);
    if (lane != 0) q.xm = um;
    if (lane != 31) q.xp = dn;
    if (x >= g.nx) return 0.0f;
    return voxel_grad(g, r, c, q.xm, q.xp, x > 0, x + 1 < g.nx, q.ym, q.yp, q.zm, q.zp);
}

constexpr int kBatch1 = 4;

// sweep 1 also writes each voxel's gradient bits (kStatEmpty where the
// voxel is not occupied), so that sweep 2 reads 4 bytes per voxel instead of
// re-evaluating the stencil
constexpr uint32_t kStatEmpty = 0xFFFFFFFFu;

// block sums of `n` doubles per warp (red[warp][k]); thread k < n of warp 0
// adds the block's k-th sum to out[k]
template <int n>
__device__ __forceinline__ void block_add(double (&red)[8][n], double* __restrict__ out)
{
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid == 0 && lane < n) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][lane];
        atomicAdd(out + lane, t);
    }
}

__global__ void __launch_bounds__(256) k_stat_sweep1(StatGrid g, float thr, double* __restrict__ sums,
                                                     unsigned long long* __restrict__ cnt,
                                                     unsigned long long* __restrict__ hist,
                                                     uint32_t* __restrict__ gbits)
{
    __shared__ unsigned h[kStatBins];
    for (int i = threadIdx.x; i < kStatBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long w0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    KSum acc[7];
    unsigned long long occ = 0;
    for (long long row = w0; row < g.nrows; row += nw) {
        Row r;
        if (!decode_row(g, row, r)) continue;
        for (int x0 = 0; x0 < g.nx; x0 += 32 * kBatch1) {
            Vals<true> q[kBatch1];
#pragma unroll
            for (int u = 0; u < kBatch1; ++u) load_chunk<true>(g, r, x0 + 32 * u + lane, lane, q[u]);
#pragma unroll
            for (int u = 0; u < kBatch1; ++u) {
                const int x = x0 + 32 * u + lane;
                const float gm = chunk_grad<true>(g, r, x, lane, q[u]);
                const float c = q[u].c;
                unsigned bin = 0xFFFFFFFFu;
                if (x < g.nx) {
                    const bool occupied = c > thr;
                    if (occupied) {
                        acc[0].add(gm);
                        ++occ;
                        bin = stat_bin(gm);
                    }
                    gbits[r.base + x] = occupied ? __float_as_uint(gm) : kStatEmpty;
                    if (x + 1 < g.nx) { const float d = q[u].xp - c; acc[1].add(d * d); }
                    if (r.yhi) { const float d = q[u].yp - c; acc[2].add(d * d); }
                    if (r.zhi) { const float d = q[u].zp - c; acc[3].add(d * d); }
                    if (x + 16 < g.nx) { const float d = q[u].x16 - c; acc[4].add(d * d); }
                    if (r.y16) { const float d = q[u].y16 - c; acc[5].add(d * d); }
                    if (r.z16) { const float d = q[u].z16 - c; acc[6].add(d * d); }
                }
                if (bin != 0xFFFFFFFFu) atomicAdd(&h[bin], 1u);   // plain shared atomics: a warp match costs more
            }
        }
    }
    __shared__ double red[8][7];
    for (int o = 16; o > 0; o >>= 1) occ += __shfl_xor_sync(0xffffffffu, occ, o);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const double t = warp_sum_d(acc[k].value());
        if (lane == 0) red[threadIdx.x >> 5][k] = t;
    }
    if (lane == 0) atomicAdd(cnt, occ);
    block_add<7>(red, sums);
    for (int i = threadIdx.x; i < kStatBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// Sweep 1 for rows whose length is a multiple of 4 on a 16-byte aligned
// field: each lane holds 4 consecutive voxels of a 128-voxel chunk, so one
// 16-byte load brings a neighbour of all four.  A neighbour past a border is
// read at offset 0 (the voxel itself): its one-sided difference then takes
// the voxel's own value exactly as voxel_grad does, and its pair difference
// is exactly 0, so neither the loads nor the six pair sums need a per-voxel
// condition.  The lane sums its four terms of each quantity (fused
// multiply-adds) before one compensated add.
__device__ __forceinline__ float f4c(const float4& v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

constexpr int kSweep1vThreads = 256;

__global__ void __launch_bounds__(kSweep1vThreads, 3) k_stat_sweep1v(StatGrid g, float thr, double* __restrict__ sums,
                                                         unsigned long long* __restrict__ cnt,
                                                         unsigned long long* __restrict__ hist,
                                                         uint32_t* __restrict__ gbits)
{
    __shared__ unsigned h[kStatBins];
    for (int i = threadIdx.x; i < kStatBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long w0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const float4* V4 = reinterpret_cast<const float4*>(g.V);
    uint4* G4 = reinterpret_cast<uint4*>(gbits);
    const int sy = g.nx >> 2, sz = (g.nx >> 2) * g.ny;   // float4 strides (the host checks 16 sz < 2^31)
    KSum acc[7];
    unsigned long long occ = 0;
    const unsigned nrows = (unsigned)g.nrows, rows_tile = (unsigned)g.rows_tile, ty = (unsigned)g.ty;
    for (unsigned row = (unsigned)w0; row < nrows; row += (unsigned)nw) {
        // the row's tile, slab and y (32-bit: the host checks the range)
        const unsigned t = row / rows_tile, rr = row - t * rows_tile;
        const int z = (int)(rr / ty), y = (int)(t * ty + (rr - (unsigned)z * ty));
        if (y >= g.ny) continue;
        const bool ylo = y > 0, yhi = y + 1 < g.ny, zlo = z > 0, zhi = z + 1 < g.nz;
        const long long base = ((long long)z * g.ny + y) * g.nx;
        const float4* R4 = V4 + (base >> 2);
        // row-uniform float4 offsets (0 past a border) and difference
        // factors, those of voxel_grad: 1/2 between two neighbours, 1 at a border
        const int oym = ylo ? sy : 0, oyp = yhi ? sy : 0;
        const int ozm = zlo ? sz : 0, ozp = zhi ? sz : 0;
        const int oy16 = y + 16 < g.ny ? 16 * sy : 0, oz16 = z + 16 < g.nz ? 16 * sz : 0;
        const float fy = g.ny < 2 ? 0.0f : ((ylo && yhi) ? 0.5f : 1.0f);
        const float fz = g.nz < 2 ? 0.0f : ((zlo && zhi) ? 0.5f : 1.0f);
        for (int x0 = 0; x0 < g.nx; x0 += 128) {
            const int x = x0 + 4 * lane;                  // the lane's first voxel
            const bool ok = x < g.nx;
            const int xi = min(x, g.nx - 4) >> 2;         // inside the row for every lane
            const float4 c = R4[xi];
            const float um = __shfl_up_sync(0xffffffffu, c.w, 1);
            const float dn = __shfl_down_sync(0xffffffffu, c.x, 1);
            if (!ok) continue;                            // only in the last chunk of a row
            const float* R = reinterpret_cast<const float*>(R4);
            const float xm0 = x == 0 ? c.x : (lane == 0 ? R[x - 1] : um);
            const float xp3 = x + 4 >= g.nx ? c.w : (lane == 31 ? R[x + 4] : dn);
            const float4 ym = R4[xi - oym], yp = R4[xi + oyp];
            const float4 zm = R4[xi - ozm], zp = R4[xi + ozp];
            const float4 x16 = R4[xi + (x + 16 < g.nx ? 4 : 0)];
            const float4 y16 = R4[xi + oy16], z16 = R4[xi + oz16];
            float pg = 0.0f, p[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            unsigned nocc = 0;
            uint32_t gb[4];
            // the y and z gradient terms and the differences to the y, z
            // and lag-16 neighbours of voxels (0, 1) and (2, 3) in packed
            // f32x2 operations (lane-wise the scalar operations)
            float2 py[2], pz[2];
            float2 pp[5] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                            make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const float2 cc = h2 ? make_float2(c.z, c.w) : make_float2(c.x, c.y);
                const float2 yp2 = h2 ? make_float2(yp.z, yp.w) : make_float2(yp.x, yp.y);
                const float2 ym2 = h2 ? make_float2(ym.z, ym.w) : make_float2(ym.x, ym.y);
                const float2 zp2 = h2 ? make_float2(zp.z, zp.w) : make_float2(zp.x, zp.y);
                const float2 zm2 = h2 ? make_float2(zm.z, zm.w) : make_float2(zm.x, zm.y);
                const float2 gy2 = __fmul2_rn(make_float2(fy, fy), __fadd2_rn(yp2, make_float2(-ym2.x, -ym2.y)));
                const float2 gz2 = __fmul2_rn(make_float2(fz, fz), __fadd2_rn(zp2, make_float2(-zm2.x, -zm2.y)));
                py[h2] = __fmul2_rn(gy2, gy2);
                pz[h2] = __fmul2_rn(gz2, gz2);
                const float2 nb[5] = {yp2, zp2, h2 ? make_float2(x16.z, x16.w) : make_float2(x16.x, x16.y),
                                      h2 ? make_float2(y16.z, y16.w) : make_float2(y16.x, y16.y),
                                      h2 ? make_float2(z16.z, z16.w) : make_float2(z16.x, z16.y)};
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float2 d2 = __fadd2_rn(nb[k], make_float2(-cc.x, -cc.y));
                    pp[k] = __ffma2_rn(d2, d2, pp[k]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float cj = f4c(c, j);
                const float xm = j ? f4c(c, j - 1) : xm0;
                const float xp = j < 3 ? f4c(c, j + 1) : xp3;
                const float fx = (j == 0 && x == 0) || (j == 3 && x + 4 >= g.nx) ? 1.0f : 0.5f;
                const float gx = fx * (xp - xm);
                const float sx = gx * gx;
                const float s2 = (j & 1) ? py[j >> 1].y : py[j >> 1].x;
                const float s3 = (j & 1) ? pz[j >> 1].y : pz[j >> 1].x;
                float sq = sx + s2;
                sq = sq + s3;
                const float gm = sqrtf(sq);
                const bool occupied = cj > thr;
                pg += occupied ? gm : 0.0f;
                nocc += occupied;
                gb[j] = occupied ? __float_as_uint(gm) : kStatEmpty;
                if (occupied) atomicAdd(&h[stat_bin(gm)], 1u);
                const float d = xp - cj;
                p[0] = fmaf(d, d, p[0]);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) p[k + 1] = pp[k].x + pp[k].y;
            G4[(base >> 2) + xi] = make_uint4(gb[0], gb[1], gb[2], gb[3]);
            occ += nocc;
            acc[0].add(pg);
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k + 1].add(p[k]);
        }
    }
    __shared__ double red[8][7];
    for (int o = 16; o > 0; o >>= 1) occ += __shfl_xor_sync(0xffffffffu, occ, o);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const double t = warp_sum_d(acc[k].value());
        if (lane == 0) red[threadIdx.x >> 5][k] = t;
    }
    if (lane == 0) atomicAdd(cnt, occ);
    block_add<7>(red, sums);
    for (int i = threadIdx.x; i < kStatBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// one voxel's gradient bits in sweep 2: its mass if above bin b*, and
// whether it is a candidate (a member of b*).  An occupied voxel's gradient
// is a non-negative float, so its bits shifted are its bin (below
// kStatBins, where stat_bin's clamp does not act); kStatEmpty shifts to
// 8191, in no bin.
__device__ __forceinline__ bool stat_take(uint32_t bits, unsigned bstar, float& above)
{
    const unsigned b = bits >> kStatShift;
    above += (b > bstar && b < (unsigned)kStatBins) ? __uint_as_float(bits) : 0.0f;
    return b == bstar;
}

constexpr int kSweep2Vec = 8;   // 16-byte loads per lane and block pass
constexpr int kSweep2Pass = 256 * 4 * kSweep2Vec;   // voxels per block pass

// Sweep 2 streams the gradient bits.  The boundary bin can hold a few per
// cent of the voxels, so candidates are gathered per block pass in shared
// memory (a warp scan and one shared atomic per warp) and the block reserves
// its range of the global list with one atomic per pass.
__global__ void __launch_bounds__(256) k_stat_sweep2(const uint32_t* __restrict__ gbits, long long M, unsigned bstar,
                                                     double* __restrict__ sums, unsigned long long* __restrict__ cnt,
                                                     uint32_t* __restrict__ cand, unsigned long long cap)
{
    __shared__ uint32_t buf[kSweep2Pass];
    __shared__ unsigned nbuf;
    __shared__ unsigned long long gbase;
    const int lane = threadIdx.x & 31;
    const long long n4 = M >> 2;
    const uint4* g4 = reinterpret_cast<const uint4*>(gbits);
    constexpr long long span = 256LL * kSweep2Vec;
    KSum above;
    for (long long base = (long long)blockIdx.x * span; base < n4; base += (long long)gridDim.x * span) {
        uint4 v[kSweep2Vec];
#pragma unroll
        for (int u = 0; u < kSweep2Vec; ++u) {
            const long long i = base + 256LL * u + threadIdx.x;
            v[u] = i < n4 ? __ldcs(g4 + i) : make_uint4(kStatEmpty, kStatEmpty, kStatEmpty, kStatEmpty);
        }
        __syncthreads();                                  // the previous pass's copy-out is done
        if (threadIdx.x == 0) nbuf = 0;
        unsigned mine = 0;
#pragma unroll
        for (int u = 0; u < kSweep2Vec; ++u) {      // four terms in float32, then one compensated add
            float pa = 0.0f;
            mine += stat_take(v[u].x, bstar, pa);
            mine += stat_take(v[u].y, bstar, pa);
            mine += stat_take(v[u].z, bstar, pa);
            mine += stat_take(v[u].w, bstar, pa);
            above.add(pa);
        }
        unsigned incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncthreads();                                  // nbuf is reset
        unsigned woff = 0;
        if (lane == 31 && incl) woff = atomicAdd(&nbuf, incl);
        unsigned off = __shfl_sync(0xffffffffu, woff, 31) + incl - mine;
        if (mine) {
#pragma unroll
            for (int u = 0; u < kSweep2Vec; ++u) {
                const uint32_t e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((e[k] >> kStatShift) == bstar) buf[off++] = e[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) gbase = nbuf ? atomicAdd(cnt + 1, (unsigned long long)nbuf) : 0ULL;
        __syncthreads();
        for (unsigned i = threadIdx.x; i < nbuf; i += blockDim.x)
            if (gbase + i < cap) cand[gbase + i] = buf[i];
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {          // the M mod 4 voxels past the last vector
        const long long i = (n4 << 2) + lane;
        const uint32_t bits = i < M ? gbits[i] : kStatEmpty;
        float pa = 0.0f;
        const bool take = stat_take(bits, bstar, pa);
        above.add(pa);
        const unsigned ball = __ballot_sync(0xffffffffu, take);
        if (ball) {
            unsigned long long o = 0;
            if (lane == 0) o = atomicAdd(cnt + 1, (unsigned long long)__popc(ball));
            o = __shfl_sync(0xffffffffu, o, 0) + (unsigned long long)__popc(ball & ((1u << lane) - 1u));
            if (take && o < cap) cand[o] = bits;
        }
    }
    __shared__ double red[8][1];
    const double t = warp_sum_d(above.value());
    if (lane == 0) red[threadIdx.x >> 5][0] = t;
    block_add<1>(red, sums + 7);
}

// candidate mass strictly above the select threshold, and its count
// (compensated float32 per thread, one FP64 atomic per block)
__global__ void __launch_bounds__(256) k_stat_tail(const uint32_t* __restrict__ cand, long long n, uint32_t tbits,
                                                   double* __restrict__ sums, unsigned long long* __restrict__ cnt)
{
    KSum s;
    unsigned nt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t b = cand[i];
        if (b > tbits) {
            s.add(__uint_as_float(b));
            ++nt;
        }
    }
    __shared__ double red[8][1];
    __shared__ unsigned long long rc[8];
    const int lane = threadIdx.x & 31;
    const double t = warp_sum_d(s.value());
    unsigned long long c = nt;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        red[threadIdx.x >> 5][0] = t;
        rc[threadIdx.x >> 5] = c;
    }
    block_add<1>(red, sums + 8);
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += rc[w];
        atomicAdd(cnt + 2, tot);
    }
}

StatGrid stat_grid(const float* V, gve_dims d)
{
    StatGrid g;
    g.V = V;
    g.nx = d.nx; g.ny = d.ny; g.nz = d.nz;
    const int nty = (d.ny + kStatTileRows - 1) / kStatTileRows;
    g.ty = (d.ny + nty - 1) / nty;
    g.rows_tile = (long long)d.nz * g.ty;
    g.nrows = g.rows_tile * nty;
    return g;
}

// persistent grid: the resident blocks, no more than the segments need
template <typename Kern>
int stat_blocks(Kern k, long long nrows, int threads = 256)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    long long b = (long long)num_sms() * per_sm;
    const int warps = threads / 32;
    const long long need = (nrows + warps - 1) / warps;
    if (b > need) b = need;
    return (int)(b < 1 ? 1 : b);
}

// sweep 2: the resident blocks, no more than the vectors need
int sweep2_blocks(long long M)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stat_sweep2, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long b = (long long)num_sms() * per_sm;
    const long long need = ((M >> 2) + 256LL * kSweep2Vec - 1) / (256LL * kSweep2Vec);
    if (b > need) b = need;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {

// optional stage events: [0] start, [1] after sweep 1, [2] end
struct StatEvents {
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool on = false;
    explicit StatEvents(bool want)
    {
        if (!want) return;
        on = true;
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) on = false;
    }
    void mark(int i, cudaStream_t s)
    {
        if (on) cudaEventRecord(ev[i], s);
    }
    ~StatEvents()
    {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

gve_status structure_stats(gve_ctx* c, const float* V, gve_dims d, double out[5], double* stage_ms, cudaStream_t s)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    const float thr = 0.02f;
    StatEvents ev(stage_ms != nullptr);
    const size_t scratch = sizeof(double) * kStatDoubles + sizeof(unsigned long long) * (kStatCounts + kStatBins);
    gve_status st;
    if ((st = ensure(c, c->a_cnt, scratch, s)) != GVE_OK) return st;
    double* sums = (double*)c->a_cnt.p;
    unsigned long long* cnt = (unsigned long long*)(sums + kStatDoubles);
    unsigned long long* hist = cnt + kStatCounts;
    cudaError_t e = cudaMemsetAsync(c->a_cnt.p, 0, scratch, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset structure scratch");
    const StatGrid sg = stat_grid(V, d);
    ev.mark(0, s);
    if ((st = ensure(c, c->a_g, sizeof(uint32_t) * M, s)) != GVE_OK) return st;
    uint32_t* gbits = (uint32_t*)c->a_g.p;
    const bool vec4 = d.nx % 4 == 0 && ((uintptr_t)V & 15) == 0 && sg.nrows < (1LL << 31) &&
                      16LL * (d.nx / 4) * d.ny < (1LL << 31);
    if (vec4)
        k_stat_sweep1v<<<stat_blocks(k_stat_sweep1v, sg.nrows, kSweep1vThreads), kSweep1vThreads, 0, s>>>(
            sg, thr, sums, cnt, hist, gbits);
    else
        k_stat_sweep1<<<stat_blocks(k_stat_sweep1, sg.nrows), 256, 0, s>>>(sg, thr, sums, cnt, hist, gbits);
    ev.mark(1, s);
    c->launches += 1;
    std::vector<unsigned long long> hh(kStatCounts + kStatBins);
    double hs[kStatDoubles];
    e = cudaMemcpyAsync(hh.data(), cnt, sizeof(unsigned long long) * hh.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "structure sweep 1");
    const long long n_occ = (long long)hh[0];
    const long long K = (n_occ + 9) / 10;
    double top = 0.0;
    if (n_occ > 0 && hs[0] > 0.0) {
        // bin b* holding the K-th largest; r of its members belong to the top K
        const unsigned long long* hb = hh.data() + kStatCounts;
        unsigned long long above_n = 0;
        int bstar = kStatBins - 1;
        for (; bstar >= 0; --bstar) {
            if (above_n + hb[bstar] >= (unsigned long long)K) break;
            above_n += hb[bstar];
        }
        if (bstar < 0) { c->err = "structure histogram holds fewer than K voxels"; return GVE_E_INTERNAL; }
        const unsigned long long nc = hb[bstar];
        const unsigned long long r = (unsigned long long)K - above_n;
        if ((st = ensure(c, c->a_keys, sizeof(uint32_t) * nc, s)) != GVE_OK) return st;
        uint32_t* cand = (uint32_t*)c->a_keys.p;
        k_stat_sweep2<<<sweep2_blocks(M), 256, 0, s>>>(gbits, M, (unsigned)bstar, sums, cnt, cand, nc);
        uint32_t tbits = 0;
        // every candidate's bits carry b* above bit kStatShift
        if ((st = radix_select<uint32_t>(c, cand, (long long)nc, nc - r, &tbits, s, (uint32_t)bstar << kStatShift,
                                         32 - kStatShift)) != GVE_OK)
            return st;
        k_stat_tail<<<grid_for((long long)nc), 256, 0, s>>>(cand, (long long)nc, tbits, sums, cnt);
        c->launches += 5;                   // sweep 2, three select passes, the tail
        unsigned long long hc[3];
        e = cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "structure sweep 2");
        if (hc[1] != nc) { c->err = "structure sweep 2 saw another candidate count"; return GVE_E_INTERNAL; }
        float T;
        memcpy(&T, &tbits, sizeof(float));
        top = (hs[7] + hs[8] + (double)(r - hc[2]) * (double)T) / hs[0];
    }
    out[0] = (double)n_occ / (double)M;
    out[1] = top;
    const int dims[3] = {d.nx, d.ny, d.nz};
    for (int li = 0; li < 2; ++li) {
        const int L = li ? 16 : 1;
        double sum = 0.0;
        int axes = 0;
        for (int a = 0; a < 3; ++a) {
            if (dims[a] <= L) continue;
            const double pairs = (double)(dims[a] - L) * (double)(M / dims[a]);
            sum += hs[1 + 3 * li + a] / pairs;
            ++axes;
        }
        out[2 + li] = axes ? sum / axes : 0.0;
    }
    out[4] = out[3] > 0.0 ? out[2] / out[3] : 0.0;
    if (stage_ms) {
        ev.mark(2, s);
        stage_ms[0] = stage_ms[1] = stage_ms[2] = 0.0;
        stage_ms[3] = (double)c->launches;
        if (ev.on && cudaEventSynchronize(ev.ev[2]) == cudaSuccess) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev.ev[0], ev.ev[1]);
            cudaEventElapsedTime(&b, ev.ev[0], ev.ev[2]);
            stage_ms[0] = a;
            stage_ms[1] = (double)b - (double)a;
            stage_ms[2] = b;
        }
    }
    return GVE_OK;
}

}  // namespace gve
