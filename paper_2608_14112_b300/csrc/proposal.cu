// proposal.cu -- the learned proposal: per-Gaussian structure features, a
// 16-64-64-64-4 GELU MLP (BF16 weights, FP32 accumulation) trained with the
// library's own forward/backward/Adam kernels, and the correction of the
// allocated amplitude and log-scales it predicts.
//
// Features of Gaussian i (allocated record, seed voxel c = round(mu)):
//   0-2   log(1 + lambda_k / (343 gbar^2)), eigenvalues of the 7^3 structure
//         tensor at c, ascending (FP64 accumulation and Jacobi)
//   3     |grad V|(c) / gbar (central differences), capped at 10
//   4-7   mean, standard deviation, min, max of V over the 5^3 window
//   8-10  allocated log-scales
//   11    allocated amplitude a
//   12    1 for a detail seed, 0 for a coverage seed
//   13    occupied fraction (V > occ) of the 5^3 window
//   14    eigengap (lambda_2 - lambda_1) / (lambda_3 + tiny)
//   15    V(c)
// Windows are clipped at the grid borders.
//
// Model buffer (float32 words, caller-owned device memory): FP32 master
// parameters [0, P), Adam first and second moments [P, 3P), feature mean and
// inverse standard deviation [3P, 3P+32) (the network sees
// clamp((x - mean) * istd, -6, 6)), BF16 copies of the parameters
// packed two per word [3P+32, 3P+32+P/2); P = 9668 with the parameter order
// W1[64][16] b1 W2[64][64] b2 W3[64][64] b3 W4[4][64] b4.  The forward pass
// uses the BF16 copies, dequantised to FP32 in shared memory.
#include <cuda_bf16.h>

#include <cmath>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kIn = 16, kH = 64, kOut = 4;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH;
constexpr int kP = kOffB4 + kOut;  // 9668
static_assert(kP == 9668, "parameter count");
constexpr int kOffM = kP, kOffV = 2 * kP, kOffNorm = 3 * kP, kOffBf = 3 * kP + 32;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x)
{
    const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// standardised input, clipped to [-kInClip, kInClip] so that a feature far
// outside the training spread cannot drive the network arbitrarily far
constexpr float kInClip = 6.f;
__device__ __forceinline__ float norm_in(float x, float mean, float istd)
{
    return fminf(fmaxf((x - mean) * istd, -kInClip), kInClip);
}

// dequantise the BF16 parameters into shared memory
__device__ __forceinline__ void load_weights(const float* model, float* sw)
{
    const __nv_bfloat16* bf = reinterpret_cast<const __nv_bfloat16*>(model + kOffBf);
    for (int i = threadIdx.x; i < kP; i += blockDim.x) sw[i] = __bfloat162float(bf[i]);
}

// ---------------- features ----------------
__device__ __forceinline__ long long vid(int nx, int ny, int x, int y, int z) { return ((long long)z * ny + y) * nx + x; }

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

__device__ void eig3(const double J6[6], double ev[3])
{
    double a[3][3] = {{J6[0], J6[3], J6[4]}, {J6[3], J6[1], J6[5]}, {J6[4], J6[5], J6[2]}};
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
        }
    }
    double l[3] = {a[0][0], a[1][1], a[2][2]};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (l[j] < l[i]) { double t = l[i]; l[i] = l[j]; l[j] = t; }
    ev[0] = l[0]; ev[1] = l[1]; ev[2] = l[2];
}

__global__ void __launch_bounds__(128) k_features(const float* __restrict__ V, int nx, int ny, int nz,
                                                  const float* __restrict__ prims, long long n, long long nd,
                                                  float gbar, float occ, float* __restrict__ F)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* p = prims + 12 * i;
    int c[3];
    const int dims[3] = {nx, ny, nz};
    for (int j = 0; j < 3; ++j) {
        float f = floorf(p[j] + 0.5f);
        int v = isfinite(f) ? (int)fminf(fmaxf(f, 0.f), (float)(dims[j] - 1)) : 0;
        c[j] = v;
    }
    double J[6] = {0, 0, 0, 0, 0, 0};
    for (int z = c[2] - 3; z <= c[2] + 3; ++z) {
        if (z < 0 || z >= nz) continue;
        for (int y = c[1] - 3; y <= c[1] + 3; ++y) {
            if (y < 0 || y >= ny) continue;
            for (int x = c[0] - 3; x <= c[0] + 3; ++x) {
                if (x < 0 || x >= nx) continue;
                double g[3];
                grad64(V, nx, ny, nz, x, y, z, g);
                J[0] += g[0] * g[0]; J[1] += g[1] * g[1]; J[2] += g[2] * g[2];
                J[3] += g[0] * g[1]; J[4] += g[0] * g[2]; J[5] += g[1] * g[2];
            }
        }
    }
    double ev[3];
    eig3(J, ev);
    const double gb2 = (double)gbar * (double)gbar * 343.0 + 1e-30;
    double g0[3];
    grad64(V, nx, ny, nz, c[0], c[1], c[2], g0);
    const double gc = sqrt(g0[0] * g0[0] + g0[1] * g0[1] + g0[2] * g0[2]);
    double s = 0, s2 = 0, mn = 1e30, mx = -1e30;
    int cnt = 0, nocc = 0;
    for (int z = c[2] - 2; z <= c[2] + 2; ++z) {
        if (z < 0 || z >= nz) continue;
        for (int y = c[1] - 2; y <= c[1] + 2; ++y) {
            if (y < 0 || y >= ny) continue;
            for (int x = c[0] - 2; x <= c[0] + 2; ++x) {
                if (x < 0 || x >= nx) continue;
                const float v = V[vid(nx, ny, x, y, z)];
                s += v; s2 += (double)v * v; mn = fmin(mn, (double)v); mx = fmax(mx, (double)v);
                ++cnt;
                nocc += v > occ;
            }
        }
    }
    const double mean = s / cnt, var = fmax(s2 / cnt - mean * mean, 0.0);
    float* f = F + 16 * i;
    for (int k = 0; k < 3; ++k) f[k] = (float)log1p(fmax(ev[k], 0.0) / gb2);
    f[3] = (float)fmin(gc / ((double)gbar + 1e-30), 10.0);
    f[4] = (float)mean;
    f[5] = (float)sqrt(var);
    f[6] = (float)mn;
    f[7] = (float)mx;
    f[8] = p[3]; f[9] = p[4]; f[10] = p[5];
    f[11] = p[10];
    f[12] = i < nd ? 1.f : 0.f;
    f[13] = (float)nocc / (float)cnt;
    f[14] = (float)((ev[1] - ev[0]) / (fmax(ev[2], 0.0) + 1e-30));
    f[15] = V[vid(nx, ny, c[0], c[1], c[2])];
}

// ---------------- MLP forward (one thread per row) ----------------
// save (optional): pre-activations z1, z2, z3 per row, [rows][3][64]
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ model, const float* __restrict__ X,
                                                 long long rows, float* __restrict__ Y, float* __restrict__ save)
{
    extern __shared__ float sw[];
    load_weights(model, sw);
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* mean = model + kOffNorm;
    const float* istd = model + kOffNorm + 16;
    float x[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = norm_in(X[16 * r + k], mean[k], istd[k]);
    float a[kH], b[kH];
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        float z = sw[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) z = fmaf(sw[kOffW1 + j * kIn + k], x[k], z);
        if (save) save[(r * 3 + 0) * kH + j] = z;
        a[j] = gelu(z);
    }
#pragma unroll 2
    for (int j = 0; j < kH; ++j) {
        float z = sw[kOffB2 + j];
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(sw[kOffW2 + j * kH + k], a[k], z);
        if (save) save[(r * 3 + 1) * kH + j] = z;
        b[j] = gelu(z);
    }
#pragma unroll 2
    for (int j = 0; j < kH; ++j) {
        float z = sw[kOffB3 + j];
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(sw[kOffW3 + j * kH + k], b[k], z);
        if (save) save[(r * 3 + 2) * kH + j] = z;
        a[j] = gelu(z);
    }
#pragma unroll
    for (int j = 0; j < kOut; ++j) {
        float z = sw[kOffB4 + j];
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(sw[kOffW4 + j * kH + k], a[k], z);
        Y[4 * r + j] = z;
    }
}

// ---------------- MLP backward ----------------
// dY = d loss / d output per row.  Accumulates parameter gradients into dP
// (FP32, zeroed by the caller).  One CTA of 128 rows: each thread carries its
// row's deltas; the weight gradient of every layer is a sum of per-row outer
// products, formed from shared-memory tiles of the CTA's deltas and inputs.
constexpr int kBR = 128;

__device__ void tile_grad(const float* D, const float* Ain, int nout, int nin, float* dW, float* db, int tid)
{
    // dW[j][k] += sum_r D[r][j] Ain[r][k];  db[j] += sum_r D[r][j]
    for (int e = tid; e < nout * nin; e += kBR) {
        const int j = e / nin, k = e % nin;
        float acc = 0.f;
        for (int r = 0; r < kBR; ++r) acc = fmaf(D[r * nout + j], Ain[r * nin + k], acc);
        atomicAdd(dW + e, acc);
    }
    for (int j = tid; j < nout; j += kBR) {
        float acc = 0.f;
        for (int r = 0; r < kBR; ++r) acc += D[r * nout + j];
        atomicAdd(db + j, acc);
    }
}

__global__ void __launch_bounds__(kBR) k_mlp_bwd(const float* __restrict__ model, const float* __restrict__ X,
                                                 const float* __restrict__ save, const float* __restrict__ dY,
                                                 long long rows, float* __restrict__ dP)
{
    extern __shared__ float sm[];
    float* sw = sm;              // kP
    float* D = sw + kP;          // [kBR][64]
    float* A = D + kBR * kH;     // [kBR][64]
    load_weights(model, sw);
    const int tid = threadIdx.x;
    const long long r = (long long)blockIdx.x * kBR + tid;
    const bool valid = r < rows;
    float z[kH], d[kH];
    // layer 4: delta = dY, input a3 = gelu(z3)
#pragma unroll
    for (int k = 0; k < kH; ++k) z[k] = valid ? save[(r * 3 + 2) * kH + k] : 0.f;
    float d4[kOut];
#pragma unroll
    for (int j = 0; j < kOut; ++j) d4[j] = valid ? dY[4 * r + j] : 0.f;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kOut; ++j) D[tid * kOut + j] = d4[j];
#pragma unroll
    for (int k = 0; k < kH; ++k) A[tid * kH + k] = valid ? gelu(z[k]) : 0.f;
    __syncthreads();
    tile_grad(D, A, kOut, kH, dP + kOffW4, dP + kOffB4, tid);
    // delta3 = (W4^T d4) * gelu'(z3)
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < kOut; ++j) acc = fmaf(sw[kOffW4 + j * kH + k], d4[j], acc);
        d[k] = valid ? acc * gelu_d(z[k]) : 0.f;
    }
    // layer 3: input a2 = gelu(z2)
#pragma unroll
    for (int k = 0; k < kH; ++k) z[k] = valid ? save[(r * 3 + 1) * kH + k] : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kH; ++k) { D[tid * kH + k] = d[k]; A[tid * kH + k] = valid ? gelu(z[k]) : 0.f; }
    __syncthreads();
    tile_grad(D, A, kH, kH, dP + kOffW3, dP + kOffB3, tid);
    // delta2 = (W3^T d3) * gelu'(z2)
    {
        float nd[kH];
#pragma unroll 4
        for (int k = 0; k < kH; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kH; ++j) acc = fmaf(sw[kOffW3 + j * kH + k], d[j], acc);
            nd[k] = valid ? acc * gelu_d(z[k]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kH; ++k) d[k] = nd[k];
    }
    // layer 2: input a1 = gelu(z1)
#pragma unroll
    for (int k = 0; k < kH; ++k) z[k] = valid ? save[(r * 3 + 0) * kH + k] : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kH; ++k) { D[tid * kH + k] = d[k]; A[tid * kH + k] = valid ? gelu(z[k]) : 0.f; }
    __syncthreads();
    tile_grad(D, A, kH, kH, dP + kOffW2, dP + kOffB2, tid);
    // delta1 = (W2^T d2) * gelu'(z1)
    {
        float nd[kH];
#pragma unroll 4
        for (int k = 0; k < kH; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kH; ++j) acc = fmaf(sw[kOffW2 + j * kH + k], d[j], acc);
            nd[k] = valid ? acc * gelu_d(z[k]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kH; ++k) d[k] = nd[k];
    }
    // layer 1: input = normalised features
    const float* mean = model + kOffNorm;
    const float* istd = model + kOffNorm + 16;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kH; ++k) D[tid * kH + k] = d[k];
#pragma unroll
    for (int k = 0; k < kIn; ++k) A[tid * kIn + k] = valid ? norm_in(X[16 * r + k], mean[k], istd[k]) : 0.f;
    __syncthreads();
    tile_grad(D, A, kH, kIn, dP + kOffW1, dP + kOffB1, tid);
}

// loss = mean over rows and outputs of (Y - T)^2; dY = 2 (Y - T) / (rows * 4)
__global__ void k_mlp_loss(const float* __restrict__ Y, const float* __restrict__ Tg, long long rows,
                           float* __restrict__ dY, double* loss)
{
    double acc = 0.0;
    const float scale = 2.f / (float)(rows * kOut);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < rows * kOut;
         e += (long long)gridDim.x * blockDim.x) {
        const float diff = Y[e] - Tg[e];
        acc += (double)diff * diff;
        if (dY) dY[e] = scale * diff;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc / (double)(rows * kOut));
}

__global__ void k_mlp_adam(float* model, const float* __restrict__ dP, float lr, float b1, float b2, float eps,
                           float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP) return;
    const float g = dP[i];
    float m = model[kOffM + i], v = model[kOffV + i];
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    model[kOffM + i] = m;
    model[kOffV + i] = v;
    const float w = model[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    model[i] = w;
    reinterpret_cast<__nv_bfloat16*>(model + kOffBf)[i] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_quantise(float* model)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kP) reinterpret_cast<__nv_bfloat16*>(model + kOffBf)[i] = __float2bfloat16_rn(model[i]);
}

// corrections: a += dA; log s += dLS (clamped to [log smin, log smax])
__global__ void k_apply(float* __restrict__ prims, const float* __restrict__ Y, long long n, float lsmin, float lsmax)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* p = prims + 12 * i;
    const float* y = Y + 4 * i;
    if (!isfinite(y[0]) || !isfinite(y[1]) || !isfinite(y[2]) || !isfinite(y[3])) return;
    p[10] += y[0];
    for (int j = 0; j < 3; ++j) p[3 + j] = fminf(fmaxf(p[3 + j] + y[1 + j], lsmin), lsmax);
}

// upstream gradient of the MLP outputs from the gradient of the loss with
// respect to the corrected records: d/d(da) = dL/da; d/d(dls_j) = dL/dls_j
// where the clamp of k_apply was inactive, else 0; rows whose outputs were
// not finite (left unapplied) get 0.
__global__ void k_proposal_dy(const float* __restrict__ prims, const float* __restrict__ gprims,
                              const float* __restrict__ Y, long long n, float lsmin, float lsmax, float* __restrict__ dY)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* p = prims + 12 * i;
    const float* g = gprims + 12 * i;
    const float* y = Y + 4 * i;
    const bool ok = isfinite(y[0]) && isfinite(y[1]) && isfinite(y[2]) && isfinite(y[3]);
    dY[4 * i] = ok ? g[10] : 0.f;
    for (int j = 0; j < 3; ++j) dY[4 * i + 1 + j] = ok && p[3 + j] > lsmin && p[3 + j] < lsmax ? g[3 + j] : 0.f;
}

// clamp interval of the corrected log-scales: the allocator's scale caps
// [0.3, max(nx, ny, nz) / 16], logarithms taken in double and rounded once,
// as the allocator stores them (a zero correction changes nothing)
float ls_min() { return (float)std::log(0.3); }
float ls_max(gve_dims d)
{
    const int mx = d.nx > d.ny ? (d.nx > d.nz ? d.nx : d.nz) : (d.ny > d.nz ? d.ny : d.nz);
    return (float)std::log((double)mx / 16.0);
}

constexpr size_t kFwdSmem = sizeof(float) * kP;
constexpr size_t kBwdSmem = sizeof(float) * (kP + 2 * kBR * kH);

gve_status set_smem(gve_ctx* c)
{
    static bool done[64] = {};
    int dev = c->device;
    if (dev >= 0 && dev < 64 && done[dev]) return GVE_OK;
    if (cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "mlp shared memory");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return GVE_OK;
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_proposal_features(gve_ctx* c, const float* field, gve_dims d, const float* prims,
                                            int64_t n, int64_t n_detail, float gbar, float occ_thresh,
                                            float* features, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!field || (n > 0 && (!prims || !features)) || n < 0 || n_detail < 0 || n_detail > n)
        return fail(c, GVE_E_INVALID, "bad feature arguments");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    if (n == 0) return GVE_OK;
    k_features<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(field, d.nx, d.ny, d.nz, prims, n, n_detail,
                                                                             gbar, occ_thresh, features);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "features");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_forward(gve_ctx* c, const float* model, const float* X, int64_t rows, float* Y,
                                      float* save, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || rows < 0 || (rows > 0 && (!X || !Y))) return fail(c, GVE_E_INVALID, "bad mlp arguments");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    gve_status st = set_smem(c);
    if (st != GVE_OK) return st;
    if (rows == 0) return GVE_OK;
    k_mlp_fwd<<<(unsigned)((rows + 127) / 128), 128, kFwdSmem, (cudaStream_t)stream>>>(model, X, rows, Y, save);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp forward");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_grad(gve_ctx* c, const float* model, const float* X, const float* target,
                                   int64_t rows, float* dP, double* loss_dev, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || !dP || rows <= 0 || !X || !target) return fail(c, GVE_E_INVALID, "bad mlp arguments");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    gve_status st = set_smem(c);
    if (st != GVE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: outputs, output gradient, saved pre-activations
    st = ensure(c, c->a_tmp, sizeof(float) * (size_t)rows * (4 + 4 + 3 * kH), s);
    if (st != GVE_OK) return st;
    float* Y = (float*)c->a_tmp.p;
    float* dY = Y + 4 * rows;
    float* save = dY + 4 * rows;
    k_mlp_fwd<<<(unsigned)((rows + 127) / 128), 128, kFwdSmem, s>>>(model, X, rows, Y, save);
    if (loss_dev) cudaMemsetAsync(loss_dev, 0, sizeof(double), s);
    k_mlp_loss<<<296, 256, 0, s>>>(Y, target, rows, dY, loss_dev);
    cudaMemsetAsync(dP, 0, sizeof(float) * kP, s);
    k_mlp_bwd<<<(unsigned)((rows + kBR - 1) / kBR), kBR, kBwdSmem, s>>>(model, X, save, dY, rows, dP);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp gradient");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_adam(gve_ctx* c, float* model, const float* dP, float lr, float beta1, float beta2,
                                   float eps, int32_t step, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || !dP || step < 1) return fail(c, GVE_E_INVALID, "bad adam arguments");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    const float bc1 = (float)(1.0 - std::pow((double)beta1, step)), bc2 = (float)(1.0 - std::pow((double)beta2, step));
    k_mlp_adam<<<(kP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(model, dP, lr, beta1, beta2, eps, bc1, bc2);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp adam");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_quantise(gve_ctx* c, float* model, void* stream)
{
    if (!c || !model) return GVE_E_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    k_mlp_quantise<<<(kP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(model);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp quantise");
    return GVE_OK;
}

extern "C" gve_status gve_proposal_apply(gve_ctx* c, const float* model, const float* features, float* prims,
                                         int64_t n, gve_dims d, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || n < 0 || (n > 0 && (!features || !prims))) return fail(c, GVE_E_INVALID, "bad apply arguments");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    if (n == 0) return GVE_OK;
    gve_status st = set_smem(c);
    if (st != GVE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure(c, c->a_tmp, sizeof(float) * 4 * (size_t)n, s);
    if (st != GVE_OK) return st;
    float* Y = (float*)c->a_tmp.p;
    k_mlp_fwd<<<(unsigned)((n + 127) / 128), 128, kFwdSmem, s>>>(model, features, n, Y, nullptr);
    k_apply<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(prims, Y, n, ls_min(), ls_max(d));
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "proposal apply");
    return GVE_OK;
}

extern "C" gve_status gve_proposal_backward(gve_ctx* c, const float* model, const float* features,
                                            const float* prims_corrected, const float* grad_prims, int64_t n,
                                            gve_dims d, int32_t accumulate, float* dP, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || !dP || n <= 0 || !features || !prims_corrected || !grad_prims)
        return fail(c, GVE_E_INVALID, "bad proposal backward arguments");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    gve_status st = set_smem(c);
    if (st != GVE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure(c, c->a_tmp, sizeof(float) * (size_t)n * (4 + 4 + 3 * kH), s);
    if (st != GVE_OK) return st;
    float* Y = (float*)c->a_tmp.p;
    float* dY = Y + 4 * n;
    float* save = dY + 4 * n;
    const unsigned g = (unsigned)((n + 127) / 128);
    k_mlp_fwd<<<g, 128, kFwdSmem, s>>>(model, features, n, Y, save);
    k_proposal_dy<<<g, 128, 0, s>>>(prims_corrected, grad_prims, Y, n, ls_min(), ls_max(d), dY);
    if (!accumulate) cudaMemsetAsync(dP, 0, sizeof(float) * kP, s);
    k_mlp_bwd<<<(unsigned)((n + kBR - 1) / kBR), kBR, kBwdSmem, s>>>(model, features, save, dY, n, dP);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "proposal backward");
    return GVE_OK;
}

// ---- training-set statistics and targets ------------------------------------
// Column mean and spread of a row-major [rows][C] float32 matrix in FP64, in
// a fixed order (so the same data give the same bits): blocks sum contiguous
// row ranges, one block adds the block sums; the spread is the square root
// of the centred sum of squares over rows - 1 (a second pass), as for the
// sample standard deviation.
namespace gve {
namespace {

constexpr int kMomBlocks = 256;

template <int C>
__global__ void __launch_bounds__(256) k_col_sums(const float* __restrict__ X, long long rows,
                                                  const double* __restrict__ mean, double* __restrict__ part)
{
    __shared__ double sm[C][8];
    const long long chunk = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    double acc[C];
#pragma unroll
    for (int k = 0; k < C; ++k) acc[k] = 0.0;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double x = (double)X[r * C + k];
            const double d = mean ? x - mean[k] : x;
            acc[k] += mean ? d * d : d;
        }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < C) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sm[threadIdx.x][w];
        part[blockIdx.x * C + threadIdx.x] = v;
    }
}

// out[k] = sum of the block partials of column k, divided by `div`
template <int C>
__global__ void k_col_final(const double* __restrict__ part, int nb, double div, double* __restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= C) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[b * C + k];
    out[k] = v / div;
}

// moments[0..C) = column means, moments[C..2C) = column spreads
template <int C>
void col_moments(const float* X, long long rows, double* moments, double* part, cudaStream_t s)
{
    k_col_sums<C><<<kMomBlocks, 256, 0, s>>>(X, rows, nullptr, part);
    k_col_final<C><<<1, 32, 0, s>>>(part, kMomBlocks, (double)rows, moments);
    k_col_sums<C><<<kMomBlocks, 256, 0, s>>>(X, rows, moments, part);
    k_col_final<C><<<1, 32, 0, s>>>(part, kMomBlocks, rows > 1 ? (double)(rows - 1) : 1.0, moments + C);
}

// the network's input standardisation from the feature moments: a feature
// whose spread is at most 1e-3 (1 + |mean|) gets weight 0
__global__ void k_set_norm(const double* __restrict__ mom, float* __restrict__ model)
{
    const int k = threadIdx.x;
    if (k >= kIn) return;
    const double mean = mom[k], sd = sqrt(mom[kIn + k]);
    const bool live = sd > 1e-3 * (1.0 + fabs(mean));
    model[kOffNorm + k] = (float)mean;
    model[kOffNorm + kIn + k] = live ? (float)(1.0 / fmax(sd, 1e-30)) : 0.f;
}

// refined minus allocated (a, log s0, log s1, log s2)
__global__ void k_targets(const float* __restrict__ p0, const float* __restrict__ p1, long long n, float* __restrict__ T)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* a = p0 + 12 * i;
    const float* b = p1 + 12 * i;
    reinterpret_cast<float4*>(T)[i] = make_float4(b[10] - a[10], b[3] - a[3], b[4] - a[4], b[5] - a[5]);
}

// scale[k] = max(spread_k, 1e-6) (float32); T[:, k] /= scale[k]
__global__ void k_target_scale(const double* __restrict__ mom, float* __restrict__ scale)
{
    const int k = threadIdx.x;
    if (k < kOut) scale[k] = (float)fmax(sqrt(mom[kOut + k]), 1e-6);
}

__global__ void k_div_cols(float* __restrict__ T, long long n, const float* __restrict__ scale)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 t = reinterpret_cast<float4*>(T)[i];
    t.x /= scale[0]; t.y /= scale[1]; t.z /= scale[2]; t.w /= scale[3];
    reinterpret_cast<float4*>(T)[i] = t;
}

// last layer rows k scaled by scale[k]: the network then predicts the
// unscaled targets
__global__ void k_fold_scale(float* __restrict__ model, const float* __restrict__ scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kOut * kH) model[kOffW4 + i] *= scale[i / kH];
    else if (i < kOut * kH + kOut) model[kOffB4 + (i - kOut * kH)] *= scale[i - kOut * kH];
}

}  // namespace
}  // namespace gve

extern "C" gve_status gve_mlp_standardise(gve_ctx* c, float* model, const float* X, int64_t rows, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || !X || rows < 1) return fail(c, GVE_E_INVALID, "bad standardisation arguments");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    gve_status st = ensure(c, c->a_cnt, sizeof(double) * (kMomBlocks * kIn + 2 * kIn), s);
    if (st != GVE_OK) return st;
    double* part = (double*)c->a_cnt.p;
    double* mom = part + kMomBlocks * kIn;
    col_moments<kIn>(X, rows, mom, part, s);
    k_set_norm<<<1, 32, 0, s>>>(mom, model);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp standardise");
    return GVE_OK;
}

extern "C" gve_status gve_proposal_targets(gve_ctx* c, const float* prims0, const float* prims1, int64_t n,
                                           float* T, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!prims0 || !prims1 || !T || n < 1) return fail(c, GVE_E_INVALID, "bad target arguments");
    if (reinterpret_cast<uintptr_t>(T) & 15u) return fail(c, GVE_E_INVALID, "targets not 16-byte aligned");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    k_targets<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(prims0, prims1, n, T);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "proposal targets");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_scale_targets(gve_ctx* c, float* T, int64_t rows, float* scale, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!T || !scale || rows < 1) return fail(c, GVE_E_INVALID, "bad target arguments");
    if (reinterpret_cast<uintptr_t>(T) & 15u) return fail(c, GVE_E_INVALID, "targets not 16-byte aligned");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    gve_status st = ensure(c, c->a_cnt, sizeof(double) * (kMomBlocks * kIn + 2 * kIn), s);
    if (st != GVE_OK) return st;
    double* part = (double*)c->a_cnt.p;
    double* mom = part + kMomBlocks * kIn;
    col_moments<kOut>(T, rows, mom, part, s);
    k_target_scale<<<1, 32, 0, s>>>(mom, scale);
    k_div_cols<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(T, rows, scale);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "scale targets");
    return GVE_OK;
}

extern "C" gve_status gve_mlp_fold_output_scale(gve_ctx* c, float* model, const float* scale, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!model || !scale) return fail(c, GVE_E_INVALID, "null argument");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    k_fold_scale<<<(kOut * kH + kOut + 255) / 256, 256, 0, s>>>(model, scale);
    k_mlp_quantise<<<(kP + 255) / 256, 256, 0, s>>>(model);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mlp fold");
    return GVE_OK;
}
