// render.cu -- mixture-field ray marching (Sec. III-A: the transfer function
// T = (c_T, alpha_T) maps the value Eq. 3 returns at sample positions along
// each ray to colour and opacity, composited front to back; grad Vt shades
// the sample).
//
// Preparation (once per primitive set): the keep coefficients, then cells of
// 8^3 voxels over the continuous volume box (cell c of an axis covers
// [8c - 1/2, 8c + 15/2)), each listing every Gaussian whose conservative
// truncation box overlaps it.  The lists come from the binner's pieces
// (count, scan, emit, stable radix sort by cell, ranges), so a cell's
// Gaussians are in index order, and their coefficients are gathered into
// cell order (48 B per pair) so that the march reads them contiguously.
//
// March: one thread per pixel, 16 x 8 pixel tiles per CTA, 8 x 4 per warp.  A thread takes
// its samples in order and groups consecutive samples of one cell (up to 8;
// 4 when shading, which carries the gradient sums); each group walks the
// cell's list once, testing every sample of the group against each record
// with the voxel path's float32 keep chain.  Sums are float32.  Ray setup and
// sample positions use explicitly rounded float32 operations in a fixed
// order, so the samples and the keep decisions are those of the CPU
// reference.
#include <climits>
#include <cmath>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr int kCellShift = 3;  // 8^3-voxel cells
constexpr float kCellInv = 0.125f;
constexpr float kLn2 = 0.693147180559945309f;
constexpr long long kMaxSamplesPerRay = 65536;

struct RenderGeom {
    int nx, ny, nz, ncx, ncy, ncz;
};

__device__ __forceinline__ int cell_axis(float p, int nc)
{
    const float f = floorf(__fmul_rn(__fadd_rn(p, 0.5f), kCellInv));
    const int c = f < 0.f ? 0 : (f > (float)(nc - 1) ? nc - 1 : (int)f);
    return c;
}

// Which cells of the box range a Gaussian's kept points can reach.  The
// kb-ellipsoid {m <= kb} lies on the near side of the plane <c - mu, x - mu>_M
// = kb |c - mu|_M (Cauchy-Schwarz in the Mahalanobis inner product, c the
// cell's centre); a cell whose whole box, dilated by the box's 0.05-voxel
// slack, lies beyond it holds no kept point: with v = c - mu, g = Sigma^-1 v,
// m2 = v.g and D = m2 - h sum |g_j| (h the dilated half edge), the cell is
// dropped when D > 0 and D^2 > kb^2 m2 (kb widened by 0.1 % for the float32
// evaluation).
struct CellCull {
    float mu[3], C[6], kb2;
    bool on;
};

__device__ __forceinline__ bool cell_kept(const CellCull& q, int cx, int cy, int cz)
{
    if (!q.on) return true;
    const float h = 0.5f * (float)(1 << kCellShift) + 0.05f;
    const float v0 = (float)(cx << kCellShift) + 0.5f * (float)((1 << kCellShift) - 1) - q.mu[0];
    const float v1 = (float)(cy << kCellShift) + 0.5f * (float)((1 << kCellShift) - 1) - q.mu[1];
    const float v2 = (float)(cz << kCellShift) + 0.5f * (float)((1 << kCellShift) - 1) - q.mu[2];
    const float g0 = q.C[0] * v0 + q.C[3] * v1 + q.C[4] * v2;
    const float g1 = q.C[3] * v0 + q.C[1] * v1 + q.C[5] * v2;
    const float g2 = q.C[4] * v0 + q.C[5] * v1 + q.C[2] * v2;
    const float m2 = v0 * g0 + v1 * g1 + v2 * g2;
    const float D = m2 - h * (fabsf(g0) + fabsf(g1) + fabsf(g2));
    return !(D > 0.f && D * D > q.kb2 * m2);
}

// cell range of Gaussian i (and its cell test); false when it lists no cell
__device__ __forceinline__ bool render_cells(const float* prims, const float4* rec, long long i, float k,
                                             const RenderGeom& g, int lo[3], int hi[3], CellCull& cull)
{
    cull.on = false;
    if (!(rec[3 * i + 2].z > 0.f)) return false;  // invalid record (weight zero)
    float mu[3], rad[3], kb = 0.f;
    const int kind = gauss_box(prims, i, k, mu, rad, &kb, cull.C);
    if (kind == 0) return false;
    const int dims[3] = {g.nx, g.ny, g.nz}, nc[3] = {g.ncx, g.ncy, g.ncz};
    if (kind == 2) {
        for (int j = 0; j < 3; ++j) { lo[j] = 0; hi[j] = nc[j] - 1; }
        return true;
    }
    bool fin = isfinite(kb);
    for (int q = 0; q < 6; ++q) fin = fin && isfinite(cull.C[q]);
    if (fin) {
        const float kw = kb * 1.001f;
        cull.kb2 = kw * kw;
        for (int j = 0; j < 3; ++j) cull.mu[j] = mu[j];
        cull.on = true;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float l = mu[j] - rad[j], h = mu[j] + rad[j];
        if (!(h >= -0.5f) || !(l <= (float)dims[j] - 0.5f)) return false;
        lo[j] = cell_axis(l, nc[j]);
        hi[j] = cell_axis(h, nc[j]);
    }
    return true;
}

__global__ void __launch_bounds__(256) k_render_count(const float* __restrict__ prims, const float4* __restrict__ rec,
                                                      long long n, float k, RenderGeom g, uint32_t* __restrict__ cnt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo[3], hi[3];
    CellCull cull;
    uint32_t c = 0;
    if (render_cells(prims, rec, i, k, g, lo, hi, cull))
        for (int cz = lo[2]; cz <= hi[2]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cx = lo[0]; cx <= hi[0]; ++cx) c += cell_kept(cull, cx, cy, cz) ? 1u : 0u;
    cnt[i] = c;
}

__global__ void __launch_bounds__(256) k_render_emit(const float* __restrict__ prims, const float4* __restrict__ rec,
                                                     long long n, float k, RenderGeom g,
                                                     const unsigned long long* __restrict__ off,
                                                     uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo[3], hi[3];
    CellCull cull;
    if (!render_cells(prims, rec, i, k, g, lo, hi, cull)) return;
    unsigned long long o = off[i];
    for (int cz = lo[2]; cz <= hi[2]; ++cz)
        for (int cy = lo[1]; cy <= hi[1]; ++cy)
            for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                if (!cell_kept(cull, cx, cy, cz)) continue;
                keys[o] = (uint32_t)(((long long)cz * g.ncy + cy) * g.ncx + cx);
                vals[o] = (uint32_t)i;
                ++o;
            }
}

// coefficients of the sorted pairs, in cell order
__global__ void __launch_bounds__(256) k_render_gather(const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                                       unsigned long long total, float4* __restrict__ crec)
{
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < total;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const long long gidx = vals[j];
        crec[3 * j] = rec[3 * gidx];
        crec[3 * j + 1] = rec[3 * gidx + 1];
        crec[3 * j + 2] = rec[3 * gidx + 2];
    }
}

struct RenderArgs {
    const float4* crec;
    const uint32_t* start;
    const uint32_t* end;
    RenderGeom g;
    float T, rho0;
    int normalized;
    float eye[3], right[3], up[3], fwd[3];
    float th;
    int W, H;
    float step, term, ratio;
    float bg[3];
    float ka, kd, ks, shin, gfloor;
    const float4* tf;
    int ntf;
    float4* image;
    unsigned long long* kept;    // [0] kept pairs, [1] tested pairs (optional)
};

// Ray through pixel (i, j): unit direction and the box interval; false for
// a miss or a degenerate camera.  Explicit roundings, in the written order.
__device__ __forceinline__ bool ray_setup(const RenderArgs& a, int i, int j, float d[3], float& t0, float& t1)
{
    const float aspect = __fdiv_rn((float)a.W, (float)a.H);
    const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)a.W), 1.0f), __fmul_rn(a.th, aspect));
    const float sy = __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * j + 1), (float)a.H)), a.th);
    float dd[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) dd[q] = __fadd_rn(__fadd_rn(a.fwd[q], __fmul_rn(sx, a.right[q])), __fmul_rn(sy, a.up[q]));
    const float n2a = __fadd_rn(__fmul_rn(dd[0], dd[0]), __fmul_rn(dd[1], dd[1]));
    const float n2 = __fadd_rn(n2a, __fmul_rn(dd[2], dd[2]));
    if (!(n2 > 0.0f) || !isfinite(n2)) return false;
    const float nrm = __fsqrt_rn(n2);
#pragma unroll
    for (int q = 0; q < 3; ++q) d[q] = __fdiv_rn(dd[q], nrm);
    t0 = 0.0f;
    t1 = INFINITY;
    const int dims[3] = {a.g.nx, a.g.ny, a.g.nz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float lo = -0.5f, hi = __fsub_rn((float)dims[q], 0.5f);
        if (d[q] == 0.0f) {
            if (a.eye[q] < lo || a.eye[q] > hi) return false;
            continue;
        }
        const float ta = __fdiv_rn(__fsub_rn(lo, a.eye[q]), d[q]), tb = __fdiv_rn(__fsub_rn(hi, a.eye[q]), d[q]);
        const float ta0 = ta < tb ? ta : tb, tb0 = ta < tb ? tb : ta;
        if (ta0 > t0) t0 = ta0;
        if (tb0 < t1) t1 = tb0;
    }
    return t0 < t1 && isfinite(t1);
}

template <bool SHADE>
__global__ void __launch_bounds__(128, SHADE ? 4 : 5) k_render(const RenderArgs a)
{
    constexpr int G = SHADE ? 4 : 8;
    // 16 x 8 pixels per CTA, 8 x 4 per warp (neighbouring rays share cells)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int j = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    unsigned long long kept = 0, tested = 0;
    if (i < a.W && j < a.H) {
        float d[3], t0 = 0.f, t1 = 0.f;
        float Tr = 1.f, C[3] = {0.f, 0.f, 0.f};
        bool done = !ray_setup(a, i, j, d, t0, t1);
        long long k = 0;
        while (!done) {
            // the next run of up to G samples inside one cell
            float px[G], py[G], pz[G];
            int gs = 0;
            uint32_t cell = 0;
#pragma unroll
            for (int s = 0; s < G; ++s) {
                px[s] = py[s] = pz[s] = 0.f;
                if (gs == s && k < kMaxSamplesPerRay) {
                    const float t = __fadd_rn(t0, __fmul_rn(__fadd_rn((float)k, 0.5f), a.step));
                    if (t < t1) {
                        const float x = __fadd_rn(a.eye[0], __fmul_rn(t, d[0]));
                        const float y = __fadd_rn(a.eye[1], __fmul_rn(t, d[1]));
                        const float z = __fadd_rn(a.eye[2], __fmul_rn(t, d[2]));
                        const uint32_t c =
                            ((uint32_t)cell_axis(z, a.g.ncz) * (uint32_t)a.g.ncy + (uint32_t)cell_axis(y, a.g.ncy)) *
                                (uint32_t)a.g.ncx + (uint32_t)cell_axis(x, a.g.ncx);
                        if (s == 0 || c == cell) {
                            px[s] = x; py[s] = y; pz[s] = z;
                            cell = c;
                            ++gs;
                            ++k;
                        }
                    }
                }
            }
            if (gs == 0) break;
            float N[G], D[G], gN[SHADE ? G : 1][3], gD[SHADE ? G : 1][3];
#pragma unroll
            for (int s = 0; s < G; ++s) {
                N[s] = D[s] = 0.f;
                if (SHADE)
                    for (int q = 0; q < 3; ++q) gN[s][q] = gD[s][q] = 0.f;
            }
            const uint32_t b = a.start[cell], e = a.end[cell];
            tested += (unsigned long long)(e - b) * (unsigned)gs;
            // the next record is loaded while the current one is tested
            const float4* rp = a.crec + 3ull * b;
            float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0;
            if (b < e) { n0 = rp[0]; n1 = rp[1]; n2 = rp[2]; }
            uint32_t kept_g = 0;
            for (uint32_t jj = b; jj < e; ++jj) {
                const float4 r0 = n0, r1 = n1, r2 = n2;
                rp += 3;
                if (jj + 1 < e) { n0 = rp[0]; n1 = rp[1]; n2 = rp[2]; }
                // the keep chain for two samples per packed instruction, in
                // keep_t's order (p - mu as p + (-mu): the same value)
                const float2 nmx = make_float2(-r0.x, -r0.x), nmy = make_float2(-r0.y, -r0.y),
                             nmz = make_float2(-r0.z, -r0.z);
                const float2 cxx = make_float2(r0.w, r0.w), cyy = make_float2(r1.x, r1.x),
                             czz = make_float2(r1.y, r1.y), cxy = make_float2(r1.z, r1.z),
                             cxz = make_float2(r1.w, r1.w), cyz = make_float2(r2.x, r2.x);
                float tt[G], dxs[G], dys[G], dzs[G];
#pragma unroll
                for (int q = 0; q < G / 2; ++q) {
                    if (2 * q < gs) {
                        const float2 dx = __fadd2_rn(make_float2(px[2 * q], px[2 * q + 1]), nmx);
                        const float2 dy = __fadd2_rn(make_float2(py[2 * q], py[2 * q + 1]), nmy);
                        const float2 dz = __fadd2_rn(make_float2(pz[2 * q], pz[2 * q + 1]), nmz);
                        const float2 b2 = __ffma2_rn(cxy, dy, __fmul2_rn(cxz, dz));
                        const float2 c2 = __ffma2_rn(dy, __ffma2_rn(cyy, dy, __fmul2_rn(cyz, dz)),
                                                     __fmul2_rn(dz, __fmul2_rn(czz, dz)));
                        const float2 t2 = __ffma2_rn(dx, __ffma2_rn(cxx, dx, b2), c2);
                        tt[2 * q] = t2.x;
                        tt[2 * q + 1] = 2 * q + 1 < gs ? t2.y : -INFINITY;  // an odd run's last lane is empty
                        dxs[2 * q] = dx.x; dxs[2 * q + 1] = dx.y;
                        dys[2 * q] = dy.x; dys[2 * q + 1] = dy.y;
                        dzs[2 * q] = dz.x; dzs[2 * q + 1] = dz.y;
                    } else {
                        tt[2 * q] = tt[2 * q + 1] = -INFINITY;
                        dxs[2 * q] = dxs[2 * q + 1] = dys[2 * q] = dys[2 * q + 1] = dzs[2 * q] = dzs[2 * q + 1] = 0.f;
                    }
                }
#pragma unroll
                for (int s = 0; s < G; ++s) {
                    {  // slots past the run hold -inf
                        const float dx = dxs[s], dy = dys[s], dz = dzs[s];
                        const float t = tt[s];
                        if (t > a.T) {
                            const float gv = ex2_approx(t);
                            N[s] = fmaf(r2.y, gv, N[s]);
                            D[s] = fmaf(r2.z, gv, D[s]);
                            ++kept_g;
                            if (SHADE) {
                                // grad G = G ln2 grad t, grad t = 2 Q d in the coefficient layout
                                const float lg = gv * kLn2;
                                const float gx = fmaf(2.f * r0.w, dx, fmaf(r1.z, dy, r1.w * dz));
                                const float gy = fmaf(r1.z, dx, fmaf(2.f * r1.x, dy, r2.x * dz));
                                const float gz = fmaf(r1.w, dx, fmaf(r2.x, dy, 2.f * r1.y * dz));
                                const float an = r2.y * lg, ad = r2.z * lg;
                                gN[s][0] = fmaf(an, gx, gN[s][0]);
                                gN[s][1] = fmaf(an, gy, gN[s][1]);
                                gN[s][2] = fmaf(an, gz, gN[s][2]);
                                gD[s][0] = fmaf(ad, gx, gD[s][0]);
                                gD[s][1] = fmaf(ad, gy, gD[s][1]);
                                gD[s][2] = fmaf(ad, gz, gD[s][2]);
                            }
                        }
                    }
                }
            }
            kept += kept_g;
            // classify, shade and composite the group's samples in order
#pragma unroll
            for (int s = 0; s < G; ++s) {
                if (s < gs && !done) {
                    float v, gv3[3] = {0.f, 0.f, 0.f};
                    if (!a.normalized) {
                        v = N[s];
                        if (SHADE)
                            for (int q = 0; q < 3; ++q) gv3[q] = gN[s][q];
                    } else if (D[s] > a.rho0) {
                        v = N[s] / D[s];
                        if (SHADE) {
                            const float inv = 1.f / (D[s] * D[s]);
                            for (int q = 0; q < 3; ++q) gv3[q] = (gN[s][q] * D[s] - N[s] * gD[s][q]) * inv;
                        }
                    } else {
                        v = N[s] / a.rho0;
                        if (SHADE)
                            for (int q = 0; q < 3; ++q) gv3[q] = gN[s][q] / a.rho0;
                    }
                    const float vc = fminf(fmaxf(v, 0.f), 1.f);
                    const float u = vc * (float)(a.ntf - 1);
                    int i0 = (int)u;
                    i0 = i0 > a.ntf - 2 ? a.ntf - 2 : i0;
                    const float fr = u - (float)i0;
                    const float4 A = __ldg(a.tf + i0), B = __ldg(a.tf + i0 + 1);
                    float c[3] = {fmaf(fr, B.x - A.x, A.x), fmaf(fr, B.y - A.y, A.y), fmaf(fr, B.z - A.z, A.z)};
                    const float a0 = fminf(fmaxf(fmaf(fr, B.w - A.w, A.w), 0.f), 1.f);
                    const float as = 1.f - powf(1.f - a0, a.ratio);
                    if (SHADE) {
                        const float gl = sqrtf(gv3[0] * gv3[0] + gv3[1] * gv3[1] + gv3[2] * gv3[2]);
                        const float ndl =
                            fabsf(gv3[0] * d[0] + gv3[1] * d[1] + gv3[2] * d[2]) / fmaxf(gl, a.gfloor);
                        const float sf = fmaf(a.kd, ndl, a.ka), sp = a.ks * powf(ndl, a.shin);
                        for (int q = 0; q < 3; ++q) c[q] = fmaf(c[q], sf, sp);
                    }
                    const float w = Tr * as;
                    for (int q = 0; q < 3; ++q) C[q] = fmaf(w, c[q], C[q]);
                    Tr = Tr * (1.f - as);
                    if (a.term > 0.f && Tr < a.term) done = true;
                }
            }
        }
        a.image[(long long)j * a.W + i] =
            make_float4(fmaf(Tr, a.bg[0], C[0]), fmaf(Tr, a.bg[1], C[1]), fmaf(Tr, a.bg[2], C[2]), 1.f - Tr);
    }
    if (a.kept) {
        for (int o = 16; o > 0; o >>= 1) {
            kept += __shfl_xor_sync(0xffffffffu, kept, o);
            tested += __shfl_xor_sync(0xffffffffu, tested, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (kept) atomicAdd(a.kept, kept);
            if (tested) atomicAdd(a.kept + 1, tested);
        }
    }
}

int key_bits_for(unsigned long long ncells)
{
    int b = 1;
    while (b < 32 && (1ull << b) < ncells) ++b;
    return b;
}

}  // namespace

}  // namespace gve

using namespace gve;

#define RTRY(x)                                \
    do {                                       \
        gve_status st_ = (x);                  \
        if (st_ != GVE_OK) return st_;         \
    } while (0)
#define RCUDA(x, what)                                        \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

extern "C" {

gve_status gve_render_prepare(gve_ctx* c, const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                              void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!o) return fail(c, GVE_E_INVALID, "null options");
    if (n < 0 || (n > 0 && !prims)) return fail(c, GVE_E_INVALID, "bad primitive array");
    if (reinterpret_cast<uintptr_t>(prims) & 15u) return fail(c, GVE_E_INVALID, "primitives not 16-byte aligned");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (d.nx > (1 << 20) || d.ny > (1 << 20) || d.nz > (1 << 20)) return fail(c, GVE_E_INVALID, "grid axis above 2^20");
    if (n > (int64_t)UINT32_MAX) return fail(c, GVE_E_INVALID, "more than 2^32 - 1 primitives");
    if (!(o->trunc_k > 0.f) || !isfinite(o->trunc_k) || !(o->rho0 > 0.f)) return fail(c, GVE_E_INVALID, "bad eval options");
    cudaStream_t s = (cudaStream_t)stream;
    RCUDA(cudaSetDevice(c->device), "cudaSetDevice");
    c->launches = 0;
    c->r_ready = false;
    RenderGeom g;
    g.nx = d.nx; g.ny = d.ny; g.nz = d.nz;
    g.ncx = ((d.nx - 1) >> kCellShift) + 1;
    g.ncy = ((d.ny - 1) >> kCellShift) + 1;
    g.ncz = ((d.nz - 1) >> kCellShift) + 1;
    const unsigned long long ncells = (unsigned long long)g.ncx * g.ncy * g.ncz;
    if (ncells >= (1ull << 32)) return fail(c, GVE_E_INVALID, "too many render cells");
    const long long nn = n > 0 ? n : 1;
    RTRY(ensure(c, c->r_rec, sizeof(float4) * 3 * nn, s));
    RTRY(ensure(c, c->r_cnt, sizeof(uint32_t) * nn, s));
    RTRY(ensure(c, c->r_off, sizeof(unsigned long long) * (nn + 1), s));
    RTRY(ensure(c, c->r_scanp, sizeof(unsigned long long) * kScanBlocks, s));
    RTRY(ensure(c, c->r_state, sizeof(DevState), s));
    RTRY(ensure(c, c->r_rng, sizeof(uint32_t) * 2 * ncells, s));
    DevState* st = (DevState*)c->r_state.p;
    RCUDA(cudaMemsetAsync(st, 0, sizeof(DevState), s), "memset render state");
    float4* rec = (float4*)c->r_rec.p;
    uint32_t* cnt = (uint32_t*)c->r_cnt.p;
    unsigned long long* off = (unsigned long long*)c->r_off.p;
    const unsigned nb = (unsigned)((nn + 255) / 256);
    if (n > 0) {
        launch_prep_rec(prims, n, o->trunc_k, rec, s);
        k_render_count<<<nb, 256, 0, s>>>(prims, rec, n, o->trunc_k, g, cnt);
        c->launches += 2;
    } else {
        RCUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), s), "memset counts");
    }
    launch_offsets(cnt, nn, off, c->r_scanp.p, st, ~0ull, 0, s);
    c->launches += 3;
    RCUDA(cudaGetLastError(), "launch (render count)");
    DevState h;
    RCUDA(cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s), "read render state");
    RCUDA(cudaStreamSynchronize(s), "render count");
    const unsigned long long total = h.total;
    if (total >= (1ull << 32)) return fail(c, GVE_E_CAPACITY, "render pairs above 2^32");
    const unsigned long long cap = total > 0 ? total : 1;
    for (int q = 0; q < 2; ++q) {
        RTRY(ensure(c, c->r_keys[q], sizeof(uint32_t) * (cap + 4), s));
        RTRY(ensure(c, c->r_vals[q], sizeof(uint32_t) * (cap + 4), s));
    }
    RTRY(ensure(c, c->r_hist, sizeof(uint32_t) * 256 * ((cap + kSortTile - 1) / kSortTile + 1), s));
    RTRY(ensure(c, c->r_crec, sizeof(float4) * 3 * cap, s));
    uint32_t* kk[2] = {(uint32_t*)c->r_keys[0].p, (uint32_t*)c->r_keys[1].p};
    uint32_t* vv[2] = {(uint32_t*)c->r_vals[0].p, (uint32_t*)c->r_vals[1].p};
    uint32_t* start = (uint32_t*)c->r_rng.p;
    RCUDA(cudaMemsetAsync(start, 0, sizeof(uint32_t) * 2 * ncells, s), "memset render ranges");
    if (total > 0) {
        k_render_emit<<<nb, 256, 0, s>>>(prims, rec, n, o->trunc_k, g, off, kk[0], vv[0]);
        const int kb = key_bits_for(ncells);
        const int sorted = launch_sort(kk, vv, &st->total, &st->overflow, cap, kb, (uint32_t*)c->r_hist.p, c->r_scanp.p, s);
        launch_ranges(kk[sorted], &st->total, &st->overflow, cap, start, start + ncells, s);
        const unsigned gb = (unsigned)std::min<unsigned long long>((total + 255) / 256, 16ull * num_sms());
        k_render_gather<<<gb, 256, 0, s>>>(rec, vv[sorted], total, (float4*)c->r_crec.p);
        c->launches += 1 + 5 * ((kb + 7) / 8) + 1 + 1;
    }
    RCUDA(cudaGetLastError(), "launch (render lists)");
    RCUDA(cudaStreamSynchronize(s), "render lists");
    c->r_dims[0] = d.nx; c->r_dims[1] = d.ny; c->r_dims[2] = d.nz;
    c->r_nc[0] = g.ncx; c->r_nc[1] = g.ncy; c->r_nc[2] = g.ncz;
    c->r_T = (float)((double)o->trunc_k * (double)o->trunc_k * kNegHalfLog2e);
    c->r_rho0 = o->rho0;
    c->r_norm = o->normalized ? 1 : 0;
    c->r_pairs = total;
    c->r_ready = true;
    return GVE_OK;
}

gve_status gve_render(gve_ctx* c, const gve_camera* cam, const gve_render_opts* o, float* image, int64_t* kept_pairs,
                      int64_t* tested_pairs, void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!c->r_ready) return fail(c, GVE_E_INVALID, "no prepared primitive set (call gve_render_prepare)");
    if (!cam || !o || !image || !o->tf_dev) return fail(c, GVE_E_INVALID, "null argument");
    if (cam->width < 1 || cam->height < 1 || cam->height > 65535 * 8 || (long long)cam->width * cam->height > (1ll << 28))
        return fail(c, GVE_E_INVALID, "image size");
    const float* cv[4] = {cam->eye, cam->right, cam->up, cam->forward};
    for (const float* v : cv)
        for (int q = 0; q < 3; ++q)
            if (!isfinite(v[q])) return fail(c, GVE_E_INVALID, "non-finite camera");
    if (!isfinite(cam->tan_half_fovy) || !(cam->tan_half_fovy > 0.f)) return fail(c, GVE_E_INVALID, "bad field of view");
    if (o->tf_n < 2) return fail(c, GVE_E_INVALID, "transfer function needs at least 2 entries");
    const double diag = std::sqrt((double)c->r_dims[0] * c->r_dims[0] + (double)c->r_dims[1] * c->r_dims[1] +
                                  (double)c->r_dims[2] * c->r_dims[2]);
    if (!(o->step >= 1.0f / 64.0f) || !isfinite(o->step) || diag / o->step > (double)kMaxSamplesPerRay)
        return fail(c, GVE_E_INVALID, "step below 1/64 voxel or above 65,536 samples per ray");
    if (!(o->ref_step > 0.f) || !isfinite(o->ref_step) || !(o->term >= 0.f) || !(o->term < 1.f))
        return fail(c, GVE_E_INVALID, "bad ref_step or term");
    if (o->shade && (!(o->gfloor > 0.f) || !isfinite(o->ka + o->kd + o->ks + o->shininess)))
        return fail(c, GVE_E_INVALID, "bad shading options");
    cudaStream_t s = (cudaStream_t)stream;
    RCUDA(cudaSetDevice(c->device), "cudaSetDevice");
    c->launches = 0;
    RenderArgs a{};
    a.crec = (const float4*)c->r_crec.p;
    a.start = (const uint32_t*)c->r_rng.p;
    const unsigned long long ncells = (unsigned long long)c->r_nc[0] * c->r_nc[1] * c->r_nc[2];
    a.end = a.start + ncells;
    a.g = RenderGeom{c->r_dims[0], c->r_dims[1], c->r_dims[2], c->r_nc[0], c->r_nc[1], c->r_nc[2]};
    a.T = c->r_T;
    a.rho0 = c->r_rho0;
    a.normalized = c->r_norm;
    for (int q = 0; q < 3; ++q) {
        a.eye[q] = cam->eye[q]; a.right[q] = cam->right[q]; a.up[q] = cam->up[q]; a.fwd[q] = cam->forward[q];
        a.bg[q] = o->background[q];
    }
    a.th = cam->tan_half_fovy;
    a.W = cam->width;
    a.H = cam->height;
    a.step = o->step;
    a.term = o->term;
    a.ratio = o->step / o->ref_step;
    a.ka = o->ka; a.kd = o->kd; a.ks = o->ks; a.shin = o->shininess; a.gfloor = o->gfloor;
    a.tf = (const float4*)o->tf_dev;
    a.ntf = o->tf_n;
    a.image = (float4*)image;
    unsigned long long* kd = nullptr;
    if (kept_pairs || tested_pairs) {
        RTRY(ensure(c, c->r_scanp, sizeof(unsigned long long) * kScanBlocks, s));
        kd = (unsigned long long*)c->r_scanp.p;
        RCUDA(cudaMemsetAsync(kd, 0, 2 * sizeof(unsigned long long), s), "memset kept");
    }
    a.kept = kd;
    const dim3 grid((unsigned)((a.W + 15) / 16), (unsigned)((a.H + 7) / 8));
    if (o->shade)
        k_render<true><<<grid, 128, 0, s>>>(a);
    else
        k_render<false><<<grid, 128, 0, s>>>(a);
    c->launches += 1;
    RCUDA(cudaGetLastError(), "launch (render)");
    if (kd) {
        unsigned long long hk[2] = {0, 0};
        RCUDA(cudaMemcpyAsync(hk, kd, sizeof(hk), cudaMemcpyDeviceToHost, s), "read kept");
        RCUDA(cudaStreamSynchronize(s), "render");
        if (kept_pairs) *kept_pairs = (int64_t)hk[0];
        if (tested_pairs) *tested_pairs = (int64_t)hk[1];
    }
    return GVE_OK;
}

}  // extern "C"
