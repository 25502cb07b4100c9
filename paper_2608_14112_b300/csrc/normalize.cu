// normalize.cu -- stage P of the encoder (Sec. III-B): the field rescaled to
// [0, 1] by its own extremes, out = (V - min) / (max - min) in float32 with
// one correctly rounded subtraction and one correctly rounded division per
// voxel (so the result is bit-identical to any IEEE float32 evaluation of the
// same two operations); a constant field maps to 0.
//
// Two streaming passes over the field (HBM bound): a min / max / finiteness
// reduction (per-block partials, then one block), the host reads the three
// results, then the scaling pass.  16-byte vector loads and stores where the
// buffers allow them.
#include <cfloat>
#include <cmath>

#include "gve_int.cuh"

namespace gve {

namespace {

struct MinMax {
    float mn, mx;
    int bad;
};

__device__ __forceinline__ void mm_add(MinMax& m, float v)
{
    if (!isfinite(v)) {
        m.bad = 1;
        return;
    }
    m.mn = fminf(m.mn, v);
    m.mx = fmaxf(m.mx, v);
}

__device__ __forceinline__ MinMax mm_block(MinMax m, MinMax* smem /* [32] */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m.mn = fminf(m.mn, __shfl_xor_sync(0xffffffffu, m.mn, o));
        m.mx = fmaxf(m.mx, __shfl_xor_sync(0xffffffffu, m.mx, o));
        m.bad |= __shfl_xor_sync(0xffffffffu, m.bad, o);
    }
    if (lane == 0) smem[w] = m;
    __syncthreads();
    if (w == 0) {
        m = lane < nw ? smem[lane] : MinMax{FLT_MAX, -FLT_MAX, 0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m.mn = fminf(m.mn, __shfl_xor_sync(0xffffffffu, m.mn, o));
            m.mx = fmaxf(m.mx, __shfl_xor_sync(0xffffffffu, m.mx, o));
            m.bad |= __shfl_xor_sync(0xffffffffu, m.bad, o);
        }
    }
    return m;
}

// per-block min / max / non-finite flag; vec = the field is 16-byte aligned
__global__ void __launch_bounds__(256) k_minmax(const float* __restrict__ V, long long M, int vec,
                                                MinMax* __restrict__ part)
{
    __shared__ MinMax sm[32];
    MinMax m{FLT_MAX, -FLT_MAX, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec) {
        const long long nv = M >> 2;
        const float4* V4 = reinterpret_cast<const float4*>(V);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
            const float4 v = __ldcs(V4 + i);
            mm_add(m, v.x);
            mm_add(m, v.y);
            mm_add(m, v.z);
            mm_add(m, v.w);
        }
        done = nv << 2;
    }
    for (long long i = done + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) mm_add(m, V[i]);
    m = mm_block(m, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void __launch_bounds__(1024) k_minmax_final(MinMax* __restrict__ part, int nb)
{
    __shared__ MinMax sm[32];
    MinMax m{FLT_MAX, -FLT_MAX, 0};
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const MinMax p = part[i];
        m.mn = fminf(m.mn, p.mn);
        m.mx = fmaxf(m.mx, p.mx);
        m.bad |= p.bad;
    }
    m = mm_block(m, sm);
    if (threadIdx.x == 0) part[nb] = m;
}

__device__ __forceinline__ float scale1(float v, float mn, float range)
{
    return range > 0.0f ? __fdiv_rn(__fsub_rn(v, mn), range) : 0.0f;
}

__global__ void __launch_bounds__(256) k_scale(const float* V, long long M, int vec, float mn, float range, float* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec) {
        const long long nv = M >> 2;
        const float4* V4 = reinterpret_cast<const float4*>(V);
        float4* O4 = reinterpret_cast<float4*>(out);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
            const float4 v = __ldcs(V4 + i);
            __stcs(O4 + i, make_float4(scale1(v.x, mn, range), scale1(v.y, mn, range), scale1(v.z, mn, range),
                                       scale1(v.w, mn, range)));
        }
        done = nv << 2;
    }
    for (long long i = done + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        out[i] = scale1(V[i], mn, range);
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_normalize(gve_ctx* c, const float* field, gve_dims d, float* out, float* minmax,
                                    void* stream)
{
    if (!c) return GVE_E_INVALID;
    if (!field || !out) return fail(c, GVE_E_INVALID, "null field");
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(c, GVE_E_INVALID, "non-positive grid size");
    if (d.nx > (1 << 24) || d.ny > (1 << 24) || d.nz > (1 << 24)) return fail(c, GVE_E_INVALID, "grid axis above 2^24");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    const long long M = (long long)d.nx * d.ny * d.nz;
    const int vec = ((reinterpret_cast<uintptr_t>(field) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    long long nb = (M / (vec ? 4 : 1) + 255) / 256;
    const long long cap = 8LL * num_sms();
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    gve_status st = ensure(c, c->a_tmp, sizeof(MinMax) * (nb + 1), s);
    if (st != GVE_OK) return st;
    MinMax* part = reinterpret_cast<MinMax*>(c->a_tmp.p);
    k_minmax<<<(unsigned)nb, 256, 0, s>>>(field, M, vec, part);
    k_minmax_final<<<1, 1024, 0, s>>>(part, (int)nb);
    c->launches += 2;
    MinMax h;
    cudaError_t e = cudaMemcpyAsync(&h, part + nb, sizeof(MinMax), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "normalize readback");
    if (h.bad) return fail(c, GVE_E_INVALID, "non-finite value in the field (nothing written)");
    const float range = h.mx - h.mn;   // one float32 subtraction, as in the kernel
    k_scale<<<(unsigned)nb, 256, 0, s>>>(field, M, vec, h.mn, range, out);
    c->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "launch (normalize)");
    if (minmax) {
        minmax[0] = h.mn;
        minmax[1] = h.mx;
    }
    return GVE_OK;
}
