// optim.cu -- the per-Gaussian chain rule and fused Adam step as a kernel
// (the arithmetic is chain_one in chain.cuh).
#include "chain.cuh"

namespace gve {

__global__ void __launch_bounds__(128) k_chain(const float* acc, float* acc_zero,
                                               float* __restrict__ prims, long long n, float* __restrict__ grad,
                                               float* __restrict__ m, float* __restrict__ v, AdamArgs ad,
                                               int do_adam, const DevState* st, const float* __restrict__ extra)
{
    if (st && st->overflow) return;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    chain_one(i, acc, acc_zero, prims, grad, m, v, ad, do_adam, extra);
}

void launch_chain(const float* acc_in, float* acc_zero, float* prims, long long n, float* grad, float* m,
                  float* v, const AdamArgs* adam, const DevState* st, cudaStream_t s, const float* extra)
{
    if (n <= 0) return;
    AdamArgs ad{};
    if (adam) ad = *adam;
    k_chain<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(acc_in, acc_zero, prims, n, grad, m, v, ad,
                                                         adam != nullptr, st, extra);
}

}  // namespace gve
