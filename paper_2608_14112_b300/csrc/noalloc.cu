// noalloc.cu -- field evaluation that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or
// arena that owns the whole device, a host that must not grow its device
// footprint after start-up, or a caller that has to run without taking the
// allocator's locks.  gve_evaluate_noalloc serves them: it takes the same
// inputs and output as gve_evaluate, needs no context, and keeps all of its
// scratch (prepared records, tile and brick pairs, sort buffers, ranges,
// device state) in one fixed file-scope device array.  That array is part of the library
// image: every GPU that loads the library holds it (kScratchBytes) until the
// process exits, whether or not the entry point is used.
//
// Limits (checked before any launch; larger requests get GVE_E_INVALID):
//   primitives        <= GVE_NOALLOC_MAX_PRIMS   (8,192)
//   bricks of 8^3     <= GVE_NOALLOC_MAX_BRICKS  (32,768, e.g. a 256^3 grid)
//   (brick, Gaussian) pairs <= GVE_NOALLOC_MAX_PAIRS (524,288) and (tile,
//   Gaussian) pairs <= 131,072 (tiles of 4^3 bricks): data dependent, found
//   on the device; a larger count returns GVE_E_CAPACITY and leaves the
//   output unwritten.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress; that first call should
// come before any stream capture.  Later calls reuse the address (a device
// reset with cudaDeviceReset unloads the module and invalidates it, so the
// library must not be used across such a reset).
//
// Device: the inputs and the output must live on the current device (checked
// with cudaPointerGetAttributes; GVE_E_INVALID otherwise), because the array
// used is the current device's copy and the launches go to the current
// device.
//
// Sharing: every call uses the same array and finds the previous call's
// contents there; the part that must start at zero (the device state) is
// cleared by each call, and the binning rewrites everything else it reads.  Calls whose work overlaps on
// the GPU (different streams, or different host threads) race on the array
// and must be serialised by the caller.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>

#include "gve_int.cuh"

namespace gve {

namespace {

constexpr long long kNaPrims = GVE_NOALLOC_MAX_PRIMS;
constexpr long long kNaBricks = GVE_NOALLOC_MAX_BRICKS;
constexpr long long kNaPairs = GVE_NOALLOC_MAX_PAIRS;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// tile pairs (stage 1 of the binning): up to 16 per primitive on average;
// more return GVE_E_CAPACITY like the brick pairs
constexpr long long kNaTilePairs = 16 * kNaPrims;
// tiles of a grid of at most kNaBricks bricks with axes of at most 2^11
// bricks (the largest count, 2,410, is a 1 x 17 x 1,927-brick grid)
constexpr long long kNaTiles = 2410;

// carve-up of the scratch array (byte offsets)
constexpr size_t kOffState = 0;
constexpr size_t kOffRec = align256(kOffState + sizeof(DevState));
constexpr size_t kOffBin = align256(kOffRec + sizeof(float4) * 3 * kNaPrims);
constexpr size_t kOffTcount = align256(kOffBin + sizeof(BinRec) * kNaPrims);
constexpr size_t kOffToff = align256(kOffTcount + sizeof(uint32_t) * kNaPrims);
constexpr size_t kOffScan = align256(kOffToff + sizeof(unsigned long long) * (kNaPrims + 1));
constexpr size_t kOffTkeys0 = align256(kOffScan + sizeof(unsigned long long) * kScanBlocks);
constexpr size_t kOffTkeys1 = align256(kOffTkeys0 + sizeof(uint32_t) * kNaTilePairs);
constexpr size_t kOffTvals0 = align256(kOffTkeys1 + sizeof(uint32_t) * kNaTilePairs);
constexpr size_t kOffTvals1 = align256(kOffTvals0 + sizeof(uint32_t) * kNaTilePairs);
constexpr size_t kOffHist = align256(kOffTvals1 + sizeof(uint32_t) * kNaTilePairs);
constexpr size_t kOffTmask = align256(kOffHist + sizeof(uint32_t) * 256 * (kNaTilePairs / kSortTile + 1));
constexpr size_t kOffCbase = align256(kOffTmask + sizeof(unsigned long long) * kNaTilePairs);
constexpr size_t kOffTrange = align256(kOffCbase + sizeof(uint32_t) * 64 * (kNaTilePairs / 32 + kNaTiles + 2));
constexpr size_t kOffBcount = align256(kOffTrange + sizeof(uint32_t) * 2 * kNaTiles);
constexpr size_t kOffBoff = align256(kOffBcount + sizeof(uint32_t) * kNaBricks);
constexpr size_t kOffRanges = align256(kOffBoff + sizeof(unsigned long long) * (kNaBricks + 1));
constexpr size_t kOffPairs = align256(kOffRanges + sizeof(uint32_t) * 2 * kNaBricks);
constexpr size_t kScratchBytes = align256(kOffPairs + sizeof(uint32_t) * kNaPairs);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// per-device address of the array; two threads resolving it at once store
// the same value
std::atomic<unsigned char*> g_scratch_ptr[kMaxDevices];

gve_status scratch_for_device(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return GVE_E_CUDA;
    unsigned char* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* q = nullptr;
        if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) {
            cudaGetLastError();
            return GVE_E_CUDA;
        }
        p = static_cast<unsigned char*>(q);
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return GVE_OK;
}

// 1 when ptr is device (or managed) memory of device dev
bool on_device(const void* ptr, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

}  // namespace gve

using namespace gve;

extern "C" gve_status gve_evaluate_noalloc(const float* prims, int64_t n, gve_dims d, const gve_eval_opts* o,
                                           float* field_out, void* stream)
{
    if (!o || !field_out || (n > 0 && !prims)) return GVE_E_INVALID;
    if (n < 0 || n > kNaPrims) return GVE_E_INVALID;
    if (prims && (reinterpret_cast<uintptr_t>(prims) & 15u)) return GVE_E_INVALID;
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return GVE_E_INVALID;
    if (d.nx > (1 << 14) || d.ny > (1 << 14) || d.nz > (1 << 14)) return GVE_E_INVALID;
    if (o->brick != 8 || !(o->trunc_k > 0.f) || !std::isfinite(o->trunc_k)) return GVE_E_INVALID;
    if (o->gaussians_per_block != 0 && o->gaussians_per_block != 32 && o->gaussians_per_block != 64)
        return GVE_E_INVALID;
    if (o->normalized && !(o->rho0 > 0.f)) return GVE_E_INVALID;
    const BinGeom g = make_geom(d, 8);
    if (g.nbricks > kNaBricks || g.ntiles > kNaTiles) return GVE_E_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GVE_E_CUDA;
    }
    if (!on_device(field_out, dev) || (n > 0 && !on_device(prims, dev))) return GVE_E_INVALID;

    unsigned char* base = nullptr;
    gve_status st = scratch_for_device(dev, &base);
    if (st != GVE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DevState* dst = reinterpret_cast<DevState*>(base + kOffState);
    BinBufs b{};
    b.rec = reinterpret_cast<float4*>(base + kOffRec);
    b.br = reinterpret_cast<BinRec*>(base + kOffBin);
    b.tcount = reinterpret_cast<uint32_t*>(base + kOffTcount);
    b.toff = reinterpret_cast<unsigned long long*>(base + kOffToff);
    b.scanp = base + kOffScan;
    b.tkeys[0] = reinterpret_cast<uint32_t*>(base + kOffTkeys0);
    b.tkeys[1] = reinterpret_cast<uint32_t*>(base + kOffTkeys1);
    b.tvals[0] = reinterpret_cast<uint32_t*>(base + kOffTvals0);
    b.tvals[1] = reinterpret_cast<uint32_t*>(base + kOffTvals1);
    b.hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    b.tmask = reinterpret_cast<unsigned long long*>(base + kOffTmask);
    b.cbase = reinterpret_cast<uint32_t*>(base + kOffCbase);
    b.cap1 = (unsigned long long)kNaTilePairs;
    b.trange = reinterpret_cast<uint32_t*>(base + kOffTrange);
    b.bcount = reinterpret_cast<uint32_t*>(base + kOffBcount);
    b.boff = reinterpret_cast<unsigned long long*>(base + kOffBoff);
    b.ranges = reinterpret_cast<uint32_t*>(base + kOffRanges);
    b.pairs = reinterpret_cast<uint32_t*>(base + kOffPairs);
    b.cap = (unsigned long long)kNaPairs;
    b.gcount = nullptr;
    b.st = dst;

    // the device state must start at zero on every call (the ranges are
    // rewritten by every binning)
    if (cudaMemsetAsync(dst, 0, sizeof(DevState), s) != cudaSuccess) return GVE_E_CUDA;
    launch_binning(b, prims, n, single_volume(g, n), o->trunc_k, 0, s);
    BrickArgs a{};
    a.g = g;
    a.start = b.ranges;
    a.end = b.ranges + g.nbricks;
    a.gids = b.pairs;
    a.rec = b.rec;
    a.st = dst;
    a.T = (float)((double)o->trunc_k * (double)o->trunc_k * kNegHalfLog2e);
    a.rho0 = o->rho0;
    a.normalized = o->normalized;
    a.mask_thresh = -1.f;
    a.inv_m = (float)(1.0 / ((double)d.nx * d.ny * d.nz));
    a.chunk = o->gaussians_per_block;
    a.field_out = field_out;
    launch_brick(kModeEval, a, s);
    if (cudaGetLastError() != cudaSuccess) return GVE_E_CUDA;
    // the pair count is only known on the device: read the overflow flag
    int overflow = 0;
    if (cudaMemcpyAsync(&overflow, &dst->overflow, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GVE_E_CUDA;
    return overflow ? GVE_E_CAPACITY : GVE_OK;
}
