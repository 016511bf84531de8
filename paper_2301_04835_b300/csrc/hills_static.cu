// Allocation-free hills sum.
//
// Some callers cannot allocate device memory: code running where a memory
// pool is owned by someone else (an MD engine's plugin that may only use the
// buffers the engine hands it), code between the phases of a caller's own
// allocator, or callers that must keep their memory footprint fixed after
// start-up.  For them this file offers one entry point that evaluates the
// metadynamics hills sum (V and dV/dxi at P points, in double precision)
// without calling cudaMalloc, cudaFree or any allocating routine.  It is a
// variant of the FP64 hills-sum kernel of hills.cu: the per-split partial sums
// that kernel keeps in handle-owned scratch live here in a fixed file-scope
// device array instead.
//
// The array is WTMD_STATIC_MAX_POINTS x 32 bytes (1 MiB); every GPU that
// loads the library holds it until the process exits.  All calls share it:
// two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it, so serialize them.  Each call writes
// every scratch entry it later reads, so the contents left by the previous
// call never leak into a result.
#include <cuda.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "wtmd_internal.cuh"

namespace {

using wtmd::dbl4;

constexpr int kHB = 256;
constexpr long long kScratchEntries = WTMD_STATIC_MAX_POINTS;

static __device__ __align__(256) dbl4 g_hills_scratch[kScratchEntries];

// Device address of g_hills_scratch.  A __device__ array exists once per CUDA
// context, and host code only holds a stand-in for it, so the address has to
// be looked up (cudaGetSymbolAddress) with the context current.  Most callers
// use the primary context of each device, and the lookup happens on their
// first call on that device; an engine that creates its own contexts gets one
// lookup per context.  Entries are kept against the context's unique id,
// which a process never reuses, so a context made after cudaDeviceReset (or a
// new context that happens to get the old handle value) is looked up afresh.
// The driver's context queries are reached through the runtime's entry-point
// lookup, so the library needs no link against libcuda.
struct ScratchEntry {
    unsigned long long ctx_id;
    void* addr;
};
constexpr int kMaxContexts = 64;
static ScratchEntry g_scratch[kMaxContexts];
static int g_n_scratch = 0;
static std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;
static bool g_ctx_fns_tried = false;

// Caller holds g_scratch_mutex.  False if the current context's id cannot be
// had (then nothing is cached and every call looks the address up).
static bool current_context_id(unsigned long long* id)
{
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!g_ctx_current || !g_ctx_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

int scratch_for_current_context(dbl4** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id)
        for (int k = 0; k < g_n_scratch; ++k)
            if (g_scratch[k].ctx_id == id) {
                *out = static_cast<dbl4*>(g_scratch[k].addr);
                return WTMD_OK;
            }
    // first call in this context (the lookup also makes the device's primary
    // context current when the caller has none)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_hills_scratch) != cudaSuccess || !p) return WTMD_ECUDA;
    if (!have_id) have_id = current_context_id(&id);
    if (have_id && g_n_scratch < kMaxContexts) g_scratch[g_n_scratch++] = ScratchEntry{id, p};
    *out = static_cast<dbl4*>(p);
    return WTMD_OK;
}

template <typename... KArgs, typename... Args>
cudaError_t launch(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

struct Prm {
    int d;
    double inv2s2[3];
    double per[3];
    double gs[3];  // dV/dxi_i = gs_i * sum_k e_k D_ki
};

template <int TH>
__device__ __forceinline__ void reduce_th(double acc[4])
{
    if constexpr (TH <= 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            for (int o = TH / 2; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    } else {
        __shared__ double red[kHB / 32][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (threadIdx.x % 32 == 0)
            for (int i = 0; i < 4; ++i) red[threadIdx.x / 32][i] = acc[i];
        __syncthreads();
        if (threadIdx.x % TH == 0) {
            const int w0 = threadIdx.x / 32;
            for (int i = 0; i < 4; ++i) {
                double s = 0.0;
                for (int w = 0; w < TH / 32; ++w) s += red[w0 + w][i];
                acc[i] = s;
            }
        }
    }
}

// Partial sums of one hill split for TP = kHB/TH points per CTA.
template <int TH>
__global__ void __launch_bounds__(kHB) static_partial_kernel(const dbl4* __restrict__ hills, long long H,
                                                             const double* __restrict__ xi, int P, Prm prm,
                                                             dbl4* __restrict__ scratch)
{
    constexpr int TP = kHB / TH;
    const int hl = threadIdx.x % TH;
    const int p = blockIdx.x * TP + threadIdx.x / TH;
    const int nsplit = gridDim.y;
    double x[3] = {0.0, 0.0, 0.0};
    if (p < P)
        for (int i = 0; i < prm.d; ++i) x[i] = xi[(size_t)p * prm.d + i];
    const long long per = (H + nsplit - 1) / nsplit;
    const long long h0 = (long long)blockIdx.y * per;
    const long long h1 = h0 + per < H ? h0 + per : H;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long k = h0 + hl; k < h1; k += TH) {
        const dbl4 h = hills[k];
        const double s[3] = {h.x, h.y, h.z};
        double dd[3] = {0.0, 0.0, 0.0}, q = 0.0;
        for (int i = 0; i < prm.d; ++i) {
            double di = x[i] - s[i];
            if (prm.per[i] > 0.0) di -= prm.per[i] * rint(di / prm.per[i]);
            dd[i] = di;
            q += di * di * prm.inv2s2[i];
        }
        const double e = h.w * exp(-q);
        acc[0] += e;
        for (int i = 0; i < prm.d; ++i) acc[1 + i] += e * dd[i];
    }
    reduce_th<TH>(acc);
    // every (split, point) entry is written, including empty hill ranges
    if (p < P && hl == 0) scratch[(size_t)blockIdx.y * P + p] = dbl4{acc[0], acc[1], acc[2], acc[3]};
}

__global__ void static_finalize_kernel(const dbl4* __restrict__ scratch, int nsplit, int P, Prm prm,
                                       double* __restrict__ V, double* __restrict__ dV)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = 0; s < nsplit; ++s) {
        const dbl4 q = scratch[(size_t)s * P + p];
        a[0] += q.x;
        a[1] += q.y;
        a[2] += q.z;
        a[3] += q.w;
    }
    V[p] = a[0];
    for (int i = 0; i < prm.d; ++i) dV[(size_t)p * prm.d + i] = prm.gs[i] * a[1 + i];
}

}  // namespace

extern "C" int wtmd_hills_eval_static(int32_t n_cv, const double* sigma, const double* period, const double* hills,
                                      int64_t n_hills, const double* xi, int64_t P, double* V_out, double* dV_out,
                                      void* stream)
{
    if (n_cv < 1 || n_cv > 3 || !sigma || n_hills < 0 || P < 0) return WTMD_EINVAL;
    if (P > WTMD_STATIC_MAX_POINTS) return WTMD_EINVAL;  // more points than the fixed scratch holds
    if (P == 0) return WTMD_OK;
    if (!xi || !V_out || !dV_out || (n_hills > 0 && !hills)) return WTMD_EINVAL;
    if ((uintptr_t)hills % 32) return WTMD_EINVAL;  // hill records are read as 32-byte vectors
    Prm prm{};
    prm.d = n_cv;
    for (int i = 0; i < 3; ++i) {
        const double sg = i < n_cv ? sigma[i] : 1.0;
        if (!(sg > 0.0) || !isfinite(sg)) return WTMD_EINVAL;
        const double pr = (i < n_cv && period) ? period[i] : 0.0;
        if (!(pr >= 0.0) || !isfinite(pr)) return WTMD_EINVAL;
        prm.inv2s2[i] = 1.0 / (2.0 * sg * sg);
        prm.per[i] = pr;
        prm.gs[i] = -1.0 / (sg * sg);
    }
    dbl4* scratch = nullptr;
    int rc = scratch_for_current_context(&scratch);
    if (rc) return rc;

    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return WTMD_ECUDA;
    const int th = P >= 1024 ? 1 : (P >= 64 ? 4 : (P >= 8 ? 32 : 256));
    const long long tp = kHB / th;
    const long long tiles = (P + tp - 1) / tp;
    long long split = (4ll * sms + tiles - 1) / tiles;
    split = std::min<long long>(split, kScratchEntries / P);  // partials must fit the fixed scratch
    split = std::min<long long>(split, std::max<int64_t>(n_hills, 1));
    split = std::max<long long>(split, 1);
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid((unsigned)tiles, (unsigned)split), block(kHB);
    const int Pi = (int)P;
    const dbl4* hl = (const dbl4*)hills;
    const long long H = n_hills;
    // each launch's own status (the caller's earlier errors are neither
    // reported here nor cleared)
    cudaError_t e;
    switch (th) {
    case 1: e = launch(static_partial_kernel<1>, grid, block, st, hl, H, xi, Pi, prm, scratch); break;
    case 4: e = launch(static_partial_kernel<4>, grid, block, st, hl, H, xi, Pi, prm, scratch); break;
    case 32: e = launch(static_partial_kernel<32>, grid, block, st, hl, H, xi, Pi, prm, scratch); break;
    default: e = launch(static_partial_kernel<256>, grid, block, st, hl, H, xi, Pi, prm, scratch); break;
    }
    if (e != cudaSuccess) return WTMD_ECUDA;
    e = launch(static_finalize_kernel, dim3((unsigned)((Pi + 255) / 256)), dim3(256), st, (const dbl4*)scratch,
               (int)split, Pi, prm, V_out, dV_out);
    return e == cudaSuccess ? WTMD_OK : WTMD_ECUDA;
}
