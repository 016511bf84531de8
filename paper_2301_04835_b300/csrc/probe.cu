// Throughput probes of the two SM pipes the FP32 hills sum runs on: the MUFU
// unit (ex2.approx) and the FP32 FMA pipe (packed FFMA2).  Each thread keeps
// 8 independent chains so latency is hidden; the grid fills every SM.  The
// measured rates, taken at the clock of the run, are the denominators of the
// hills-sum roofline next to the nominal unit-count x clock figures.
#include "wtmd_internal.cuh"

namespace wtmd {

// A cooperative grid in which CTA `absent` leaves at once: the others wait at
// the grid barrier for an arrival that never comes, give up after `limit`
// cycles and record ST_TIMEOUT (absent < 0: everyone arrives).
__global__ void barrier_probe_kernel(unsigned* bar, unsigned* status, int absent, long long limit)
{
    if ((int)blockIdx.x == absent) return;
    grid_barrier(bar, gridDim.x, status, limit);
}

__global__ void __launch_bounds__(256) probe_ex2_kernel(int iters, float seed, float* out)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = seed + 0.01f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_ffma2_kernel(int iters, float seed, float* out)
{
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = make_float2(seed + k, seed - k);
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(0.001f, 0.002f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].x + x[k].y;
    if (s == 12345.678f) out[0] = s;
}

}  // namespace wtmd

// kind 0: MUFU ex2 per second; kind 1: FP32 FMA lane-operations per second
// (packed FFMA2 counted as two).  *ms receives the kernel time.
extern "C" int wtmd_probe_peak(int32_t kind, double* ops_per_s, double* ms)
{
    using namespace wtmd;
    if (!ops_per_s || (kind != 0 && kind != 1)) return WTMD_EINVAL;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return WTMD_ENOMEM;
    const int blocks = sms * 8, threads = 256, iters = kind == 0 ? 4096 : 8192;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        if (kind == 0) probe_ex2_kernel<<<blocks, threads>>>(iters, 0.5f, out);
        else probe_ffma2_kernel<<<blocks, threads>>>(iters, 0.5f, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return WTMD_ECUDA;
    const double ops = (double)blocks * threads * iters * 8.0 * (kind == 0 ? 1.0 : 2.0);  // FFMA2 = 2 lane FMAs
    *ops_per_s = ops / (best * 1e-3);
    if (ms) *ms = best;
    return WTMD_OK;
}

extern "C" int wtmd_barrier_probe(int32_t blocks, int32_t absent, int64_t limit_cycles, int32_t* timed_out)
{
    if (blocks < 1 || absent >= blocks || limit_cycles < 1 || limit_cycles > wtmd::kWaitLimit) return WTMD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return WTMD_ECUDA;
    if (blocks > sms) return WTMD_EINVAL;  // one CTA per SM: all co-resident
    unsigned* buf = nullptr;  // [0..3] barrier, [4] status
    if (cudaMalloc(&buf, 8 * sizeof(unsigned)) != cudaSuccess) return WTMD_ENOMEM;
    int rc = WTMD_OK;
    if (cudaMemset(buf, 0, 8 * sizeof(unsigned)) != cudaSuccess) rc = WTMD_ECUDA;
    if (!rc) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(64);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        unsigned* status = buf + 4;
        if (cudaLaunchKernelEx(&cfg, wtmd::barrier_probe_kernel, buf, status, (int)absent, (long long)limit_cycles) !=
                cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            rc = WTMD_ECUDA;
        unsigned st = 0;
        if (!rc && cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) rc = WTMD_ECUDA;
        if (!rc && timed_out) *timed_out = (st & wtmd::ST_TIMEOUT) ? 1 : 0;
    }
    cudaFree(buf);
    return rc;
}
