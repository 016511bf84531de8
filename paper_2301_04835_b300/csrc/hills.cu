// Hills sum of metadynamics (PySAGES paper, Sec. 2.1.5): the bias is a sum of
// Gaussians deposited during the run,
//     V(xi) = sum_k w_k exp(-sum_i (xi_i - s_ki)^2 / (2 sigma_i^2)),
//     dV/dxi_i = -sum_k w_k exp(...) (xi_i - s_ki) / sigma_i^2,
// evaluated at P points against the H hills of the handle.
//
// FP32 path (the throughput kernel).  Per hill and point the work is d
// subtractions, d fused multiply-adds for the exponent, one MUFU ex2, one add
// for V and d fused multiply-adds for the gradient: no dense contraction, so
// no tensor cores.  To keep the instruction count at that minimum:
//   * centres are stored pre-scaled and negated, n_ki = -(s_ki - c_i) a_i with
//     a_i = sqrt(log2(e) / 2) / sigma_i, and heights as -log2(w_k), so that
//     exp(-D^2/(2 sigma^2)) w = 2^-(sum (xi^_i + n_ki)^2 - log2 w) needs no
//     extra multiply;
//   * two hills are processed per instruction with the packed f32x2 FADD2 /
//     FFMA2 of sm_100+ (hills are stored pair-interleaved: one 32-byte record
//     per pair holds both hills' coordinates side by side);
//   * hill records are staged in shared memory by the bulk-copy (TMA) engine
//     into a 4-stage ring guarded by mbarriers, so every loaded record is
//     reused by all points of the CTA;
//   * per-thread FP32 chunk sums are folded into compensated FP32 (TwoSum)
//     accumulators after every 128-pair chunk (no FP64 in the loop),
//     and the hill-range splits are reduced in a fixed order by the CTA that
//     finishes last (one launch, deterministic, no CTA waits for another).
// FP64 path: the same sum in double with exp(), for parity at 1e-12.
#include "wtmd_internal.cuh"

namespace wtmd {

constexpr int HB = 256;         // threads per CTA
constexpr int CHUNK = 128;      // hill pairs per ring stage (4 KB)
constexpr int NST = 4;          // ring stages

struct HillPrmF32 {
    double a[3];   // scale of the CVs
    float per[3];  // scaled period (0 = not periodic)
    float iper[3];
};

struct HillPrmF64 {
    double inv2s2[3];  // 1 / (2 sigma^2)
    double per[3];
};

// Sum over `TH` consecutive lanes (TH a power of two <= 32).
template <int TH> __device__ __forceinline__ double lane_sum(double v)
{
#pragma unroll
    for (int o = TH / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce the 4 accumulators over the TH hill lanes of each point; lane 0 of
// every point gets the totals.  TH <= 32: shuffles; TH > 32: shuffles then
// shared memory across the TH/32 warps of the point.
template <int TH> __device__ __forceinline__ void reduce_lanes(double acc[4])
{
    if constexpr (TH <= 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = lane_sum<TH>(acc[i]);
    } else {
        __shared__ double red[HB / 32][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = lane_sum<32>(acc[i]);
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (lane == 0)
            for (int i = 0; i < 4; ++i) red[warp][i] = acc[i];
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

// Output of a hills-sum launch: V [P], dV [P][dvs] (first D columns), the
// gradient scale gs (dV_i = gs_i * sum_k e_k D_ki in the kernel's units), a
// launch ticket and the status word.
template <typename R> struct HillOut {
    R* V;
    R* dV;
    int dvs;
    int D;
    double gs[3];
    unsigned* ticket;  // null: partials only (a separate finalize kernel reduces them)
    unsigned* status;
};

// L2 load that bypasses L1 (the partials were written by other CTAs of the
// same launch).
__device__ __forceinline__ dbl4 ldcg4(const dbl4* p)
{
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    return dbl4{a.x, a.y, b.x, b.y};
}

// Every CTA calls this after writing its partial sums.  The CTA that takes the
// last ticket sums the splits of every point in split order (the same order
// whichever CTA is last, so the result is deterministic), writes V and dV and
// resets the ticket for the next launch.  No CTA waits for another.
template <typename R>
__device__ void finalize_if_last(const dbl4* partial, int P, const HillOut<R>& o)
{
    if (!o.ticket) return;
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(o.ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int S = gridDim.y;
    auto emit = [&](int p, const double a[4]) {
        const double g[3] = {o.gs[0] * a[1], o.gs[1] * a[2], o.gs[2] * a[3]};
        if (!isfinite(a[0]) || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2])) atomicOr(o.status, ST_NUMERIC);
        if (o.V) o.V[p] = (R)a[0];
        if (o.dV)
            for (int i = 0; i < o.D; ++i) o.dV[(size_t)p * o.dvs + i] = (R)g[i];
    };
    if (P <= 8) {
        // few points: the whole CTA strides over the splits of each point
        __shared__ double red[HB / 32][4];
        const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
        for (int p = 0; p < P; ++p) {
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                const dbl4 q = ldcg4(partial + (size_t)s * P + p);
                a[0] += q.x;
                a[1] += q.y;
                a[2] += q.z;
                a[3] += q.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = lane_sum<32>(a[i]);
            if (lane == 0)
                for (int i = 0; i < 4; ++i) red[warp][i] = a[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                double t[4] = {0.0, 0.0, 0.0, 0.0};
                for (int w = 0; w < (int)(blockDim.x / 32); ++w)
                    for (int i = 0; i < 4; ++i) t[i] += red[w][i];
                emit(p, t);
            }
            __syncthreads();
        }
    } else if (S <= 8) {
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            for (int s = 0; s < S; ++s) {
                const dbl4 q = ldcg4(partial + (size_t)s * P + p);
                a[0] += q.x;
                a[1] += q.y;
                a[2] += q.z;
                a[3] += q.w;
            }
            emit(p, a);
        }
    } else {
        const int lane = threadIdx.x % 32, nw = blockDim.x / 32;
        for (int p = threadIdx.x / 32; p < P; p += nw) {
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            for (int s = lane; s < S; s += 32) {
                const dbl4 q = ldcg4(partial + (size_t)s * P + p);
                a[0] += q.x;
                a[1] += q.y;
                a[2] += q.z;
                a[3] += q.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = lane_sum<32>(a[i]);
            if (lane == 0) emit(p, a);
        }
    }
    if (threadIdx.x == 0) *o.ticket = 0u;
}

// Separate reduction of the splits when P x splits is large: one warp per
// point (lanes stride over the splits, fixed shuffle tree).
template <typename R>
__global__ void __launch_bounds__(256) hills_finalize_kernel(const dbl4* __restrict__ partial, int S, int P,
                                                             HillOut<R> o)
{
    const int lane = threadIdx.x % 32;
    const int p = blockIdx.x * 8 + threadIdx.x / 32;
    if (p >= P) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = lane; s < S; s += 32) {
        const dbl4 q = partial[(size_t)s * P + p];
        a[0] += q.x;
        a[1] += q.y;
        a[2] += q.z;
        a[3] += q.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = lane_sum<32>(a[i]);
    if (lane == 0) {
        const double g[3] = {o.gs[0] * a[1], o.gs[1] * a[2], o.gs[2] * a[3]};
        if (!isfinite(a[0]) || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2])) atomicOr(o.status, ST_NUMERIC);
        if (o.V) o.V[p] = (R)a[0];
        if (o.dV)
            for (int i = 0; i < o.D; ++i) o.dV[(size_t)p * o.dvs + i] = (R)g[i];
    }
}

// ---- compensated-FP32 reduction path of the FP32 kernel (no FP64 ops until
// the one conversion per point) ----
struct CF4 {
    cf v[4];
};

__device__ __forceinline__ void store_cf4(dbl4* slot, const CF4& a)
{
    float4* q = reinterpret_cast<float4*>(slot);
    q[0] = make_float4(a.v[0].hi, a.v[0].lo, a.v[1].hi, a.v[1].lo);
    q[1] = make_float4(a.v[2].hi, a.v[2].lo, a.v[3].hi, a.v[3].lo);
}
__device__ __forceinline__ CF4 load_cf4(const dbl4* slot)
{
    const float4* q = reinterpret_cast<const float4*>(slot);
    const float4 a = __ldcg(q), b = __ldcg(q + 1);
    return CF4{{cf{a.x, a.y}, cf{a.z, a.w}, cf{b.x, b.y}, cf{b.z, b.w}}};
}
__device__ __forceinline__ void cf4_add(CF4& a, const CF4& b)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) a.v[i] = cf_add(a.v[i], b.v[i]);
}
template <int W> __device__ __forceinline__ void cf4_lane_sum(CF4& a)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) a.v[i] = cf_add(a.v[i], cf_shfl_xor(a.v[i], o));
}

// Reduce over the TH hill lanes of each point (lane 0 of the point gets it).
template <int TH> __device__ __forceinline__ void reduce_lanes_cf(CF4& a)
{
    if constexpr (TH <= 32) {
        cf4_lane_sum<TH>(a);
    } else {
        __shared__ CF4 red[HB / 32];
        cf4_lane_sum<32>(a);
        if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = a;
        __syncthreads();
        if (threadIdx.x % TH == 0) {
            CF4 t = red[threadIdx.x / 32];
            for (int w = 1; w < TH / 32; ++w) cf4_add(t, red[threadIdx.x / 32 + w]);
            a = t;
        }
    }
}

__device__ __forceinline__ void emit_cf(int p, const CF4& a, const HillOut<float>& o)
{
    const double v = cf_val(a.v[0]);
    const double g[3] = {o.gs[0] * cf_val(a.v[1]), o.gs[1] * cf_val(a.v[2]), o.gs[2] * cf_val(a.v[3])};
    if (!isfinite(v) || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2])) atomicOr(o.status, ST_NUMERIC);
    if (o.V) o.V[p] = (float)v;
    if (o.dV)
        for (int i = 0; i < o.D; ++i) o.dV[(size_t)p * o.dvs + i] = (float)g[i];
}

// Sum of the S splits of point p by the whole CTA (fixed order: thread
// strides, xor tree, warps in order); the result is valid in thread 0.
__device__ __forceinline__ CF4 cta_split_sum(const dbl4* partial, int S, int P, int p)
{
    __shared__ CF4 red[HB / 32];
    CF4 a{};
    for (int s = threadIdx.x; s < S; s += blockDim.x) cf4_add(a, load_cf4(partial + (size_t)s * P + p));
    cf4_lane_sum<32>(a);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = a;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) cf4_add(a, red[w]);
    __syncthreads();
    return a;
}

// As finalize_if_last, for the compensated partials of the FP32 kernel.
__device__ void finalize_if_last_cf(const dbl4* partial, int P, const HillOut<float>& o)
{
    if (!o.ticket) return;
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(o.ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int S = gridDim.y;
    if (P <= 8) {
        for (int p = 0; p < P; ++p) {
            const CF4 a = cta_split_sum(partial, S, P, p);
            if (threadIdx.x == 0) emit_cf(p, a, o);
        }
    } else {
        const int lane = threadIdx.x % 32, nw = blockDim.x / 32;
        for (int p = threadIdx.x / 32; p < P; p += nw) {
            CF4 a{};
            for (int s = lane; s < S; s += 32) cf4_add(a, load_cf4(partial + (size_t)s * P + p));
            cf4_lane_sum<32>(a);
            if (lane == 0) emit_cf(p, a, o);
        }
    }
    if (threadIdx.x == 0) *o.ticket = 0u;
}

__global__ void __launch_bounds__(256) hills_finalize_cf_kernel(const dbl4* __restrict__ partial, int S, int P,
                                                                HillOut<float> o)
{
    const int lane = threadIdx.x % 32;
    const int p = blockIdx.x * 8 + threadIdx.x / 32;
    if (p >= P) return;
    CF4 a{};
    for (int s = lane; s < S; s += 32) cf4_add(a, load_cf4(partial + (size_t)s * P + p));
    cf4_lane_sum<32>(a);
    if (lane == 0) emit_cf(p, a, o);
}

__device__ __forceinline__ float2 wrap2(float2 d, float per, float iper)
{
    float2 k = __fmul2_rn(d, make_float2(iper, iper));
    k.x = rintf(k.x);
    k.y = rintf(k.y);
    return __ffma2_rn(make_float2(-per, -per), k, d);
}

template <int D, int TH, bool PER, typename PT>
__global__ void __launch_bounds__(HB) hills_f32_kernel(const float4* __restrict__ hp, const long long* __restrict__ cnt,
                                                       const PT* __restrict__ xi, int xs, int P,
                                                       const double* __restrict__ ctr, HillPrmF32 prm,
                                                       dbl4* __restrict__ partial, HillOut<float> out)
{
    constexpr int TP = HB / TH;  // points per CTA
    __shared__ __align__(128) float4 ring[NST][2 * CHUNK];
    __shared__ __align__(8) uint64_t bar[NST];

    const int tid = threadIdx.x;
    const int hl = tid % TH;
    const int p = blockIdx.x * TP + tid / TH;
    const int nsplit = gridDim.y;

    // scaled, centred point: the subtraction of the centre is done in FP64 so
    // that the FP32 coordinate keeps its relative precision near the hills
    float xh[3] = {0.f, 0.f, 0.f};
    if (p < P) {
#pragma unroll
        for (int i = 0; i < D; ++i) xh[i] = (float)(((double)xi[(size_t)p * xs + i] - ctr[i]) * prm.a[i]);
    }
    const float2 X0 = make_float2(xh[0], xh[0]);
    const float2 X1 = make_float2(xh[1], xh[1]);
    const float2 X2 = make_float2(xh[2], xh[2]);

    const long long count = *cnt;
    const long long npairs = (count + 1) >> 1;
    const long long nch = (npairs + CHUNK - 1) / CHUNK;
    const long long per = (nch + nsplit - 1) / nsplit;
    const long long c0 = (long long)blockIdx.y * per;
    const long long c1 = c0 + per < nch ? c0 + per : nch;
    const int nmine = c1 > c0 ? (int)(c1 - c0) : 0;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < NST && s < nmine; ++s) {
            mbar_arrive_expect_tx(&bar[s], CHUNK * 32);
            bulk_g2s(ring[s], hp + (size_t)(c0 + s) * CHUNK * 2, CHUNK * 32, &bar[s]);
        }
    }

    // chunk sums are folded into compensated FP32 accumulators (hi + lo,
    // Knuth's TwoSum): ~48-bit sums without FP64 instructions, which are slow
    // on this part
    CF4 acc{};
    auto fold = [&](int i, float x) { acc.v[i] = cf_add(acc.v[i], x); };
    int c = 0;
    for (; c < nmine; ++c) {
        const int s = c % NST;
        const uint32_t parity = (uint32_t)(c / NST) & 1u;
        const bool ok = mbar_wait_bounded(&bar[s], parity, out.status);
        if (!__syncthreads_and(ok)) break;
        const float4* sh = ring[s];
        float2 v = make_float2(0.f, 0.f), g0 = v, g1 = v, g2 = v;
#pragma unroll 4
        for (int q = hl; q < CHUNK; q += TH) {
            const float4 A = sh[2 * q];
            const float4 B = sh[2 * q + 1];
            float2 d0 = __fadd2_rn(X0, make_float2(A.x, A.y));
            if constexpr (PER) d0 = wrap2(d0, prm.per[0], prm.iper[0]);
            float2 t = __ffma2_rn(d0, d0, make_float2(B.z, B.w));
            float2 d1, d2;
            if constexpr (D >= 2) {
                d1 = __fadd2_rn(X1, make_float2(A.z, A.w));
                if constexpr (PER) d1 = wrap2(d1, prm.per[1], prm.iper[1]);
                t = __ffma2_rn(d1, d1, t);
            }
            if constexpr (D >= 3) {
                d2 = __fadd2_rn(X2, make_float2(B.x, B.y));
                if constexpr (PER) d2 = wrap2(d2, prm.per[2], prm.iper[2]);
                t = __ffma2_rn(d2, d2, t);
            }
            const float2 e = make_float2(ex2_approx(-t.x), ex2_approx(-t.y));
            v = __fadd2_rn(v, e);
            g0 = __ffma2_rn(e, d0, g0);
            if constexpr (D >= 2) g1 = __ffma2_rn(e, d1, g1);
            if constexpr (D >= 3) g2 = __ffma2_rn(e, d2, g2);
        }
        fold(0, v.x);
        fold(0, v.y);
        fold(1, g0.x);
        fold(1, g0.y);
        if constexpr (D >= 2) {
            fold(2, g1.x);
            fold(2, g1.y);
        }
        if constexpr (D >= 3) {
            fold(3, g2.x);
            fold(3, g2.y);
        }
        __syncthreads();  // stage s consumed by every thread
        if (tid == 0 && c + NST < nmine) {
            mbar_arrive_expect_tx(&bar[s], CHUNK * 32);
            bulk_g2s(ring[s], hp + (size_t)(c0 + c + NST) * CHUNK * 2, CHUNK * 32, &bar[s]);
        }
    }
    if (c < nmine) {
        // timed out (recorded in the status word): let the copies already
        // issued land, then take part in the ticket so the next launch starts
        // from a clean ticket
        if (tid == 0)
            for (int k = c; k < nmine && k < c + NST; ++k)
                mbar_wait_bounded(&bar[k % NST], (uint32_t)(k / NST) & 1u, out.status);
        __syncthreads();
    } else {
        reduce_lanes_cf<TH>(acc);
        if (p < P && hl == 0) store_cf4(partial + (size_t)blockIdx.y * P + p, acc);
    }
    finalize_if_last_cf(partial, P, out);
}

template <int TH, bool PER>
__global__ void __launch_bounds__(HB) hills_f64_kernel(const dbl4* __restrict__ hills, const long long* __restrict__ cnt,
                                                       const double* __restrict__ xi, int xs, int P, int D,
                                                       HillPrmF64 prm, dbl4* __restrict__ partial,
                                                       HillOut<double> out)
{
    constexpr int TP = HB / TH;
    const int tid = threadIdx.x;
    const int hl = tid % TH;
    const int p = blockIdx.x * TP + tid / TH;
    const int nsplit = gridDim.y;
    double x[3] = {0.0, 0.0, 0.0};
    if (p < P)
        for (int i = 0; i < D; ++i) x[i] = xi[(size_t)p * xs + i];
    const long long count = *cnt;
    const long long per = (count + nsplit - 1) / nsplit;
    const long long h0 = (long long)blockIdx.y * per;
    const long long h1 = h0 + per < count ? h0 + per : count;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long k = h0 + hl; k < h1; k += TH) {
        const dbl4 h = hills[k];
        const double s[3] = {h.x, h.y, h.z};
        double dd[3] = {0.0, 0.0, 0.0}, q = 0.0;
        for (int i = 0; i < D; ++i) {
            double di = x[i] - s[i];
            if (PER && prm.per[i] > 0.0) di -= prm.per[i] * rint(di / prm.per[i]);
            dd[i] = di;
            q += di * di * prm.inv2s2[i];
        }
        const double e = h.w * exp(-q);
        acc[0] += e;
        for (int i = 0; i < D; ++i) acc[1 + i] += e * dd[i];
    }
    reduce_lanes<TH>(acc);
    if (p < P && hl == 0) partial[(size_t)blockIdx.y * P + p] = dbl4{acc[0], acc[1], acc[2], acc[3]};
    finalize_if_last<double>(partial, P, out);
}

// ----------------------------------------------------------------------------
// FP32 hill layout
// ----------------------------------------------------------------------------
__global__ void store_hills32_kernel(const dbl4* __restrict__ h64, long long k0, long long k1, double a0, double a1,
                                     double a2, const double* __restrict__ ctr, float* __restrict__ out)
{
    const long long k = k0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= k1) return;
    const dbl4 h = h64[k];
    const double c0 = ctr[0], c1 = ctr[1], c2 = ctr[2];
    const long long base = (k >> 1) * 8 + (k & 1);
    out[base + 0] = (float)(-(h.x - c0) * a0);
    out[base + 2] = (float)(-(h.y - c1) * a1);
    out[base + 4] = (float)(-(h.z - c2) * a2);
    out[base + 6] = (float)(-log2(h.w));
}

void store_hills32_range(wtmd_t* h, long long k0, long long k1)
{
    if (k1 <= k0) return;
    const int nb = (int)((k1 - k0 + 255) / 256);
    store_hills32_kernel<<<nb, 256, 0, h->stream>>>((const dbl4*)h->hills64, k0, k1, h->a[0], h->a[1], h->a[2],
                                                    h->ctr, (float*)h->hills32);
}

void store_hills32(wtmd_t* h)
{
    long long n = 0;
    cudaMemcpyAsync(&n, h->count, sizeof(n), cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
    store_hills32_range(h, 0, n);
}

// ----------------------------------------------------------------------------
// launch
// ----------------------------------------------------------------------------
struct Plan {
    int th;
    int split;
};

static int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// Tile heuristic: few points -> many hill lanes per point; many points ->
// one thread per point.  Splits fill ~4 CTAs per SM over the hill range.
static Plan plan_for(long long P, long long cap_pairs)
{
    Plan pl;
    if (P >= 1024) pl.th = 1;
    else if (P >= 64) pl.th = 4;
    else if (P >= 8) pl.th = 32;
    else pl.th = 256;
    const long long tp = HB / pl.th;
    const long long tiles = (P + tp - 1) / tp;
    // few points: ~2 CTAs per SM (each CTA then streams several chunks and
    // the final reduction stays short); many points: ~4 per SM
    const long long want = (P < 64 ? 2ll : 4ll) * num_sms();
    long long split = (want + tiles - 1) / tiles;
    const long long nch = (cap_pairs + CHUNK - 1) / CHUNK;
    if (split > nch) split = nch;
    if (split < 1) split = 1;
    if (split > 65535) split = 65535;
    pl.split = (int)split;
    return pl;
}

template <int D, bool PER, typename PT>
static void launch_f32_d(int th, dim3 grid, cudaStream_t st, const float4* hp, const long long* cnt, const PT* xi,
                         int xs, int P, const double* ctr, const HillPrmF32& prm, dbl4* part, const HillOut<float>& o)
{
    switch (th) {
    case 1: hills_f32_kernel<D, 1, PER, PT><<<grid, HB, 0, st>>>(hp, cnt, xi, xs, P, ctr, prm, part, o); break;
    case 4: hills_f32_kernel<D, 4, PER, PT><<<grid, HB, 0, st>>>(hp, cnt, xi, xs, P, ctr, prm, part, o); break;
    case 32: hills_f32_kernel<D, 32, PER, PT><<<grid, HB, 0, st>>>(hp, cnt, xi, xs, P, ctr, prm, part, o); break;
    default: hills_f32_kernel<D, 256, PER, PT><<<grid, HB, 0, st>>>(hp, cnt, xi, xs, P, ctr, prm, part, o); break;
    }
}

template <typename PT>
static void launch_f32_pt(int d, bool per, int th, dim3 grid, cudaStream_t st, const float4* hp, const long long* cnt,
                          const PT* x, int xs, int P, const double* ctr, const HillPrmF32& prm, dbl4* part,
                          const HillOut<float>& status)
{
    switch (d * 2 + (per ? 1 : 0)) {
    case 2: launch_f32_d<1, false, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    case 3: launch_f32_d<1, true, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    case 4: launch_f32_d<2, false, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    case 5: launch_f32_d<2, true, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    case 6: launch_f32_d<3, false, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    default: launch_f32_d<3, true, PT>(th, grid, st, hp, cnt, x, xs, P, ctr, prm, part, status); break;
    }
}

template <bool PER>
static void launch_f64_t(int th, dim3 grid, cudaStream_t st, const dbl4* hills, const long long* cnt, const double* xi,
                         int xs, int P, int D, const HillPrmF64& prm, dbl4* part, const HillOut<double>& o)
{
    switch (th) {
    case 1: hills_f64_kernel<1, PER><<<grid, HB, 0, st>>>(hills, cnt, xi, xs, P, D, prm, part, o); break;
    case 4: hills_f64_kernel<4, PER><<<grid, HB, 0, st>>>(hills, cnt, xi, xs, P, D, prm, part, o); break;
    case 32: hills_f64_kernel<32, PER><<<grid, HB, 0, st>>>(hills, cnt, xi, xs, P, D, prm, part, o); break;
    default: hills_f64_kernel<256, PER><<<grid, HB, 0, st>>>(hills, cnt, xi, xs, P, D, prm, part, o); break;
    }
}

int hills_plan_override_th = 0;     // autotuner / benchmark hooks (0 = heuristic)
int hills_plan_override_split = 0;

// Make sure the split-partials scratch is large enough for P points with the
// plan launch_hills will pick (call outside graph capture).
int launch_hills_partial_prealloc(wtmd_t* h, int64_t P)
{
    Plan pl = plan_for(P, h->cap_pairs);
    for (auto& t : h->tuned)
        if (t.first == ((P << 2) | h->d)) pl.th = t.second.th, pl.split = t.second.split;
    if (hills_plan_override_split) pl.split = hills_plan_override_split;
    const size_t need = (size_t)pl.split * (size_t)P * sizeof(dbl4);
    if (need > h->partial_bytes) {
        cudaFree(h->partial);
        h->partial = nullptr;
        h->partial_bytes = 0;
        WTMD_CUDA_TRY(h, cudaMalloc(&h->partial, need));
        h->partial_bytes = need;
    }
    return WTMD_OK;
}

int launch_hills(wtmd_t* h, const void* xi, bool xi_f64, int xs, int64_t P, void* V, void* dV, int dvs)
{
    if (P <= 0) return WTMD_OK;
    if (P > (1ll << 30)) {
        h->err = "hills: too many points";
        return WTMD_EINVAL;
    }
    Plan pl = plan_for(P, h->cap_pairs);
    for (auto& t : h->tuned)
        if (t.first == ((P << 2) | h->d)) pl.th = t.second.th, pl.split = t.second.split;
    if (hills_plan_override_th) pl.th = hills_plan_override_th;
    if (hills_plan_override_split) pl.split = hills_plan_override_split;
    const int tp = HB / pl.th;
    const long long tiles = (P + tp - 1) / tp;
    if (tiles > 0x7fffffff) return WTMD_EINVAL;
    const size_t need = (size_t)pl.split * (size_t)P * sizeof(dbl4);
    if (need > h->partial_bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(h->stream, &cs);
        if (cs != cudaStreamCaptureStatusNone) {
            h->err = "hills: scratch too small during graph capture";
            return WTMD_EINVAL;
        }
        cudaFree(h->partial);  // implicitly synchronizes
        h->partial = nullptr;
        h->partial_bytes = 0;
        WTMD_CUDA_TRY(h, cudaMalloc(&h->partial, need));
        h->partial_bytes = need;
    }
    dim3 grid((unsigned)tiles, (unsigned)pl.split);
    // small reductions are done by the CTA that finishes last (saves a
    // launch); large ones by a separate, parallel finalize kernel
    const bool fused = (long long)pl.split * P <= 16384;
    bool per = false;
    for (int i = 0; i < h->d; ++i) per = per || h->cv[i].period > 0.0;
    double gs[3] = {0.0, 0.0, 0.0};
    if (h->prec == WTMD_F32) {
        HillPrmF32 prm{};
        for (int i = 0; i < 3; ++i) {
            prm.a[i] = h->a[i];
            const double pp = i < h->d ? h->cv[i].period * h->a[i] : 0.0;
            prm.per[i] = (float)pp;
            prm.iper[i] = pp > 0.0 ? (float)(1.0 / pp) : 0.f;
            gs[i] = -2.0 * 0.69314718055994530942 * h->a[i];
        }
        auto part = (dbl4*)h->partial;
        const int Pi = (int)P;
        HillOut<float> o{(float*)V, (float*)dV, dvs, h->d, {gs[0], gs[1], gs[2]}, fused ? h->ticket : nullptr,
                         h->status};
        if (xi_f64)
            launch_f32_pt<double>(h->d, per, pl.th, grid, h->stream, h->hills32, h->count, (const double*)xi, xs, Pi,
                                  h->ctr, prm, part, o);
        else
            launch_f32_pt<float>(h->d, per, pl.th, grid, h->stream, h->hills32, h->count, (const float*)xi, xs, Pi,
                                 h->ctr, prm, part, o);
        mark(h, "hills_sum_f32");
        if (!fused) {
            hills_finalize_cf_kernel<<<(Pi + 7) / 8, 256, 0, h->stream>>>(part, pl.split, Pi, o);
            mark(h, "hills_finalize");
        }
    } else {
        HillPrmF64 prm{};
        for (int i = 0; i < 3; ++i) {
            const double sg = h->cfg.sigma[i] > 0 ? h->cfg.sigma[i] : 1.0;
            prm.inv2s2[i] = 1.0 / (2.0 * sg * sg);
            prm.per[i] = i < h->d ? h->cv[i].period : 0.0;
            gs[i] = -1.0 / (sg * sg);
        }
        auto part = (dbl4*)h->partial;
        const int Pi = (int)P;
        HillOut<double> o{(double*)V, (double*)dV, dvs, h->d, {gs[0], gs[1], gs[2]}, fused ? h->ticket : nullptr,
                          h->status};
        if (per)
            launch_f64_t<true>(pl.th, grid, h->stream, (const dbl4*)h->hills64, h->count, (const double*)xi, xs, Pi,
                               h->d, prm, part, o);
        else
            launch_f64_t<false>(pl.th, grid, h->stream, (const dbl4*)h->hills64, h->count, (const double*)xi, xs, Pi,
                                h->d, prm, part, o);
        mark(h, "hills_sum_f64");
        if (!fused) {
            hills_finalize_kernel<double><<<(Pi + 7) / 8, 256, 0, h->stream>>>(part, pl.split, Pi, o);
            mark(h, "hills_finalize");
        }
    }
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

}  // namespace wtmd
