// Device-side pieces of the hills sum shared by hills.cu (the standalone
// kernels) and walkers.cu (the persistent multi-walker step): constants,
// parameters, compensated reductions and the FP32 (point tile, hill split)
// task.  See hills.cu for the design.
#pragma once

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
    double gs[3];   // dV/dxi_i = gs_i * (sum of the i-th gradient term)
    float gsf[3];   // gs rounded to FP32 (emit_cf)
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
    // FP32 throughout: a compensated pair rounds to the nearest float by one
    // addition, and a dependent FP64 operation costs ~64 cycles on this GPU
    // (a division or square root ~700), far more than this sum's FP32 work
    const float v = a.v[0].hi + a.v[0].lo;
    const float g[3] = {o.gsf[0] * (a.v[1].hi + a.v[1].lo), o.gsf[1] * (a.v[2].hi + a.v[2].lo),
                        o.gsf[2] * (a.v[3].hi + a.v[3].lo)};
    if (!isfinite(v) || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2])) atomicOr(o.status, ST_NUMERIC);
    if (o.V) o.V[p] = v;
    if (o.dV)
        for (int i = 0; i < o.D; ++i) o.dV[(size_t)p * o.dvs + i] = g[i];
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
__device__ inline void finalize_if_last_cf(const dbl4* partial, int P, const HillOut<float>& o)
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


__device__ __forceinline__ float2 wrap2(float2 d, float per, float iper)
{
    float2 k = __fmul2_rn(d, make_float2(iper, iper));
    k.x = rintf(k.x);
    k.y = rintf(k.y);
    return __ffma2_rn(make_float2(-per, -per), k, d);
}

// One (point tile, hill split) task of the FP32 hills sum; writes the
// compensated partial sums of the tile's points for this split.  `fresh`:
// the mbarriers are new (false: they served an earlier task of this CTA and
// are invalidated and re-initialized first).  Returns false on a timeout.
template <int D, int TH, bool PER, typename PT>
__device__ bool hills_f32_task(const float4* __restrict__ hp, const long long* __restrict__ k0p,
                               const long long* __restrict__ cnt, const PT* __restrict__ xi, int xs, int P,
                               const double* __restrict__ ctr, const HillPrmF32& prm, dbl4* __restrict__ partial,
                               unsigned* status, int tile, int split, int nsplit, float4 (*ring)[2 * CHUNK],
                               uint64_t* bar, bool fresh)
{
    constexpr int TP = HB / TH;  // points per CTA
    const int tid = threadIdx.x;
    const int hl = tid % TH;
    const int p = tile * TP + tid / TH;

    // hills [k0, count) as pair records (k0 even); the split's pairs
    // [q0, q1) are balanced to within one pair over the splits, and go
    // through the ring in chunks of up to CHUNK pairs (any pair starts on a
    // 32-byte boundary, so a chunk may start anywhere)
    const long long k0 = k0p ? *k0p : 0;
    const long long count = *cnt;
    const long long npairs = count > k0 ? ((count + 1) >> 1) - (k0 >> 1) : 0;
    hp += (size_t)(k0 >> 1) * 2;
    const long long q0 = npairs * split / nsplit;
    const long long nq = npairs * (split + 1) / nsplit - q0;
    const int nmine = (int)((nq + CHUNK - 1) / CHUNK);
    auto chunk_pairs = [&](int k) { return (int)(nq - (long long)k * CHUNK < CHUNK ? nq - (long long)k * CHUNK : CHUNK); };

    __syncthreads();  // a previous task of this CTA is done with the ring
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            if (!fresh) mbar_inval(&bar[s]);
            mbar_init(&bar[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < NST && s < nmine; ++s) {
            mbar_arrive_expect_tx(&bar[s], (uint32_t)chunk_pairs(s) * 32u);
            bulk_g2s(ring[s], hp + (size_t)(q0 + (long long)s * CHUNK) * 2, (uint32_t)chunk_pairs(s) * 32u, &bar[s]);
        }
    }
    // The hill records and counts were written before the preceding kernel
    // started; the points may come from it (its CVs).  Under a programmatic
    // dependent launch the first copies above overlap that kernel's tail.
    pdl_wait();
    pdl_trigger();  // a kernel launched after this one may start its loads

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

    // chunk sums are folded into compensated FP32 accumulators (hi + lo,
    // Knuth's TwoSum): ~48-bit sums without FP64 instructions, which are slow
    // on this part
    CF4 acc{};
    auto fold = [&](int i, float x) { acc.v[i] = cf_add(acc.v[i], x); };
    int c = 0;
    for (; c < nmine; ++c) {
        const int s = c % NST;
        const uint32_t parity = (uint32_t)(c / NST) & 1u;
        const bool ok = mbar_wait_bounded(&bar[s], parity, status);
        if (!__syncthreads_and(ok)) break;
        const float4* sh = ring[s];
        const int ncp = chunk_pairs(c);
        float2 v = make_float2(0.f, 0.f), g0 = v, g1 = v, g2 = v;
#pragma unroll 4
        for (int q = hl; q < ncp; q += TH) {
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
            const int n = chunk_pairs(c + NST);
            mbar_arrive_expect_tx(&bar[s], (uint32_t)n * 32u);
            bulk_g2s(ring[s], hp + (size_t)(q0 + (long long)(c + NST) * CHUNK) * 2, (uint32_t)n * 32u, &bar[s]);
        }
    }
    if (c < nmine) {
        // timed out (recorded in the status word): let the copies already
        // issued land before the ring is reused or the CTA exits
        if (tid == 0)
            for (int k = c; k < nmine && k < c + NST; ++k)
                mbar_wait_bounded(&bar[k % NST], (uint32_t)(k / NST) & 1u, status);
        __syncthreads();
        return false;
    }
    reduce_lanes_cf<TH>(acc);
    if (p < P && hl == 0) store_cf4(partial + (size_t)split * P + p, acc);
    return true;
}




}  // namespace wtmd
