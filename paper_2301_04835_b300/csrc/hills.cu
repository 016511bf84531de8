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
// Few points (P <= 8, e.g. the CVs of one walker in a step) would leave the
// copy ring's pipeline mostly filling and draining, so a second FP32 kernel
// takes whole hill pairs straight from global memory, all P points per
// thread, with the same arithmetic and the same fixed-order reductions; the
// plan autotuner times both kinds.
// FP64 path: the same sum in double with exp(), for parity at 1e-12.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hills_dev.cuh"

namespace wtmd {
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

// Fixed-order sum of the S split partials of the FP32 kernel, FIN_P points
// per CTA (more CTAs than one per 32 points: at a few hundred points the
// partials are several MB, and the read needs more SMs than P / 32): lane l
// of warp w takes point FIN_P b + l % FIN_P and splits g, g + 128, ...
// with g = 4 w + l / FIN_P (each split's FIN_P records are one 256-byte
// read); the four groups of a warp meet by a fixed xor tree, and one thread
// per point adds the 32 warp sums in warp order.
constexpr int FIN_W = 32;  // warps per finalize CTA
constexpr int FIN_P = 8;   // points per finalize CTA
__global__ void __launch_bounds__(FIN_W * 32) hills_finalize_cf_kernel(const dbl4* __restrict__ partial, int S, int P,
                                                                      HillOut<float> o)
{
    __shared__ CF4 red[FIN_W][FIN_P];
    // a programmatic dependent of the split kernel (its launch overlaps that
    // kernel's run): the partials are read after the wait
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int p = blockIdx.x * FIN_P + lane % FIN_P;
    constexpr int G = FIN_W * 32 / FIN_P;  // split groups
    CF4 a{};
    if (p < P) {
#pragma unroll 4
        for (int s = 4 * w + lane / FIN_P; s < S; s += G) cf4_add(a, load_cf4(partial + (size_t)s * P + p));
    }
#pragma unroll
    for (int off = FIN_P; off < 32; off <<= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) a.v[i] = cf_add(a.v[i], cf_shfl_xor(a.v[i], off));
    if (lane < FIN_P) red[w][lane] = a;
    __syncthreads();
    if (w == 0 && lane < FIN_P && p < P) {
        CF4 t = red[0][lane];
        for (int k = 1; k < FIN_W; ++k) cf4_add(t, red[k][lane]);
        emit_cf(p, t, o);
    }
}

template <int D, int TH, bool PER, typename PT>
__global__ void __launch_bounds__(HB) hills_f32_kernel(const float4* __restrict__ hp, const long long* __restrict__ k0p,
                                                       const long long* __restrict__ cnt,
                                                       const PT* __restrict__ xi, int xs, int P,
                                                       const double* __restrict__ ctr, HillPrmF32 prm,
                                                       dbl4* __restrict__ partial, HillOut<float> out)
{
    __shared__ __align__(128) float4 ring[NST][2 * CHUNK];
    __shared__ __align__(8) uint64_t bar[NST];
    // on a timeout the CTA still takes part in the ticket so that the next
    // launch starts from a clean ticket (the status word reports the error)
    hills_f32_task<D, TH, PER, PT>(hp, k0p, cnt, xi, xs, P, ctr, prm, partial, out.status, blockIdx.x, blockIdx.y,
                                   gridDim.y, ring, bar, true);
    finalize_if_last_cf(partial, P, out);
}

// Few points (P <= SMALL_P, e.g. one walker's CVs in a step): the hill range
// is split over the CTAs and every thread takes hill pairs q = tid, tid + HB,
// ... of its CTA's range straight from global memory (32-byte records,
// coalesced across the warp), its first pairs loaded before the dependency
// wait since the hills do not depend on the preceding kernel.  Each pair is
// evaluated against every point with the same packed arithmetic as the
// copy-ring kernel; per-thread sums are folded into compensated FP32 and
// reduced over the CTA in a fixed order, and the splits by the last CTA.
// No copy ring and no mbarrier: the latency of one load round trip, not of
// a pipeline's fill.
constexpr int SMALL_P = 8;

// Packed evaluation of SB hill pairs (A, B records) against NP points X
// (pre-scaled, duplicated into both halves), added to the per-point sums.
template <int D, bool PER, int NP, int SB>
__device__ __forceinline__ void pairs_eval(const float4 (&A)[SB], const float4 (&B)[SB], const float2 (&X)[NP][3],
                                           int P, const HillPrmF32& prm, float2 (&v)[NP], float2 (&g0)[NP],
                                           float2 (&g1)[NP], float2 (&g2)[NP])
{
#pragma unroll
    for (int j = 0; j < SB; ++j) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (p >= P) break;
            float2 d0 = __fadd2_rn(X[p][0], make_float2(A[j].x, A[j].y));
            if constexpr (PER) d0 = wrap2(d0, prm.per[0], prm.iper[0]);
            float2 t = __ffma2_rn(d0, d0, make_float2(B[j].z, B[j].w));
            float2 d1, d2;
            if constexpr (D >= 2) {
                d1 = __fadd2_rn(X[p][1], make_float2(A[j].z, A[j].w));
                if constexpr (PER) d1 = wrap2(d1, prm.per[1], prm.iper[1]);
                t = __ffma2_rn(d1, d1, t);
            }
            if constexpr (D >= 3) {
                d2 = __fadd2_rn(X[p][2], make_float2(B[j].x, B[j].y));
                if constexpr (PER) d2 = wrap2(d2, prm.per[2], prm.iper[2]);
                t = __ffma2_rn(d2, d2, t);
            }
            const float2 e = make_float2(ex2_approx(-t.x), ex2_approx(-t.y));
            v[p] = __fadd2_rn(v[p], e);
            g0[p] = __ffma2_rn(e, d0, g0[p]);
            if constexpr (D >= 2) g1[p] = __ffma2_rn(e, d1, g1[p]);
            if constexpr (D >= 3) g2[p] = __ffma2_rn(e, d2, g2[p]);
        }
    }
}

// The points of a few-points launch, scaled and duplicated for the packed
// arithmetic: X_pi = (xi_pi - c_i) a_i.
template <int D, int NP, typename PT>
__device__ __forceinline__ void points_scaled(const PT* __restrict__ xi, int xs, int P, const double* __restrict__ ctr,
                                              const HillPrmF32& prm, float2 (&X)[NP][3])
{
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float v = 0.f;
            if (p < P && i < D) v = (float)(((double)xi[(size_t)p * xs + i] - ctr[i]) * prm.a[i]);
            X[p][i] = make_float2(v, v);
        }
}

// The hill pairs [q0, q1) of a CTA's split, thread tid of T taking pairs
// q0 + tid + k T, in batches of SB (each batch's loads issued before any is
// used; the first batch before the dependency wait).
template <int SB> struct PairBatch {
    float4 A[SB], B[SB];
    __device__ __forceinline__ void load(const float4* __restrict__ hp, long long qb, long long q1, int T)
    {
#pragma unroll
        for (int j = 0; j < SB; ++j) {
            const long long q = qb + (long long)j * T;
            if (q < q1) {
                A[j] = __ldg(hp + 2 * q);
                B[j] = __ldg(hp + 2 * q + 1);
            } else {  // no hill: zero weight (height 2^-inf)
                A[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                B[j] = make_float4(0.f, 0.f, INFINITY, INFINITY);
            }
        }
    }
};

template <int D, bool PER, int NP, typename PT>
__global__ void __launch_bounds__(HB) hills_f32_small_kernel(const float4* __restrict__ hp,
                                                             const long long* __restrict__ k0p,
                                                             const long long* __restrict__ cnt,
                                                             const PT* __restrict__ xi, int xs, int P,
                                                             const double* __restrict__ ctr, HillPrmF32 prm,
                                                             dbl4* __restrict__ partial, HillOut<float> out)
{
    const int tid = threadIdx.x;
    const long long k0 = k0p ? *k0p : 0;
    const long long count = *cnt;
    const long long npairs = count > k0 ? ((count + 1) >> 1) - (k0 >> 1) : 0;
    hp += (size_t)(k0 >> 1) * 2;
    const long long per = (npairs + gridDim.y - 1) / gridDim.y;
    const long long q0 = (long long)blockIdx.y * per;
    const long long q1 = q0 + per < npairs ? q0 + per : npairs;
    constexpr int SB = 4;
    PairBatch<SB> pb;
    const long long qa = q0 + tid;
    pb.load(hp, qa, q1, HB);
    pdl_wait();
    pdl_trigger();
    float2 X[NP][3];
    points_scaled<D, NP, PT>(xi, xs, P, ctr, prm, X);
    float2 v[NP], g0[NP], g1[NP], g2[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) v[p] = g0[p] = g1[p] = g2[p] = make_float2(0.f, 0.f);
    for (long long qb = qa; qb < q1; qb += (long long)SB * HB) {
        if (qb != qa) pb.load(hp, qb, q1, HB);
        pairs_eval<D, PER, NP, SB>(pb.A, pb.B, X, P, prm, v, g0, g1, g2);
    }
    __shared__ CF4 red[HB / 32];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (p >= P) break;
        CF4 a{};
        a.v[0] = cf_add(cf_add(a.v[0], v[p].x), v[p].y);
        a.v[1] = cf_add(cf_add(a.v[1], g0[p].x), g0[p].y);
        a.v[2] = cf_add(cf_add(a.v[2], g1[p].x), g1[p].y);
        a.v[3] = cf_add(cf_add(a.v[3], g2[p].x), g2[p].y);
        cf4_lane_sum<32>(a);
        __syncthreads();  // red[] free from the previous point
        if (tid % 32 == 0) red[tid / 32] = a;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < HB / 32; ++w) cf4_add(a, red[w]);
            store_cf4(partial + (size_t)blockIdx.y * P + p, a);
        }
    }
    finalize_if_last_cf(partial, P, out);
}

// Few points on one thread-block cluster: the CL CTAs of the cluster split
// the hill range, and each copies its share of the pair records into shared
// memory with one bulk (TMA) copy issued before the dependency wait, so the
// records are on chip when the points are known.  The split sums meet in
// rank 0's shared memory: each rank pushes its compensated sums there with
// asynchronous stores counted on a barrier of rank 0 and leaves; rank 0 adds
// them by a fixed xor tree over 16 lanes (lane r holds rank r) and writes V
// and dV.  One cluster barrier, arrived at on entry and passed before the
// first push (rank 0's barrier is initialised by then); no global partials,
// fences or tickets; deterministic.  For short hill lists (a walker's point in a step), where
// the reduction, not the streaming, is the cost.  Records beyond the shared
// share (lists longer than the capacity the launch was sized for) are read
// from global memory.
// Threads per CTA of the cluster kernel and pairs a thread takes per
// batch (its shared-memory loads issued together): for one or two points a
// CTA's share is a few thousand pairs, and 16 warps with four independent
// pairs in flight each hide the shared-memory and MUFU latencies that 8
// warps with one pair left exposed; more points keep 8 warps and one pair
// (their per-point registers).
__host__ __device__ constexpr int cluster_threads(int NP) { return NP <= 2 ? 512 : 256; }
__host__ __device__ constexpr int cluster_batch(int NP) { return NP <= 2 ? 4 : 1; }

// Rank 0's last step (warp 1): lane r takes rank r's sums and a fixed xor
// tree over 16 lanes adds them (lanes >= CL hold 0; four dependent levels
// instead of a chain over the ranks); lane 0 writes V and dV.  Not inlined:
// the kernel also runs it once on zeros with no outputs before its
// dependency wait, so that these instructions are in the SM's instruction
// cache when the real sums arrive (run cold, the tree and the writes took
// ~1-2 us, nearly all of it instruction fetch).
template <int NP>
__device__ __noinline__ void cluster_tail(const CF4 (*rsum)[NP], int Pn, unsigned CL, unsigned r, HillOut<float> out)
{
    for (int p = 0; p < Pn; ++p) {
        CF4 mine{};
        if (r < CL) mine = rsum[r][p];
        cf4_lane_sum<16>(mine);
        if (r == 0) emit_cf(p, mine, out);
    }
}

template <int D, bool PER, int NP, typename PT>
__global__ void __launch_bounds__(cluster_threads(NP)) hills_f32_cluster_kernel(const float4* __restrict__ hp,
                                                                const long long* __restrict__ k0p,
                                                                const long long* __restrict__ cnt,
                                                                const PT* __restrict__ xi, int xs, int P,
                                                                const double* __restrict__ ctr, HillPrmF32 prm,
                                                                HillOut<float> out, int smem_pairs)
{
    extern __shared__ __align__(128) float4 crec[];  // [smem_pairs][2]
    __shared__ __align__(8) uint64_t cbar, rbar;
    __shared__ __align__(16) CF4 rsum[16][NP];  // rank 0: rank r's sums, pushed by rank r
    __shared__ __align__(16) float4 dryrec[10];  // five zero pair records for the dry pass
    const int tid = threadIdx.x;
    const long long k0 = k0p ? *k0p : 0;
    const long long count = *cnt;
    const long long npairs = count > k0 ? ((count + 1) >> 1) - (k0 >> 1) : 0;
    hp += (size_t)(k0 >> 1) * 2;
    const unsigned rank = cluster_ctarank(), CL = cluster_nctarank();
    const int Pn = P < NP ? P : NP;
    const long long per = (npairs + CL - 1) / CL;
    const long long q0 = (long long)rank * per;
    const long long nq = q0 < npairs ? (per < npairs - q0 ? per : npairs - q0) : 0;
    const int npf = (int)(nq < smem_pairs ? nq : smem_pairs);
    if (tid == 0) {
        mbar_init(&cbar, 1);
        mbar_init(&rbar, 1);
        fence_mbar_init();
        // rank 0 expects 32 bytes per point from every other rank
        if (rank == 0) mbar_arrive_expect_tx(&rbar, (CL - 1) * (unsigned)Pn * 32u);
        if (npf > 0) {
            mbar_arrive_expect_tx(&cbar, (uint32_t)npf * 32u);
            bulk_g2s(crec, hp + 2 * q0, (uint32_t)npf * 32u, &cbar);
        }
    }
    if (tid < 10) dryrec[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();  // the barriers are initialised before anyone waits on them
    cluster_arrive_relaxed();
    if (rank == 0 && tid >= 32 && tid < 64) {
        // the tail once on zeros (no ranks read, no outputs): instruction
        // cache warm-up while the CV launch runs
        HillOut<float> none = out;
        none.V = nullptr;
        none.dV = nullptr;
        cluster_tail<NP>(rsum, 1, 0u, (unsigned)(tid - 32), none);
    }
    constexpr int T = cluster_threads(NP), SB = cluster_batch(NP), NW = T / 32;
    __shared__ CF4 red[NW];
    // Two passes over one copy of the code: a dry pass before the dependency
    // wait (zero points, five zero pair records taken by every thread, sums
    // reduced but not pushed) brings the instructions into the SM's caches
    // while the CV launch runs; the real pass follows the wait.
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const bool dry = pass == 0;
        float2 X[NP][3];
#pragma unroll
        for (int p = 0; p < NP; ++p) X[p][0] = X[p][1] = X[p][2] = make_float2(0.f, 0.f);
        if (!dry) {
            pdl_wait();
            pdl_trigger();
            cluster_wait();  // every rank's barriers are initialised (long since, by now)
            points_scaled<D, NP, PT>(xi, xs, P, ctr, prm, X);
        }
        float2 v[NP], g0[NP], g1[NP], g2[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) v[p] = g0[p] = g1[p] = g2[p] = make_float2(0.f, 0.f);
        const float4* src = dry ? dryrec : crec;
        const long long nqp = dry ? 5 : nq;
        const long long npfp = dry ? 5 : npf;
        const int st = dry ? 1 : T;
        const bool landed = dry || npf == 0 || mbar_wait_bounded(&cbar, 0, out.status);
        if (landed) {
            long long k = dry ? 0 : tid;
            for (; k + (SB - 1) * st < npfp; k += SB * st) {
                float4 A[SB], B[SB];
#pragma unroll
                for (int j = 0; j < SB; ++j) {
                    A[j] = src[2 * (k + j * st)];
                    B[j] = src[2 * (k + j * st) + 1];
                }
                pairs_eval<D, PER, NP, SB>(A, B, X, P, prm, v, g0, g1, g2);
            }
            for (; k < nqp; k += st) {  // the rest of the shared share, then records beyond it
                float4 A[1], B[1];
                if (k < npfp) {
                    A[0] = src[2 * k];
                    B[0] = src[2 * k + 1];
                } else {
                    A[0] = __ldg(hp + 2 * (q0 + k));
                    B[0] = __ldg(hp + 2 * (q0 + k) + 1);
                }
                pairs_eval<D, PER, NP, 1>(A, B, X, P, prm, v, g0, g1, g2);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (p >= Pn) break;
            CF4 a{};
            a.v[0] = cf_add(cf_add(a.v[0], v[p].x), v[p].y);
            a.v[1] = cf_add(cf_add(a.v[1], g0[p].x), g0[p].y);
            a.v[2] = cf_add(cf_add(a.v[2], g1[p].x), g1[p].y);
            a.v[3] = cf_add(cf_add(a.v[3], g2[p].x), g2[p].y);
            cf4_lane_sum<32>(a);
            __syncthreads();  // red[] free from the previous point (or pass)
            if (tid % 32 == 0) red[tid / 32] = a;
            __syncthreads();
            // the warps' sums by a fixed xor tree on warp 1 (warp 0, which
            // issued the bulk copy, is kept out of the tail; lane w holds warp
            // w), pushed to rank 0 by its lane 0 (every rank pushes every
            // point, whatever its copy did, so rank 0's count completes);
            // rank 0 keeps its own
            if (tid >= 32 && tid < 64) {
                CF4 t{};
                if (tid - 32 < NW) t = red[tid - 32];
                cf4_lane_sum<NW>(t);
                if (tid != 32 || dry) continue;
                if (rank == 0) {
                    rsum[0][p] = t;
                } else {
                    float4* q = reinterpret_cast<float4*>(&rsum[rank][p]);
                    st_async_f4(q, 0, make_float4(t.v[0].hi, t.v[0].lo, t.v[1].hi, t.v[1].lo), &rbar);
                    st_async_f4(q + 1, 0, make_float4(t.v[2].hi, t.v[2].lo, t.v[3].hi, t.v[3].lo), &rbar);
                }
            }
        }
    }
    if (tid == 0) mbar_inval(&cbar);
    if (rank != 0 || tid < 32 || tid >= 64) return;
    // rank 0, warp 1: wait for the other ranks' pushes (longer than any
    // rank's own bounded copy wait, after which that rank still pushes;
    // rank 0's own sums were written by lane 0 of this warp), then lane r
    // takes rank r's sums and a fixed xor tree over 16 lanes adds them (lanes
    // >= CL hold 0; four dependent levels instead of a chain over the ranks)
    bool got = mbar_try_wait_cluster(&rbar, 0);
    if (!got) {
        const long long t0 = clock64();
        while (!(got = mbar_try_wait_cluster(&rbar, 0)) && clock64() - t0 <= (1ll << 33)) {
        }
        if (!got && tid == 32) atomicOr(out.status, ST_TIMEOUT);
    }
    if (!got) return;
    cluster_tail<NP>(rsum, Pn, CL, (unsigned)(tid - 32), out);
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
static bool cluster16_ok();
static int cluster_smem_pairs(long long cap_pairs, int CL);

static Plan plan_for(long long P, long long cap_pairs, bool fp32)
{
    Plan pl;
    // a walker's few points on a list whose cluster shares fit in shared
    // memory: the cluster kernel (records staged by TMA before the
    // dependency wait, sums met in distributed shared memory)
    if (fp32 && P <= SMALL_P) {
        const int cl = cluster16_ok() ? 16 : 8;
        if ((cap_pairs + cl - 1) / cl <= cluster_smem_pairs(cap_pairs, cl)) {
            pl.th = -1;
            pl.split = cl;
            return pl;
        }
    }
    if (P >= 1024) pl.th = 1;
    else if (P >= 64) pl.th = 4;
    else if (P > SMALL_P) pl.th = 32;
    else pl.th = fp32 ? 0 : 256;  // 0: the few-points kernel (FP32 handles)
    const long long tp = pl.th ? HB / pl.th : P;
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

// pdl: launch with programmatic stream serialization, so that the kernel's
// CTAs start (and issue their first hill copies) while the preceding kernel
// finishes; the task waits for that kernel before it reads the points.
template <int D, int TH, bool PER, typename PT>
static void launch_f32_k(dim3 grid, cudaStream_t st, bool pdl, const float4* hp, const long long* k0p,
                         const long long* cnt, const PT* xi, int xs, int P, const double* ctr, const HillPrmF32& prm,
                         dbl4* part, const HillOut<float>& o)
{
    if (pdl)
        launch_pdl(hills_f32_kernel<D, TH, PER, PT>, grid, dim3(HB), 0, st, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o);
    else
        hills_f32_kernel<D, TH, PER, PT><<<grid, HB, 0, st>>>(hp, k0p, cnt, xi, xs, P, ctr, prm, part, o);
}

template <int D, bool PER, int NP, typename PT>
static void launch_f32_small(dim3 grid, cudaStream_t st, bool pdl, const float4* hp, const long long* k0p,
                             const long long* cnt, const PT* xi, int xs, int P, const double* ctr,
                             const HillPrmF32& prm, dbl4* part, const HillOut<float>& o)
{
    if (pdl)
        launch_pdl(hills_f32_small_kernel<D, PER, NP, PT>, grid, dim3(HB), 0, st, hp, k0p, cnt, xi, xs, P, ctr, prm,
                   part, o);
    else
        hills_f32_small_kernel<D, PER, NP, PT><<<grid, HB, 0, st>>>(hp, k0p, cnt, xi, xs, P, ctr, prm, part, o);
}

// The cluster kernel: one cluster of CL CTAs (CL > 8 needs the
// non-portable cluster size), a programmatic dependent when pdl is set.
// Pair records a CTA of the cluster kernel keeps in shared memory: its share
// of the handle's capacity, at most 160 KB.
static int cluster_smem_pairs(long long cap_pairs, int CL)
{
    return (int)std::min<long long>((cap_pairs + CL - 1) / CL, (160 * 1024) / 32);
}

template <int D, bool PER, int NP, typename PT>
static cudaError_t launch_f32_cluster(int CL, long long cap_pairs, cudaStream_t st, bool pdl, const float4* hp,
                                      const long long* k0p, const long long* cnt, const PT* xi, int xs, int P,
                                      const double* ctr, const HillPrmF32& prm, const HillOut<float>& o)
{
    auto k = hills_f32_cluster_kernel<D, PER, NP, PT>;
    const int sp = cluster_smem_pairs(cap_pairs, CL);
    const size_t smem = (size_t)sp * 32;
    // the kernel's attributes, once per device (the first launch comes
    // before any capture: the step's force evaluation or a direct sum)
    static bool set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!set[dev]) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        set[dev] = true;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1, CL);
    cfg.blockDim = dim3(cluster_threads(NP));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[3];
    int n = 0;
    at[n].id = cudaLaunchAttributeClusterDimension;
    at[n].val.clusterDim.x = 1;
    at[n].val.clusterDim.y = CL;
    at[n].val.clusterDim.z = 1;
    ++n;
    if (pdl) {
        at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    at[n].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    at[n].val.sharedMemCarveout = 100;
    ++n;
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, k, hp, k0p, cnt, xi, xs, P, ctr, prm, o, sp);
}

template <int D, bool PER, typename PT>
static void launch_f32_d(int th, dim3 grid, cudaStream_t st, bool pdl, const float4* hp, const long long* k0p,
                         const long long* cnt, const PT* xi, int xs, int P, const double* ctr, const HillPrmF32& prm,
                         dbl4* part, const HillOut<float>& o, long long cap_pairs)
{
    if (th < 0) {  // the cluster kernel (P <= SMALL_P), one cluster of grid.y CTAs
        if (P == 1) launch_f32_cluster<D, PER, 1, PT>((int)grid.y, cap_pairs, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, o);
        else launch_f32_cluster<D, PER, SMALL_P, PT>((int)grid.y, cap_pairs, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, o);
        return;
    }
    if (th == 0) {  // the few-points kernel (P <= SMALL_P), grid (1, splits)
        if (P == 1) launch_f32_small<D, PER, 1, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o);
        else launch_f32_small<D, PER, SMALL_P, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o);
        return;
    }
    switch (th) {
    case 1: launch_f32_k<D, 1, PER, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o); break;
    case 4: launch_f32_k<D, 4, PER, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o); break;
    case 32: launch_f32_k<D, 32, PER, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o); break;
    default: launch_f32_k<D, 256, PER, PT>(grid, st, pdl, hp, k0p, cnt, xi, xs, P, ctr, prm, part, o); break;
    }
}

template <typename PT>
static void launch_f32_pt(int d, bool per, int th, dim3 grid, cudaStream_t st, bool pdl, const float4* hp,
                          const long long* k0p, const long long* cnt, const PT* x, int xs, int P, const double* ctr,
                          const HillPrmF32& prm, dbl4* part, const HillOut<float>& o, long long cap_pairs)
{
    switch (d * 2 + (per ? 1 : 0)) {
    case 2: launch_f32_d<1, false, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
    case 3: launch_f32_d<1, true, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
    case 4: launch_f32_d<2, false, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
    case 5: launch_f32_d<2, true, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
    case 6: launch_f32_d<3, false, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
    default: launch_f32_d<3, true, PT>(th, grid, st, pdl, hp, k0p, cnt, x, xs, P, ctr, prm, part, o, cap_pairs); break;
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

// Make sure the split-partials scratch is large enough for P points with the
// plan launch_hills will pick (call outside graph capture).
int launch_hills_partial_prealloc(wtmd_t* h, int64_t P)
{
    Plan pl = plan_for(P, h->cap_pairs, h->prec == WTMD_F32);
    for (auto& t : h->tuned)
        if (t.first == ((P << 2) | h->d)) pl.th = t.second.th, pl.split = t.second.split;
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
    return launch_hills_range(h, xi, xi_f64, xs, P, V, dV, dvs, nullptr, h->count, 0, false);
}

int launch_hills_range(wtmd_t* h, const void* xi, bool xi_f64, int xs, int64_t P, void* V, void* dV, int dvs,
                       const long long* k0p, const long long* k1p, long long max_hills, bool pdl)
{
    // the plan's split covers at most max_hills hills (0: the capacity)
    const long long cap_pairs = max_hills > 0 ? std::min<long long>(h->cap_pairs, (max_hills + 1) / 2) : h->cap_pairs;
    if (P <= 0) return WTMD_OK;
    if (P > (1ll << 30)) {
        h->err = "hills: too many points";
        return WTMD_EINVAL;
    }
    Plan pl = plan_for(P, cap_pairs, h->prec == WTMD_F32);
    for (auto& t : h->tuned)
        if (max_hills <= 0 && t.first == ((P << 2) | h->d)) pl.th = t.second.th, pl.split = t.second.split;
    if (pl.th <= 0 && (h->prec != WTMD_F32 || P > SMALL_P)) pl.th = 256;  // a tuned plan for another handle kind
    const int tp = pl.th > 0 ? HB / pl.th : (int)P;
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
        HillOut<float> o{(float*)V, (float*)dV, dvs, h->d, {gs[0], gs[1], gs[2]},
                         {(float)gs[0], (float)gs[1], (float)gs[2]}, fused ? h->ticket : nullptr, h->status};
        if (xi_f64)
            launch_f32_pt<double>(h->d, per, pl.th, grid, h->stream, pdl, h->hills32, k0p, k1p, (const double*)xi,
                                  xs, Pi, h->ctr, prm, part, o, cap_pairs);
        else
            launch_f32_pt<float>(h->d, per, pl.th, grid, h->stream, pdl, h->hills32, k0p, k1p, (const float*)xi, xs,
                                 Pi, h->ctr, prm, part, o, cap_pairs);
        mark(h, "hills_sum_f32");
        if (!fused) {
            WTMD_CUDA_TRY(h, launch_pdl(hills_finalize_cf_kernel, dim3((Pi + FIN_P - 1) / FIN_P), dim3(FIN_W * 32), 0,
                                        h->stream, (const dbl4*)part, pl.split, Pi, o));
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
        HillOut<double> o{(double*)V, (double*)dV, dvs, h->d, {gs[0], gs[1], gs[2]},
                          {(float)gs[0], (float)gs[1], (float)gs[2]}, fused ? h->ticket : nullptr, h->status};
        if (per)
            launch_f64_t<true>(pl.th, grid, h->stream, (const dbl4*)h->hills64, k1p, (const double*)xi, xs, Pi,
                               h->d, prm, part, o);
        else
            launch_f64_t<false>(pl.th, grid, h->stream, (const dbl4*)h->hills64, k1p, (const double*)xi, xs, Pi,
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

// Whether clusters of 16 CTAs of the cluster kernel can run on this device
// (a non-portable size).
static bool cluster16_probe()
{
    auto k = hills_f32_cluster_kernel<2, false, 1, double>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1, 16);
    cfg.blockDim = dim3(cluster_threads(1));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 16;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

static bool cluster16_ok()
{
    static int known[64] = {0};  // 0 unknown, 1 yes, 2 no, per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (!known[dev]) known[dev] = cluster16_probe() ? 1 : 2;
    return known[dev] == 1;
}

// A plan set by the caller (wtmd_hills_plan), checked like the tuner's
// candidates.
int hills_set_plan(wtmd_t* h, int64_t P, int lanes, int splits)
{
    const bool few = h->prec == WTMD_F32 && P >= 1 && P <= SMALL_P;
    bool ok = P >= 1 && P <= (1 << 24) && splits >= 1 && splits <= 65535;
    if (lanes == 0) ok = ok && few;
    else if (lanes == -1) ok = ok && few && (splits == 8 || (splits == 16 && cluster16_ok()));
    else ok = ok && (lanes == 1 || lanes == 4 || lanes == 32 || lanes == 256);
    if (!ok) {
        h->err = "hills plan: lanes must be 1, 4, 32, 256, 0 or -1 (FP32, P <= 8; -1 with splits 8 or 16)";
        return WTMD_EINVAL;
    }
    const long long key = (P << 2) | h->d;
    h->tuned.erase(std::remove_if(h->tuned.begin(), h->tuned.end(), [&](const std::pair<long long, Tuned>& t) {
                       return t.first == key;
                   }),
                   h->tuned.end());
    h->tuned.push_back({key, Tuned{lanes, splits}});
    return WTMD_OK;
}

// Plan autotuner for P points: times every (hill lanes per point, hill
// splits) candidate on the handle's current hill list and keeps the fastest
// for later launches with P points (step path, bias_eval, hills_eval).
int hills_tune(wtmd_t* h, int64_t P, int* th_out, int* split_out, double* ms_out)
{
    if (P < 1 || P > (1 << 24)) {
        h->err = "hills_tune: P out of range";
        return WTMD_EINVAL;
    }
    const int d = h->d;
    const size_t rs = h->prec == WTMD_F32 ? sizeof(float) : sizeof(double);
    double c[3] = {0.0, 0.0, 0.0};
    WTMD_CUDA_TRY(h, cudaMemcpy(c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost));
    std::vector<char> host((size_t)P * d * rs);
    for (int64_t p = 0; p < P; ++p)
        for (int i = 0; i < d; ++i) {
            const double v = std::isnan(c[i]) ? 0.0 : c[i];
            if (h->prec == WTMD_F32) reinterpret_cast<float*>(host.data())[p * d + i] = (float)v;
            else reinterpret_cast<double*>(host.data())[p * d + i] = v;
        }
    void *xi = nullptr, *V = nullptr, *dV = nullptr;
    WTMD_CUDA_TRY(h, cudaMalloc(&xi, host.size()));
    WTMD_CUDA_TRY(h, cudaMalloc(&V, (size_t)P * rs));
    WTMD_CUDA_TRY(h, cudaMalloc(&dV, (size_t)P * d * rs));
    WTMD_CUDA_TRY(h, cudaMemcpy(xi, host.data(), host.size(), cudaMemcpyHostToDevice));
    const long long key = (P << 2) | d;
    h->tuned.erase(std::remove_if(h->tuned.begin(), h->tuned.end(), [&](const std::pair<long long, Tuned>& t) {
                       return t.first == key;
                   }),
                   h->tuned.end());
    const long long nch = (h->cap_pairs + CHUNK - 1) / CHUNK;
    // 0: the few-points kernel, -1: the cluster kernel (split = cluster
    // size), candidates for FP32 handles with P <= SMALL_P
    const int ths[] = {-1, 0, 1, 4, 32, 256};
    const int splits[] = {1, 2, 4, 8, 16, 32, 64, 96, 128, 148, 192, 296, 444, 592, 888, 1184};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    const Plan p0 = plan_for(P, h->cap_pairs, h->prec == WTMD_F32);
    Tuned bt = {p0.th, p0.split};
    int rc = WTMD_OK;
    for (int th : ths) {
        if (th <= 0 && (h->prec != WTMD_F32 || P > SMALL_P)) continue;
        const long long tiles = th > 0 ? (P + HB / th - 1) / (HB / th) : 1;
        for (int sp : splits) {
            if (sp > nch || tiles * sp > (1ll << 20) || (size_t)sp * P * sizeof(dbl4) > (256ull << 20)) continue;
            if (th < 0 && !(sp == 8 || (sp == 16 && cluster16_ok()))) continue;
            h->tuned.push_back({key, Tuned{th, sp}});
            for (int r = 0; r < 2 && rc == WTMD_OK; ++r) rc = launch_hills(h, xi, h->prec == WTMD_F64, d, P, V, dV, d);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 10 && rc == WTMD_OK; ++r) rc = launch_hills(h, xi, h->prec == WTMD_F64, d, P, V, dV, d);
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            h->tuned.pop_back();
            if (rc) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = Tuned{th, sp};
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xi);
    cudaFree(V);
    cudaFree(dV);
    if (rc) return rc;
    h->tuned.push_back({key, bt});
    if (th_out) *th_out = bt.th;
    if (split_out) *split_out = bt.split;
    if (ms_out) *ms_out = best / 10.0;
    return WTMD_OK;
}

}  // namespace wtmd
