// FP32 tile form of the switching-function coordination CV, shared by the
// standalone CV kernels (cv.cu) and the persistent single-system step
// (sys_step.cu).  The CV (not defined in the PySAGES paper, Sec. 2.2 lists
// CVs of this kind): xi = scale * sum_{i in A} sum_{j in B, j != i} s(r_ij),
// s(r) = 1 / (1 + (r/r0)^n) (the rational switch (1-x^n)/(1-x^2n)).
#pragma once

#include "wtmd_internal.cuh"

namespace wtmd {

constexpr int CT_T = 256;
constexpr int CT_B = 256;  // partners per CTA (8 warps x 32)

// ---------------------------------------------------------------------------
// FP32 form of the tile kernel.  A CTA takes 64 members of A, two per lane
// (tile members lane and lane + 32), and a chunk of CT_B partners, so that
// every arithmetic instruction of the pair loop serves two pairs through the
// packed f32x2 operations.  Partners are staged pre-negated and duplicated
// into both halves, (-x,-x,-y,-y) and (-z,-z,w,w), so a difference is one
// packed add.  The minimum image rounds d/L by the 1.5 * 2^23 shift
// (exact for |d/L| < 2^22) instead of a conversion instruction.
//
// The kernel ends with its partials: nothing waits on another CTA.  The CV
// value needs no second pass: each CTA rounds its share
// scale * (sum of s over its pairs, its self pairs removed) to a multiple of
// 2^-q and adds it to xi with a double atomic.  q is chosen on the host so
// that every partial sum of such shares is a double exactly; the additions
// are then exact and the result does not depend on their order.  J stays in
// factored form, row partials [W][chunk][A] and column partials
// [W][tile][B], contracted per atom in a fixed order by `coord_jfin_kernel`,
// which in a step runs beside the hills sum (that needs xi only).
//
// The body below is shared by the standalone kernel (cv.cu) and the
// persistent single-system step (sys_step.cu): it takes its thread index,
// a hook called between the index reads and the position reads (the
// dependency wait of a programmatic launch) and the barrier of the threads
// that run it.
// ---------------------------------------------------------------------------
constexpr int C2_A = 64;   // targets per CTA (two per lane)

// Factored J of an FP32 tile coordination CV (see coord_j_parts).
struct CoordParts {
    const float4* rowpart = nullptr;  // [W][nbchunk][nA]
    const float4* colpart = nullptr;  // [W][ntile][nB_stride]
    const int* inv_a = nullptr;       // [max_wn]: position in A or -1
    const int* inv_b = nullptr;       // [max_wn]: position in B or -1; null: B = all atoms
    const double* scw = nullptr;      // [W] scale
    int nA = 0, nbchunk = 0, ntile = 0, nB_stride = 0;
};
constexpr int C2_U = 8;    // rotation steps whose pair terms are computed together
static_assert(CT_B == CT_T, "one staged partner per thread");

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// d - L rint(d / L) for two pairs along one axis (L = hi + lo in two floats);
// iL = hi = lo = 0 on an open axis leaves d unchanged.
__device__ __forceinline__ float2 min_image2(float2 d, float2 iL, float2 nhi, float2 nlo)
{
    float2 n = __ffma2_rn(d, iL, f2(12582912.f));
    n = __fadd2_rn(n, f2(-12582912.f));
    d = __ffma2_rn(n, nhi, d);
    return __ffma2_rn(n, nlo, d);
}


// One CTA's work of an FP32 tile coordination CV for one walker: the walker's
// arrays are already offset (pos = first atom, rowpart/colpart = the walker's
// partials, xi = the walker's CV value).
struct CoordTile2 {
    const float4* pos;
    int nw;           // atoms of the walker
    const int* A;     // walker-local indices of A
    int nA;
    const int* B;     // walker-local indices of B, or null: all atoms
    int nB;
    int nbchunk, ntile;
    Box box;
    float inv_r0sq;
    int h;            // n / 2
    float gpref;      // -n / r0^2
    float4* rowpart;  // [nbchunk][nA]
    float4* colpart;  // [ntile][nB_stride]
    int nB_stride;
    double scw;       // scale
    double* xi;       // the walker's CV value (accumulated)
    const int* inv_b; // position in B of each walker atom, or null
    double xq, ixq;   // 2^q and 2^-q of the exact share quantum
};

// Tile (of C2_A members of A) x chunk (of CT_B partners) for CT_T threads
// tid = 0 .. CT_T-1 (warp-aligned).  Wait is called once before the first
// position read, Sync is the barrier of the CT_T threads.
template <int HC, class Wait, class Sync>
__device__ __forceinline__ void coord_tile2_body(const CoordTile2& t, int tile, int chunk, int tid, float4* srcA,
                                                 float4* srcB, float4 (*rowred)[C2_A], double* xred, Wait wait,
                                                 Sync sync)
{
    const int nBw = t.B ? t.nB : t.nw;
    const int lane = tid % 32, warp = tid / 32;
    const int b0 = chunk * CT_B;
    const int mb = min(CT_B, nBw - b0);
    // index lists are constant: read before waiting for the positions
    const int ia0 = tile * C2_A + lane, ia1 = ia0 + 32;
    const int a0 = ia0 < t.nA ? t.A[ia0] : -1, a1 = ia1 < t.nA ? t.A[ia1] : -1;
    const int q = tid;
    const int jq = q < mb ? (t.B ? t.B[b0 + q] : b0 + q) : -1;
    // scale times the share quantum 2^q (thread 0 rounds the CTA's share)
    const double sxq = tid == 0 ? t.scw * t.xq : 0.0;
    // position in B of this lane's targets (for their self pairs), in the
    // warps that sum the rows
    int pbs = -1;
    if (warp == 2 || warp == 3) {
        const int a = warp == 2 ? a0 : a1;
        if (a >= 0) pbs = t.inv_b ? t.inv_b[a] : (a < t.nw ? a : -1);
    }
    wait();
    // the partner's and both targets' positions in one round trip, before
    // the shared-memory stores (which the compiler will not move loads past)
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), t0 = p, t1 = p;
    if (jq >= 0) p = t.pos[jq];
    if (a0 >= 0) t0 = t.pos[a0];
    if (a1 >= 0) t1 = t.pos[a1];
    if (jq >= 0) {
        srcA[q] = make_float4(-p.x, -p.x, -p.y, -p.y);
        srcB[q] = make_float4(-p.z, -p.z, 1.f, 1.f);
    } else {  // padding: weight 0
        srcA[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        srcB[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float2 tx = make_float2(t0.x, t1.x), ty = make_float2(t0.y, t1.y), tz = make_float2(t0.z, t1.z);
    // an empty target lane adds nothing to the columns
    const float2 gpl = make_float2(a0 >= 0 ? t.gpref : 0.f, a1 >= 0 ? t.gpref : 0.f);
    float2 iL[3], nhi[3], nlo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool per = t.box.Lf[k] > 0.f;
        iL[k] = f2(per ? t.box.invLf[k] : 0.f);
        nhi[k] = f2(per ? -t.box.Lf[k] : 0.f);
        nlo[k] = f2(per ? -t.box.Llo[k] : 0.f);
    }
    sync();
    // rotation over the warp's 32 partners: the column sum of a partner
    // (both targets of the lane added) moves one lane down per step and ends
    // in the partner's own lane.  A shuffle orders the code around it, so the
    // pair terms of C2_U steps are computed first (independent, interleaved)
    // and then passed along.
    float2 gx = f2(0.f), gy = gx, gz = gx, sv = gx;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    const int base = warp * 32, from = (lane + 1) & 31;
    const float2 inv2 = f2(t.inv_r0sq), one2 = f2(1.f);
#pragma unroll 1
    for (int k0 = 0; k0 < 32; k0 += C2_U) {
        float hx[C2_U], hy[C2_U], hz[C2_U];
#pragma unroll
        for (int u = 0; u < C2_U; ++u) {
            const int m = base + ((lane + k0 + u) & 31);
            const float4 pa = srcA[m], pb = srcB[m];
            const float2 dx = min_image2(__fadd2_rn(tx, make_float2(pa.x, pa.y)), iL[0], nhi[0], nlo[0]);
            const float2 dy = min_image2(__fadd2_rn(ty, make_float2(pa.z, pa.w)), iL[1], nhi[1], nlo[1]);
            const float2 dz = min_image2(__fadd2_rn(tz, make_float2(pb.x, pb.y)), iL[2], nhi[2], nlo[2]);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 y = __fmul2_rn(r2, inv2);
            float2 yh1;  // y^(h-1)
            if constexpr (HC == 1) {
                yh1 = one2;
            } else if constexpr (HC > 1) {
                yh1 = y;
#pragma unroll
                for (int e = 2; e < HC; ++e) yh1 = __fmul2_rn(yh1, y);
            } else {
                yh1 = one2;
                for (int e = 1; e < t.h; ++e) yh1 = __fmul2_rn(yh1, y);
            }
            const float2 den = __ffma2_rn(yh1, y, one2);
            const float2 s = __fmul2_rn(make_float2(rcp_approx(den.x), rcp_approx(den.y)), make_float2(pb.z, pb.w));
            sv = __fadd2_rn(sv, s);
            const float2 gr = __fmul2_rn(__fmul2_rn(s, s), __fmul2_rn(yh1, gpl));
            const float2 px = __fmul2_rn(gr, dx), py = __fmul2_rn(gr, dy), pz = __fmul2_rn(gr, dz);
            gx = __fadd2_rn(gx, px);
            gy = __fadd2_rn(gy, py);
            gz = __fadd2_rn(gz, pz);
            hx[u] = px.x + px.y;
            hy[u] = py.x + py.y;
            hz[u] = pz.x + pz.y;
        }
#pragma unroll
        for (int u = 0; u < C2_U; ++u) {
            cx = __shfl_sync(0xffffffffu, cx + hx[u], from);
            cy = __shfl_sync(0xffffffffu, cy + hy[u], from);
            cz = __shfl_sync(0xffffffffu, cz + hz[u], from);
        }
    }
    if (base + lane < mb) t.colpart[(size_t)tile * t.nB_stride + b0 + base + lane] = make_float4(-cx, -cy, -cz, 0.f);
    rowred[warp][lane] = make_float4(gx.x, gy.x, gz.x, sv.x);
    rowred[warp][lane + 32] = make_float4(gx.y, gy.y, gz.y, sv.y);
    sync();
    // rows of the chunk (warps 2 and 3 -- warp 0 was measured ~1.2 us slower
    // here -- summing the warps' partials in order) and this CTA's share of
    // the CV value; the pair of a target with itself added s(0) in the chunk
    // that holds it as a partner
    if (warp == 2 || warp == 3) {
        const int r = tid - 64, ia = tile * C2_A + r;
        cf xs{0.f, 0.f};
        if (ia < t.nA) {
            float4 u = rowred[0][r];
            for (int k = 1; k < CT_T / 32; ++k) {
                const float4 v = rowred[k][r];
                u.x += v.x;
                u.y += v.y;
                u.z += v.z;
                u.w += v.w;
            }
            t.rowpart[(size_t)chunk * t.nA + ia] = u;
            if (pbs >= b0 && pbs < b0 + mb) u.w -= rcp_approx(1.f);
            xs.hi = u.w;
        }
        // compensated FP32 (a dependent FP64 operation costs ~64 cycles on
        // this GPU); the share is rounded to the exact quantum in FP64 once
        for (int off = 16; off > 0; off >>= 1) xs = cf_add(xs, cf_shfl_xor(xs, off));
        if (lane == 0) reinterpret_cast<float2*>(xred)[warp - 2] = make_float2(xs.hi, xs.lo);
    }
    sync();
    if (tid == 0) {
        const float2 u = reinterpret_cast<const float2*>(xred)[0], v = reinterpret_cast<const float2*>(xred)[1];
        const cf c = cf_add(cf{u.x, u.y}, cf{v.x, v.y});
        atomicAdd(t.xi, rint(((double)c.hi + (double)c.lo) * sxq) * t.ixq);
    }
}

// J of one atom of walker w from the FP32 tile partials, given its position
// pb in B and ia in A (-1: not a member) and the walker's scale f: its
// column sums over the tiles, then its row sums over the chunks, each in
// increasing order, times the scale.  coord_j_parts takes the atom's local
// index li instead and reads the three itself.
__device__ __forceinline__ float4 coord_j_parts_at(const CoordParts& p, int w, int pb, int ia, float f)
{
    // the first JB column and JB row partials are in flight together; the
    // sums run columns then rows, each in increasing order
    constexpr int JB = 8;
    const int nt = pb >= 0 ? p.ntile : 0, nc = ia >= 0 ? p.nbchunk : 0;
    const float4* cb = p.colpart + (size_t)w * p.ntile * p.nB_stride + (pb >= 0 ? pb : 0);
    const float4* rb = p.rowpart + (size_t)w * p.nbchunk * p.nA + (ia >= 0 ? ia : 0);
    float4 cu[JB], ru[JB];
#pragma unroll
    for (int q = 0; q < JB; ++q) {
        cu[q] = q < nt ? __ldcg(cb + (size_t)q * p.nB_stride) : make_float4(0.f, 0.f, 0.f, 0.f);
        ru[q] = q < nc ? __ldcg(rb + (size_t)q * p.nA) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
    for (int q = 0; q < JB; ++q)
        if (q < nt) {
            sx += cu[q].x;
            sy += cu[q].y;
            sz += cu[q].z;
        }
    for (int t = JB; t < nt; ++t) {
        const float4 u = __ldcg(cb + (size_t)t * p.nB_stride);
        sx += u.x;
        sy += u.y;
        sz += u.z;
    }
#pragma unroll
    for (int q = 0; q < JB; ++q)
        if (q < nc) {
            sx += ru[q].x;
            sy += ru[q].y;
            sz += ru[q].z;
        }
    for (int c = JB; c < nc; ++c) {
        const float4 u = __ldcg(rb + (size_t)c * p.nA);
        sx += u.x;
        sy += u.y;
        sz += u.z;
    }
    return make_float4(f * sx, f * sy, f * sz, 0.f);
}

__device__ __forceinline__ float4 coord_j_parts(const CoordParts& p, int w, int li)
{
    return coord_j_parts_at(p, w, p.inv_b ? p.inv_b[li] : li, p.inv_a[li], (float)p.scw[w]);
}

}  // namespace wtmd
