// Device-side pieces of the MD step shared by the per-kernel step
// (engine.cu, deposit.cu) and the persistent multi-walker step (walkers.cu):
// the thermostat noise, the first half of BAOAB for one atom, and deposition.
//
// BAOAB (Leimkuhler & Matthews 2013): B v += dt/2 F/m; A x += dt/2 v;
// O v = c1 v + sqrt((1 - c1^2) kT/m) R, c1 = exp(-friction dt); A x += dt/2 v;
// forces; B.  The noise of particle i at step t is Philox4x32-10 with key
// (seed lo, seed hi) and counter (t lo, i, t hi, 0); its four words become
// uniforms and two Box-Muller pairs (first three normals used).
//
// Deposition (PySAGES paper, Sec. 2.1.5): every `stride` steps each walker
// appends one hill at its current CVs; height w0 (standard metadynamics) or
// w0 exp(-V(s) / (kT (gamma - 1))) (well-tempered), computed in FP64 from the
// V of the hills that existed before this step's deposits.
#pragma once

#include "wtmd_internal.cuh"

namespace wtmd {

template <typename R> struct Normal3 {
    R g[3];
};

template <typename R> __device__ __forceinline__ Normal3<R> noise3(uint64_t seed, long long step, uint32_t i);

template <> __device__ __forceinline__ Normal3<double> noise3<double>(uint64_t seed, long long step, uint32_t i)
{
    const U4 r = philox10((uint32_t)step, i, (uint32_t)((unsigned long long)step >> 32), 0u, (uint32_t)seed,
                          (uint32_t)(seed >> 32));
    const double k = 2.3283064365386963e-10;  // 2^-32
    const double u0 = ((double)r.v[0] + 0.5) * k, u1 = ((double)r.v[1] + 0.5) * k;
    const double u2 = ((double)r.v[2] + 0.5) * k, u3 = ((double)r.v[3] + 0.5) * k;
    const double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
    double s1, c1, c3;
    sincospi(2.0 * u1, &s1, &c1);
    c3 = cospi(2.0 * u3);
    Normal3<double> n;
    n.g[0] = a * c1;
    n.g[1] = a * s1;
    n.g[2] = b * c3;
    return n;
}

template <> __device__ __forceinline__ Normal3<float> noise3<float>(uint64_t seed, long long step, uint32_t i)
{
    const U4 r = philox10((uint32_t)step, i, (uint32_t)((unsigned long long)step >> 32), 0u, (uint32_t)seed,
                          (uint32_t)(seed >> 32));
    // 24 significant bits: u = (floor(x / 2^8) + 1/2) 2^-24, in (0, 1)
    const float k = 5.9604644775390625e-08f;  // 2^-24
    const float u0 = ((float)(r.v[0] >> 8) + 0.5f) * k, u1 = ((float)(r.v[1] >> 8) + 0.5f) * k;
    const float u2 = ((float)(r.v[2] >> 8) + 0.5f) * k, u3 = ((float)(r.v[3] >> 8) + 0.5f) * k;
    const float a = sqrtf(-2.0f * logf(u0)), b = sqrtf(-2.0f * logf(u2));
    float s1, c1;
    sincospif(2.0f * u1, &s1, &c1);
    Normal3<float> n;
    n.g[0] = a * c1;
    n.g[1] = a * s1;
    n.g[2] = b * cospif(2.0f * u3);
    return n;
}

// B-A-O-A half of a BAOAB step of one particle (x, v, f in registers) with
// the normal deviates g of its step.
template <typename R>
__device__ __forceinline__ void baoa_update(R4<R>& xi, R4<R>& vi, const R4<R>& fi, const R* g, R half, R inv_m, R c1,
                                            R c2, int dims)
{
    auto baoa = [&](R& xx, R& vv, R ff, R gg) {
        vv += half * ff * inv_m;
        xx += half * vv;
        vv = c1 * vv + c2 * gg;
        xx += half * vv;
    };
    baoa(xi.x, vi.x, fi.x, g[0]);
    baoa(xi.y, vi.y, fi.y, g[1]);
    if (dims > 2) baoa(xi.z, vi.z, fi.z, g[2]);
}

// B-A-O-A half of a BAOAB step for atom i at step t (the closing B follows
// the force evaluation).
template <typename R>
__device__ __forceinline__ void baoab_first_atom(long long i, long long t, R4<R>* __restrict__ x, R4<R>* __restrict__ v,
                                                 const R4<R>* __restrict__ f, uint64_t seed, R half, R inv_m, R c1,
                                                 R c2, int dims)
{
    const Normal3<R> n = noise3<R>(seed, t, (uint32_t)i);
    R4<R> xi = x[i], vi = v[i];
    const R4<R> fi = f[i];
    baoa_update<R>(xi, vi, fi, n.g, half, inv_m, c1, c2, dims);
    x[i] = xi;
    v[i] = vi;
}

struct DepPrm {
    long long stride;
    long long cap;
    int W, d;
    double w0, inv_dT;  // inv_dT = 1/(kT (gamma - 1)); 0 for standard metadynamics
    double a[3];        // FP32 layout scale
};

DepPrm dep_prm(const wtmd_t* h);  // deposit.cu

// FP64 bias grid (Sec. 2.1.5): bins per axis, node spacing dx, the lower
// edge lo (node k sits at the cell centre lo + (k + 1/2) dx), the hill
// widths as 1/(2 sigma^2) and the period of a periodic CV (0: none).
struct GridPrm {
    int d;
    int bins[3];
    int off[3];  // offset of axis i in the per-hill factor table
    double lo[3], dx[3], inv2s2[3], per[3];
};

GridPrm grid_prm(const wtmd_t* h);  // deposit.cu

// Grid update after a deposit (dep = {first new hill, count}): the factors
// f[n][off_i + k] = exp(-D^2/(2 sigma_i^2)) of new hill n on axis i at cell
// centre k (minimum image on a periodic axis), then every cell adds
// w_n prod_i f[n][off_i + k_i] over the new hills in order.  Items q0,
// q0 + qs, ... of each loop are this thread's.
__device__ __forceinline__ void grid_factors(const GridPrm& g, const long long* __restrict__ dep,
                                             const dbl4* __restrict__ h64, int tot, double* __restrict__ fac,
                                             long long q0, long long qs)
{
    const long long nnew = dep[1];
    const long long first = dep[0];
    for (long long q = q0; q < nnew * tot; q += qs) {
        const long long n = q / tot;
        const int j = (int)(q % tot);
        int i = 0;
        while (i + 1 < g.d && j >= g.off[i + 1]) ++i;
        const int k = j - g.off[i];
        const dbl4 h = h64[first + n];
        const double s = i == 0 ? h.x : (i == 1 ? h.y : h.z);
        double D = g.lo[i] + (k + 0.5) * g.dx[i] - s;
        if (g.per[i] > 0.0) D -= g.per[i] * rint(D / g.per[i]);
        fac[q] = exp(-D * D * g.inv2s2[i]);
    }
}

__device__ __forceinline__ void grid_add(const GridPrm& g, const long long* __restrict__ dep,
                                         const dbl4* __restrict__ h64, int tot, const double* __restrict__ fac,
                                         long long ncell, double* __restrict__ grid, long long c0, long long cs)
{
    const long long nnew = dep[1];
    if (nnew == 0) return;
    const long long first = dep[0];
    for (long long cidx = c0; cidx < ncell; cidx += cs) {
        int k[3] = {0, 0, 0};
        long long rem = cidx;
        for (int i = g.d - 1; i >= 0; --i) {
            k[i] = (int)(rem % g.bins[i]);
            rem /= g.bins[i];
        }
        double v = grid[cidx];
        for (long long n = 0; n < nnew; ++n) {
            double e = h64[first + n].w;
            for (int i = 0; i < g.d; ++i) e *= fac[n * tot + g.off[i] + k[i]];
            v += e;
        }
        grid[cidx] = v;
    }
}

// The staged form of grid_point: every address first, then every load
// (unrolled: one round of latency), then the sums in corner order.
template <int D, int NC, int NV>
__device__ __forceinline__ void grid_point_staged(const GridPrm& g, const double* __restrict__ grid,
                                                  const long long* cstride, const int* k0, const int* k1,
                                                  const double* t, double& v, double* gr)
{
    double val[NC][NV], wgt[NC], span[NC][D];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        int k[D];
        double w = 1.0;
        long long node = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const bool up = (c >> i) & 1;
            k[i] = up ? k1[i] : k0[i];
            w *= up ? t[i] : 1.0 - t[i];
            node += k[i] * cstride[i];
        }
        wgt[c] = w;
        val[c][0] = grid[node];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int n = g.bins[i];
            int kp, km;
            if (g.per[i] > 0.0) {
                kp = k[i] + 1 == n ? 0 : k[i] + 1;
                km = k[i] == 0 ? n - 1 : k[i] - 1;
                span[c][i] = 2.0 * g.dx[i];
            } else {
                kp = min(k[i] + 1, n - 1);
                km = max(k[i] - 1, 0);
                span[c][i] = kp - km == 2 ? 2.0 * g.dx[i] : g.dx[i];
            }
            val[c][1 + 2 * i] = grid[node + (kp - k[i]) * cstride[i]];
            val[c][2 + 2 * i] = grid[node + (km - k[i]) * cstride[i]];
        }
    }
    v = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) gr[i] = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        v += wgt[c] * val[c][0];
#pragma unroll
        for (int i = 0; i < D; ++i) gr[i] += wgt[c] * ((val[c][1 + 2 * i] - val[c][2 + 2 * i]) / span[c][i]);
    }
}

// Bias and gradient read from the grid instead of summed over the hills (the
// paper's accuracy-for-speed option, Sec. 2.1.5): the grid keeps V at cell
// centres; the gradient at a node along axis i is the central difference of
// its neighbours (one-sided at the ends of a non-periodic axis, wrapped on a
// periodic one), and V and dV/dxi at the point x are multilinear
// interpolations of the node values over the 2^d surrounding nodes.  A
// non-periodic coordinate is clamped to the outermost nodes.  FP64.
// STAGED: every node address first, then every load (one round of memory
// latency, 2^d (1 + 2d) values in registers); otherwise corner by corner
// with few registers, for a caller whose register budget is tight.  Both
// forms add the same terms in the same order.
template <int D, bool STAGED = true>
__device__ __forceinline__ void grid_point(const GridPrm& g, const double* __restrict__ grid, const double* x,
                                           double& v, double* gr)
{
    constexpr int NC = 1 << D;       // corner nodes
    constexpr int NV = 1 + 2 * D;    // per corner: the node and its two neighbours on each axis
    long long cstride[D];
    cstride[D - 1] = 1;
#pragma unroll
    for (int i = D - 2; i >= 0; --i) cstride[i] = cstride[i + 1] * g.bins[i + 1];
    int k0[D], k1[D];
    double t[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const int n = g.bins[i];
        double u = (x[i] - g.lo[i]) / g.dx[i] - 0.5;
        if (g.per[i] > 0.0) {
            u -= (double)n * floor(u / (double)n);
            if (!(u >= 0.0 && u < (double)n)) u = 0.0;  // rounding at n, or a non-finite / huge coordinate
            k0[i] = (int)floor(u);
            k1[i] = k0[i] + 1 == n ? 0 : k0[i] + 1;
        } else {
            u = fmin(fmax(u, 0.0), (double)(n - 1));
            k0[i] = min((int)floor(u), n - 2);
            k1[i] = k0[i] + 1;
        }
        t[i] = u - (double)k0[i];
    }
    if constexpr (!STAGED) {
        v = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) gr[i] = 0.0;
#pragma unroll 1
        for (int c = 0; c < NC; ++c) {
            double w = 1.0;
            long long node = 0;
            int k[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const bool up = (c >> i) & 1;
                k[i] = up ? k1[i] : k0[i];
                w *= up ? t[i] : 1.0 - t[i];
                node += k[i] * cstride[i];
            }
            v += w * grid[node];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int n = g.bins[i];
                int kp, km;
                double sp;
                if (g.per[i] > 0.0) {
                    kp = k[i] + 1 == n ? 0 : k[i] + 1;
                    km = k[i] == 0 ? n - 1 : k[i] - 1;
                    sp = 2.0 * g.dx[i];
                } else {
                    kp = min(k[i] + 1, n - 1);
                    km = max(k[i] - 1, 0);
                    sp = kp - km == 2 ? 2.0 * g.dx[i] : g.dx[i];
                }
                gr[i] += w * ((grid[node + (kp - k[i]) * cstride[i]] - grid[node + (km - k[i]) * cstride[i]]) / sp);
            }
        }
    } else {
        grid_point_staged<D, NC, NV>(g, grid, cstride, k0, k1, t, v, gr);
    }
}

// Harmonic bias of one walker about its window centre (Sec. 2.1.1; one
// window per walker for umbrella sampling, Sec. 2.1.2):
// V = sum_c k_c/2 (xi_c - xi0_c)^2, dV/dxi_c = k_c (xi_c - xi0_c), the
// difference by the minimum image on a periodic CV.  With `sum` the walker's
// xi is added to its window sums (the caller counts the sample).
template <typename R>
__device__ __forceinline__ void harmonic_point(int d, const double* k, const double* per, const double* __restrict__ xi,
                                               const double* __restrict__ centre, R* V, R* dV,
                                               double* __restrict__ sum)
{
    double v = 0.0;
    for (int c = 0; c < d; ++c) {
        const double x = xi[c];
        double D = x - centre[c];
        if (per[c] > 0.0) D -= per[c] * rint(D / per[c]);
        v += 0.5 * k[c] * D * D;
        dV[c] = (R)(k[c] * D);
        if (sum) sum[c] += x;
    }
    *V = (R)v;
}

// Deposition by one CTA (all its threads call this): every `stride` steps
// each walker appends a hill at its CVs with height w0 exp(-V inv_dT) in
// FP64 (walker order), then the step counter advances.  deposit_block_at
// takes the step counter and the hill count (pre[0], pre[1]) and the layout
// centre (cpre) as thread 0 read them earlier (they change only here, so a
// kernel can read them before its dependency wait); deposit_block reads
// them itself.
template <typename R>
__device__ void deposit_block_at(const DepPrm& p, const long long* pre, const double* cpre,
                                 const double* __restrict__ xi, const R* __restrict__ V, long long* __restrict__ count,
                                 long long* __restrict__ step, long long* __restrict__ dep, double* __restrict__ ctr,
                                 dbl4* __restrict__ h64, float* __restrict__ h32, unsigned* status)
{
    __shared__ long long base;
    __shared__ int doit;
    __shared__ double c[3];
    if (threadIdx.x == 0) {
        const long long t = pre[0];
        doit = p.stride > 0 && (t + 1) % p.stride == 0;
        base = pre[1];
        if (doit && base + p.W > p.cap) {
            atomicOr(status, ST_CAPACITY);
            doit = 0;
        }
        dep[0] = base;
        dep[1] = doit ? p.W : 0;
        // the centre of the scaled FP32 layout is fixed by the first hill
        // when no grid defined it
        double cc[3] = {cpre[0], cpre[1], cpre[2]};
        if (doit && isnan(cc[0]))
            for (int i = 0; i < 3; ++i) ctr[i] = cc[i] = i < p.d ? xi[i] : 0.0;
        for (int i = 0; i < 3; ++i) c[i] = cc[i];
    }
    __syncthreads();
    if (doit) {
        for (int w = threadIdx.x; w < p.W; w += blockDim.x) {
            const long long k = base + w;
            double s[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < p.d; ++i) s[i] = xi[w * 4 + i];
            const double hgt = p.w0 * exp(-(double)V[w] * p.inv_dT);
            h64[k] = dbl4{s[0], s[1], s[2], hgt};
            const long long b = (k >> 1) * 8 + (k & 1);
            h32[b + 0] = (float)(-(s[0] - c[0]) * p.a[0]);
            h32[b + 2] = (float)(-(s[1] - c[1]) * p.a[1]);
            h32[b + 4] = (float)(-(s[2] - c[2]) * p.a[2]);
            h32[b + 6] = (float)(-log2(hgt));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (doit) *count = base + p.W;
        *step = pre[0] + 1;
    }
}

template <typename R>
__device__ void deposit_block(const DepPrm& p, const double* __restrict__ xi, const R* __restrict__ V,
                              long long* __restrict__ count, long long* __restrict__ step, long long* __restrict__ dep,
                              double* __restrict__ ctr, dbl4* __restrict__ h64, float* __restrict__ h32,
                              unsigned* status)
{
    __shared__ long long pre[2];
    __shared__ double cpre[3];
    if (threadIdx.x == 0) {
        pre[0] = *step;
        pre[1] = *count;
        for (int i = 0; i < 3; ++i) cpre[i] = ctr[i];
    }
    deposit_block_at<R>(p, pre, cpre, xi, V, count, step, dep, ctr, h64, h32, status);
}

}  // namespace wtmd
