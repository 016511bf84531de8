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
    auto baoa = [&](R& xx, R& vv, R ff, R g) {
        vv += half * ff * inv_m;
        xx += half * vv;
        vv = c1 * vv + c2 * g;
        xx += half * vv;
    };
    baoa(xi.x, vi.x, fi.x, n.g[0]);
    baoa(xi.y, vi.y, fi.y, n.g[1]);
    if (dims > 2) baoa(xi.z, vi.z, fi.z, n.g[2]);
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

// Deposition by one CTA (all its threads call this): every `stride` steps
// each walker appends a hill at its CVs with height w0 exp(-V inv_dT) in
// FP64 (walker order), then the step counter advances.
template <typename R>
__device__ void deposit_block(const DepPrm& p, const double* __restrict__ xi, const R* __restrict__ V,
                              long long* __restrict__ count, long long* __restrict__ step, long long* __restrict__ dep,
                              double* __restrict__ ctr, dbl4* __restrict__ h64, float* __restrict__ h32,
                              unsigned* status)
{
    __shared__ long long base;
    __shared__ int doit;
    __shared__ double c[3];
    if (threadIdx.x == 0) {
        const long long t = *step;
        doit = p.stride > 0 && (t + 1) % p.stride == 0;
        base = *count;
        if (doit && base + p.W > p.cap) {
            atomicOr(status, ST_CAPACITY);
            doit = 0;
        }
        dep[0] = base;
        dep[1] = doit ? p.W : 0;
        // the centre of the scaled FP32 layout is fixed by the first hill
        // when no grid defined it
        if (doit && isnan(ctr[0]))
            for (int i = 0; i < 3; ++i) ctr[i] = i < p.d ? xi[i] : 0.0;
        for (int i = 0; i < 3; ++i) c[i] = ctr[i];
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
        *step = *step + 1;
    }
}

}  // namespace wtmd
