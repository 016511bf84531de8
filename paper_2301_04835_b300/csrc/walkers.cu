// Many walkers of uneven size in one persistent launch per MD step.
//
// Walkers are independent systems (Lennard-Jones clusters in open space, or
// each in its own periodic box of the configured size) that share one hill
// list; the paper runs replicas as separate simulations (Sec. 2, replicas
// through concurrent.futures / MPI).  One cooperative kernel does a whole
// step for all walkers, with bounded grid barriers between the phases:
//   P0  first half of BAOAB for every atom;
//   P1  (walker, target tile) tasks, handed out by an atomic queue in order
//       of decreasing cost: the walker's positions are staged in shared
//       memory and one all-pairs loop gives the LJ force, the coordination
//       row sum and its gradient (A = B = all atoms) of each target, plus the
//       targets' first and second moments for Rg; the walker's last task
//       finishes its CVs;
//   P2  the bias at every walker's CVs, from the bias source of the handle:
//       hills: P2a the hills sum for all walker points over the shared hill
//              list (the FP32 bulk-copy ring task of hills.cu), one partial
//              per hill split, P2b a fixed-order reduction of the splits;
//       grid:  the FP64 grid read by interpolation (Sec. 2.1.5), one thread
//              per walker;
//       harmonic windows: each walker's harmonic bias about its own centre
//              (Sec. 2.1.1; umbrella windows, Sec. 2.1.2), with the window
//              sums of xi accumulated in a step;
//   P3  deposition (CTA 0) and, for every atom, the bias force -J^T dV/dxi
//       added to the LJ force and the closing half kick.
// The FP64 bias grid, when configured, is updated by the two grid kernels
// that follow (they exit at once on steps without a deposit; harmonic
// windows deposit nothing).  In a periodic box every pair difference and
// every Rg member is taken by the minimum image (Rg members relative to the
// walker's first atom, as in the per-kernel path).
// Tile sizes, CTAs per SM and the hill split count come from the autotuner
// (wtmd_autotune).  Every reduction has a fixed order: deterministic.
#include <algorithm>
#include <vector>

#include "hills_dev.cuh"
#include "step_dev.cuh"

namespace wtmd {

int launch_grid_update(wtmd_t* h);

constexpr int WK_T = 256;

struct WkArgs {
    int W;
    long long N;
    const int64_t* woff;
    const int* wn;
    const int* aw;
    const int4* tasks;  // (walker, first target, end target, task index within walker), by decreasing cost
    int ntasks;
    int T;              // targets per task
    const int* tbase;   // [W] first partial slot of the walker's tasks
    const int* tcount;  // [W]
    double* tpart;      // [ntasks][2]
    unsigned* ticket;   // [W]
    float4* rgc;        // [2W]: Rg centre relative to the first member and Jacobian factor; then the first member
    float4* x;
    float4* v;
    float4* f;
    float rc2, sig2, eps24, half, inv_m, c1, c2;
    uint64_t seed;
    long long* step;
    int d, cv_coord, cv_rg;
    float inv_r0sq;
    int hpow;
    const double* coord_scw;  // [W]
    double rg_scale;
    int rg_intensive;
    float4* J;  // [d][N]
    double* xi;
    // hills
    const float4* hp;
    const long long* cnt;
    const double* ctr;
    HillPrmF32 hprm;
    dbl4* hpart;
    int hsplit;
    HillOut<float> hout;
    // deposition
    DepPrm dep;
    long long* count;
    long long* depw;
    double* ctrw;
    dbl4* h64;
    float* h32;
    unsigned* bar;
    unsigned* status;
    int max_wn;
    long long wait_limit;  // grid-barrier wait bound (SM cycles)
    // periodic box (PER kernels): edge as Lf + Llo, 1/L; 0 on an open axis
    Box box;
    // bias source: 0 hills, 1 harmonic windows, 2 grid
    int bias;
    const double* hcen;  // [W][4] window centres
    double* hsum;        // [W][4] window sums of xi, then the sample count
    double hk[3], hper[3];
    GridPrm g;
    const double* grid;
};

// Targets per pair task of an n-atom walker: the plan's T, or for a smaller
// walker the least power of two >= n (>= 32), so that its threads split the
// sources instead of idling.
__host__ __device__ inline int wk_targets(int n, int T)
{
    int t = 32;
    while (t < n && t < T) t <<= 1;
    return t;
}

struct PairAcc {
    float fx, fy, fz, gx, gy, gz, sv;
};

// Staged walker positions, two atoms per pair of float4 records, negated:
// pair m holds (-x_2m, -x_2m+1, -y_2m, -y_2m+1), (-z_2m, -z_2m+1, w_2m, w_2m+1)
// with weight w = 1 (a walker of odd size pads its last pair with a far
// point of weight 0).  Each pair instruction of the loop below then serves
// two sources (packed f32x2).
constexpr float WK_FAR = -1.0e4f;  // negated coordinate of the padding point

__device__ __forceinline__ float4 wk_atom(const float4* __restrict__ wpos, int q)
{
    const float4 A = wpos[q & ~1], B = wpos[(q & ~1) + 1];
    return (q & 1) ? make_float4(-A.y, -A.w, -B.y, 0.f) : make_float4(-A.x, -A.z, -B.x, 0.f);
}

struct PairAcc2 {
    float2 fx, fy, fz, gx, gy, gz, sv;
};

// Minimum image of two differences at once: n = rint(d / L) by the
// 1.5 * 2^23 rounding constant (exact for |d / L| < 2^22), then
// d - n Lf - n Llo with the box edge as two floats; an open axis has
// 1/L = L = 0 and keeps d.
__device__ __forceinline__ float2 wk_wrap2(float2 d, float2 iL, float2 nLf, float2 nLlo)
{
    const float2 n = __fadd2_rn(__ffma2_rn(d, iL, make_float2(12582912.f, 12582912.f)),
                                make_float2(-12582912.f, -12582912.f));
    return __ffma2_rn(n, nLlo, __ffma2_rn(n, nLf, d));
}

// LJ force and coordination terms of target i (position p) against the
// source pairs [m0, m1), its own pair with itself left out (replaced by the
// padding point).  One approximate reciprocal of r^2 serves both: with
// y = r^2/r0^2 and s = 1/(1 + y^h), ds/dx = -n y^h s^2 dx / r^2 (n = 2h).
// H > 0 fixes the exponent h at compile time, H = 0 reads it from the
// arguments and caps y^h at 1e30 (beyond it s and ds/dx are below FP32's
// range anyway, and the cap keeps y^h s^2 finite for far pairs and the
// padding point).  PER: minimum-image differences; the padding point and
// the left-out self pair (weight 0) are then moved to r^2 = rc^2, where the
// LJ cutoff drops them and the coordination terms are 0.
template <int H, bool PER>
__device__ __forceinline__ void pair_range2(const float4* __restrict__ wpos, float4 p, int i, int m0, int m1,
                                            const WkArgs& a, PairAcc2& c)
{
    const bool co = a.cv_coord >= 0;
    const float2 px = make_float2(p.x, p.x), py = make_float2(p.y, p.y), pz = make_float2(p.z, p.z);
    const float2 one = make_float2(1.f, 1.f), inv = make_float2(a.inv_r0sq, a.inv_r0sq);
    const float2 nneg = make_float2(-2.f * (float)a.hpow, -2.f * (float)a.hpow);
    const float2 sig2 = make_float2(a.sig2, a.sig2), e24 = make_float2(a.eps24, a.eps24);
    const float2 two = make_float2(2.f, 2.f), mone = make_float2(-1.f, -1.f);
    float2 iL[3], nLf[3], nLlo[3];
    if constexpr (PER) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            iL[k] = make_float2(a.box.invLf[k], a.box.invLf[k]);
            nLf[k] = make_float2(-a.box.Lf[k], -a.box.Lf[k]);
            nLlo[k] = make_float2(-a.box.Llo[k], -a.box.Llo[k]);
        }
    }
    const int mi = i >> 1;
#pragma unroll 2
    for (int m = m0; m < m1; ++m) {
        float4 A = wpos[2 * m], B = wpos[2 * m + 1];
        if (m == mi) {
            if (i & 1) {
                A.y = WK_FAR;
                A.w = WK_FAR;
                B.y = WK_FAR;
                B.w = 0.f;
            } else {
                A.x = WK_FAR;
                A.z = WK_FAR;
                B.x = WK_FAR;
                B.z = 0.f;
            }
        }
        float2 dx = __fadd2_rn(px, make_float2(A.x, A.y)), dy = __fadd2_rn(py, make_float2(A.z, A.w)),
               dz = __fadd2_rn(pz, make_float2(B.x, B.y));
        if constexpr (PER) {
            dx = wk_wrap2(dx, iL[0], nLf[0], nLlo[0]);
            dy = wk_wrap2(dy, iL[1], nLf[1], nLlo[1]);
            dz = wk_wrap2(dz, iL[2], nLf[2], nLlo[2]);
        }
        float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        if constexpr (PER) {
            r2.x = B.z != 0.f ? r2.x : a.rc2;
            r2.y = B.w != 0.f ? r2.y : a.rc2;
        }
        const float2 ir2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
        if (co) {
            const float2 y = __fmul2_rn(r2, inv);
            float2 yh = y;
            if constexpr (H > 0) {
#pragma unroll
                for (int k = 1; k < H; ++k) yh = __fmul2_rn(yh, y);
            } else {
                for (int k = 1; k < a.hpow; ++k) yh = __fmul2_rn(yh, y);
                yh.x = fminf(yh.x, 1e30f);
                yh.y = fminf(yh.y, 1e30f);
            }
            const float2 den = __fadd2_rn(one, yh);
            const float2 sw = make_float2(rcp_approx(den.x), rcp_approx(den.y));
            const float2 sg = __fmul2_rn(sw, make_float2(B.z, B.w));  // weighted s
            c.sv = __fadd2_rn(c.sv, sg);
            const float2 gr = __fmul2_rn(__fmul2_rn(__fmul2_rn(nneg, yh), __fmul2_rn(sg, sw)), ir2);
            c.gx = __ffma2_rn(gr, dx, c.gx);
            c.gy = __ffma2_rn(gr, dy, c.gy);
            c.gz = __ffma2_rn(gr, dz, c.gz);
        }
        const float2 sr2 = __fmul2_rn(sig2, ir2);
        const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
        float2 fr = __fmul2_rn(__fmul2_rn(e24, __fmul2_rn(sr6, __ffma2_rn(sr6, two, mone))), ir2);
        fr.x = r2.x < a.rc2 ? fr.x : 0.f;
        fr.y = r2.y < a.rc2 ? fr.y : 0.f;
        c.fx = __ffma2_rn(fr, dx, c.fx);
        c.fy = __ffma2_rn(fr, dy, c.fy);
        c.fz = __ffma2_rn(fr, dz, c.fz);
    }
}

template <int D, int H, bool PER>
__global__ void __launch_bounds__(WK_T, 4) walkers_step_kernel(const __grid_constant__ WkArgs a, int mode)
{
    extern __shared__ __align__(128) unsigned char wk_smem[];
    float4 (*ring)[2 * CHUNK] = reinterpret_cast<float4 (*)[2 * CHUNK]>(wk_smem);
    uint64_t* hbar = reinterpret_cast<uint64_t*>(wk_smem + sizeof(float4) * NST * 2 * CHUNK);
    float4* wpos = reinterpret_cast<float4*>(wk_smem + sizeof(float4) * NST * 2 * CHUNK + 128);
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x;

    // ---- P0: B-A-O-A
    if (mode == 0) {
        const long long t = *a.step;
        for (long long i = (long long)blockIdx.x * WK_T + tid; i < a.N; i += (long long)G * WK_T)
            baoab_first_atom<float>(i, t, a.x, a.v, a.f, a.seed, a.half, a.inv_m, a.c1, a.c2, 3);
        if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return;
    }

    // ---- P1: pair tasks, taken from a queue in decreasing cost (greedy
    // balance); the walker's last task finishes its CVs
    {
        __shared__ float red[WK_T][7];
        __shared__ cf tw[WK_T / 32][5];
        __shared__ int next, last;
        for (;;) {
            __syncthreads();  // the previous task is done with wpos, red, tw
            if (tid == 0) next = (int)atomicAdd(a.bar + 2, 1u);
            __syncthreads();
            const int task = next;
            if (task >= a.ntasks) break;
            const int4 tk = a.tasks[task];
            const int w = tk.x, t0 = tk.y, t1 = tk.z;
            const int n = a.wn[w];
            const long long o = a.woff[w];
            const int T = wk_targets(n, a.T), Gs = WK_T / T;
            const int ti = tid % T, sl = tid / T;
            const int np = (n + 1) / 2;
            for (int q = tid; q < np; q += WK_T) {
                const float4 u = a.x[o + 2 * q];
                const bool two = 2 * q + 1 < n;
                const float4 v = two ? a.x[o + 2 * q + 1] : make_float4(-WK_FAR, -WK_FAR, -WK_FAR, 0.f);
                wpos[2 * q] = make_float4(-u.x, -v.x, -u.y, -v.y);
                wpos[2 * q + 1] = make_float4(-u.z, -v.z, 1.f, two ? 1.f : 0.f);
            }
            __syncthreads();
            const int i = t0 + ti;
            const bool act = i < t1;
            PairAcc acc{};
            if (act) {
                const float4 p = wk_atom(wpos, i);
                PairAcc2 c2{};
                const int m0 = (int)((long long)np * sl / Gs), m1 = (int)((long long)np * (sl + 1) / Gs);
                pair_range2<H, PER>(wpos, p, i, m0, m1, a, c2);
                acc.fx = c2.fx.x + c2.fx.y;
                acc.fy = c2.fy.x + c2.fy.y;
                acc.fz = c2.fz.x + c2.fz.y;
                acc.gx = c2.gx.x + c2.gx.y;
                acc.gy = c2.gy.x + c2.gy.y;
                acc.gz = c2.gz.x + c2.gz.y;
                acc.sv = c2.sv.x + c2.sv.y;
            }
            // sum the source slices of each target in slice order
            red[tid][0] = acc.fx;
            red[tid][1] = acc.fy;
            red[tid][2] = acc.fz;
            red[tid][3] = acc.gx;
            red[tid][4] = acc.gy;
            red[tid][5] = acc.gz;
            red[tid][6] = acc.sv;
            __syncthreads();
            // task moments: coordination row sum, and for Rg the sums of
            // u = x - x_0 and |u|^2 (x_0 = the walker's first atom, which
            // keeps the shifted second moment well conditioned)
            cf mom[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (sl == 0 && act) {
                float v[7];
                for (int k = 0; k < 7; ++k) v[k] = red[ti][k];
                for (int g = 1; g < Gs; ++g)
                    for (int k = 0; k < 7; ++k) v[k] += red[g * T + ti][k];
                a.f[o + i] = make_float4(v[0], v[1], v[2], 0.f);
                if (a.cv_coord >= 0) {
                    const float jf = (float)(2.0 * a.coord_scw[w]);  // A = B: both orderings of each pair
                    a.J[(size_t)a.cv_coord * a.N + o + i] = make_float4(jf * v[3], jf * v[4], jf * v[5], 0.f);
                    mom[0] = cf{v[6], 0.f};
                }
                if (a.cv_rg >= 0) {
                    const float4 p = wk_atom(wpos, i), p0 = wk_atom(wpos, 0);
                    float ux = p.x - p0.x, uy = p.y - p0.y, uz = p.z - p0.z;
                    if constexpr (PER) {
                        ux = min_image<float>(ux, a.box, 0);
                        uy = min_image<float>(uy, a.box, 1);
                        uz = min_image<float>(uz, a.box, 2);
                    }
                    mom[1] = cf{ux, 0.f};
                    mom[2] = cf{uy, 0.f};
                    mom[3] = cf{uz, 0.f};
                    mom[4] = cf{fmaf(ux, ux, fmaf(uy, uy, uz * uz)), 0.f};
                }
            }
            for (int k = 0; k < 5; ++k)
                for (int off = 16; off > 0; off >>= 1) mom[k] = cf_add(mom[k], cf_shfl_xor(mom[k], off));
            if (tid % 32 == 0)
                for (int k = 0; k < 5; ++k) tw[tid / 32][k] = mom[k];
            __syncthreads();
            if (tid == 0) {
                double* slot = a.tpart + 5 * (size_t)(a.tbase[w] + tk.w);
                for (int k = 0; k < 5; ++k) {
                    cf t = tw[0][k];
                    for (int q = 1; q < WK_T / 32; ++q) t = cf_add(t, tw[q][k]);
                    slot[k] = cf_val(t);
                }
                __threadfence();
                last = atomicAdd(&a.ticket[w], 1u) == (unsigned)a.tcount[w] - 1;
            }
            __syncthreads();
            // the walker's last task sums the task moments: warp 0, lanes
            // over tasks, then a fixed xor tree
            if (last && tid < 32) {
                __threadfence();
                double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                const double* base = a.tpart + 5 * (size_t)a.tbase[w];
                for (int k = tid; k < a.tcount[w]; k += 32)
                    for (int q = 0; q < 5; ++q) m[q] += __ldcg(base + 5 * k + q);
                for (int q = 0; q < 5; ++q)
                    for (int off = 16; off > 0; off >>= 1) m[q] += __shfl_xor_sync(0xffffffffu, m[q], off);
                if (tid == 0) {
                    if (a.cv_coord >= 0) a.xi[w * 4 + a.cv_coord] = a.coord_scw[w] * m[0];
                    if (a.cv_rg >= 0) {
                        const double cx = m[1] / n, cy = m[2] / n, cz = m[3] / n;
                        const double Q = fmax(m[4] - n * (cx * cx + cy * cy + cz * cz), 0.0);
                        const double rg = sqrt(Q / n);
                        double sc = a.rg_scale != 0.0 ? a.rg_scale : 1.0;
                        if (a.rg_intensive) sc /= cbrt((double)n);
                        a.xi[w * 4 + a.cv_rg] = sc * rg;
                        a.rgc[w] = make_float4((float)cx, (float)cy, (float)cz, (float)(sc / (n * rg)));
                        a.rgc[a.W + w] = wk_atom(wpos, 0);
                    }
                    a.ticket[w] = 0u;
                }
            }
        }
    }
    if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return;

    if (a.bias == 0) {
        // ---- P2a: hills partials for all walker points
        const int tiles = (a.W + WK_T - 1) / WK_T;
        bool fresh = true;
        for (int task = blockIdx.x; task < tiles * a.hsplit; task += G) {
            if (!hills_f32_task<D, 1, false, double>(a.hp, nullptr, a.cnt, a.xi, 4, a.W, a.ctr, a.hprm, a.hpart, a.status,
                                                     task / a.hsplit, task % a.hsplit, a.hsplit, ring, hbar, fresh))
                return;
            fresh = false;
        }
        if (!fresh) {
            __syncthreads();
            if (tid == 0)
                for (int s = 0; s < NST; ++s) mbar_inval(&hbar[s]);
        }
        if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return;

        // ---- P2b: V and dV/dxi per walker, one CTA per walker (thread
        // strides over the splits, xor tree, warps in order)
        for (int p = blockIdx.x; p < a.W; p += G) {
            const CF4 acc = cta_split_sum(a.hpart, a.hsplit, a.W, p);
            if (tid == 0) emit_cf(p, acc, a.hout);
        }
    } else {
        // ---- P2: harmonic windows or the grid, one thread per walker (the
        // grid read corner by corner: few registers)
        for (int p = blockIdx.x * WK_T + tid; p < a.W; p += G * WK_T) {
            if (a.bias == 1) {
                harmonic_point<float>(a.d, a.hk, a.hper, a.xi + p * 4, a.hcen + p * 4, a.hout.V + p, a.hout.dV + p * 4,
                                      mode == 0 ? a.hsum + p * 4 : nullptr);
                if (mode == 0 && p == 0) a.hsum[a.W * 4] += 1.0;
            } else {
                double x[D], v, gr[D];
#pragma unroll
                for (int q = 0; q < D; ++q) x[q] = a.xi[p * 4 + q];
                grid_point<D, false>(a.g, a.grid, x, v, gr);
                a.hout.V[p] = (float)v;
#pragma unroll
                for (int q = 0; q < D; ++q) a.hout.dV[p * 4 + q] = (float)gr[q];
            }
        }
    }
    if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return;

    // ---- P3: deposition (CTA 0), bias force and closing kick
    if (mode == 0 && blockIdx.x == 0)
        deposit_block<float>(a.dep, a.xi, a.hout.V, a.count, a.step, a.depw, a.ctrw, a.h64, a.h32, a.status);
    for (long long i = (long long)blockIdx.x * WK_T + tid; i < a.N; i += (long long)G * WK_T) {
        const int w = a.aw[i];
        float4 F = a.f[i];
        if (a.cv_coord >= 0) {
            const float g = a.hout.dV[w * 4 + a.cv_coord];
            const float4 j = a.J[(size_t)a.cv_coord * a.N + i];
            F.x -= g * j.x;
            F.y -= g * j.y;
            F.z -= g * j.z;
        }
        if (a.cv_rg >= 0) {
            const float g = a.hout.dV[w * 4 + a.cv_rg];
            const float4 c = a.rgc[w], o = a.rgc[a.W + w];
            const float4 p = a.x[i];
            float ux = p.x - o.x, uy = p.y - o.y, uz = p.z - o.z;
            if constexpr (PER) {
                ux = min_image<float>(ux, a.box, 0);
                uy = min_image<float>(uy, a.box, 1);
                uz = min_image<float>(uz, a.box, 2);
            }
            F.x -= g * c.w * (ux - c.x);
            F.y -= g * c.w * (uy - c.y);
            F.z -= g * c.w * (uz - c.z);
        }
        a.f[i] = F;
        if (mode == 0) {
            float4 v = a.v[i];
            v.x += a.half * a.inv_m * F.x;
            v.y += a.half * a.inv_m * F.y;
            v.z += a.half * a.inv_m * F.z;
            a.v[i] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using WkKernel = void (*)(WkArgs, int);

// n = 6 (h = 3) gets a kernel with the exponent fixed at compile time
// (and no cap on y^h: with r0 >= 1e-2 the padding point's y^3 stays below
// FP32's range); a periodic box gets the minimum-image kernels.
template <bool PER> static WkKernel wk_kernel_t(int d, bool h3)
{
    if (d == 1) return h3 ? walkers_step_kernel<1, 3, PER> : walkers_step_kernel<1, 0, PER>;
    return h3 ? walkers_step_kernel<2, 3, PER> : walkers_step_kernel<2, 0, PER>;
}

static WkKernel wk_kernel(const wtmd_t* h)
{
    bool h3 = true;
    for (int c = 0; c < h->d; ++c)
        if (h->cv[c].kind == WTMD_CV_COORDINATION) h3 = h->cv[c].nn == 6 && h->cv[c].r0 >= 1e-2;
    const bool per = h->cfg.box[0] > 0.0 || h->cfg.box[1] > 0.0 || h->cfg.box[2] > 0.0;
    return per ? wk_kernel_t<true>(h->d, h3) : wk_kernel_t<false>(h->d, h3);
}

static size_t wk_smem_bytes(const wtmd_t* h)
{
    return sizeof(float4) * NST * 2 * CHUNK + 128 + sizeof(float4) * (size_t)(h->max_wn + 1);
}

static int wk_build(wtmd_t* h, int T, int bps, int hsplit_mult)
{
    WalkerPlan& k = h->wk;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = wk_smem_bytes(h);
    const void* fn = (const void*)wk_kernel(h);
    WTMD_CUDA_TRY(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int occ = 0;
    WTMD_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, WK_T, sm));
    if (occ < 1) {
        h->err = "persistent walker kernel does not fit on an SM";
        return WTMD_EINVAL;
    }
    bps = std::max(1, std::min(bps, occ));
    // tasks, sorted by cost
    std::vector<int4> tasks;
    std::vector<int> tbase(h->W), tcount(h->W);
    int slot = 0;
    for (int w = 0; w < h->W; ++w) {
        const int n = (int)h->wn_h[w];
        tbase[w] = slot;
        const int tw = wk_targets(n, T);
        tcount[w] = (n + tw - 1) / tw;
        for (int q = 0; q < tcount[w]; ++q) tasks.push_back(make_int4(w, q * tw, std::min(n, (q + 1) * tw), q));
        slot += tcount[w];
    }
    std::stable_sort(tasks.begin(), tasks.end(), [&](const int4& x, const int4& y) {
        return (long long)(x.z - x.y) * h->wn_h[x.x] > (long long)(y.z - y.y) * h->wn_h[y.x];
    });
    cudaFree(k.tasks);
    cudaFree(k.tbase);
    cudaFree(k.tcount);
    cudaFree(k.tpart);
    k.tasks = nullptr;
    k.tbase = k.tcount = nullptr;
    k.tpart = nullptr;
    WTMD_CUDA_TRY(h, cudaMalloc(&k.tasks, sizeof(int4) * tasks.size()));
    WTMD_CUDA_TRY(h, cudaMalloc(&k.tbase, sizeof(int) * h->W));
    WTMD_CUDA_TRY(h, cudaMalloc(&k.tcount, sizeof(int) * h->W));
    WTMD_CUDA_TRY(h, cudaMalloc(&k.tpart, sizeof(double) * 5 * slot));
    WTMD_CUDA_TRY(h, cudaMemcpy(k.tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemcpy(k.tbase, tbase.data(), sizeof(int) * h->W, cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemcpy(k.tcount, tcount.data(), sizeof(int) * h->W, cudaMemcpyHostToDevice));
    if (!k.ticket) {
        WTMD_CUDA_TRY(h, cudaMalloc(&k.ticket, sizeof(unsigned) * h->W));
        WTMD_CUDA_TRY(h, cudaMemset(k.ticket, 0, sizeof(unsigned) * h->W));
        WTMD_CUDA_TRY(h, cudaMalloc(&k.rgc, sizeof(float4) * 2 * h->W));
        WTMD_CUDA_TRY(h, cudaMalloc(&k.bar, sizeof(unsigned) * 4));  // count, generation, task queue, spare
        WTMD_CUDA_TRY(h, cudaMemset(k.bar, 0, sizeof(unsigned) * 4));
    }
    k.T = T;
    k.bps = bps;
    k.grid = bps * sms;
    k.ntasks = (int)tasks.size();
    k.hsplit = std::max(1, std::min(hsplit_mult * k.grid, (int)((h->cap_pairs + CHUNK - 1) / CHUNK)));
    const size_t need = (size_t)k.hsplit * h->W * sizeof(dbl4);
    if (need > h->partial_bytes) {
        cudaFree(h->partial);
        h->partial = nullptr;
        h->partial_bytes = 0;
        WTMD_CUDA_TRY(h, cudaMalloc(&h->partial, need));
        h->partial_bytes = need;
    }
    k.smem = wk_smem_bytes(h);
    return WTMD_OK;
}

int walkers_enable(wtmd_t* h)
{
    if (h->prec != WTMD_F32 || h->cfg.engine != WTMD_ENGINE_LJ) {
        h->err = "persistent walkers need an FP32 handle with the LJ engine";
        return WTMD_EINVAL;
    }
    if (h->ncv != h->d || h->d > 2) {
        h->err = "persistent walkers need 1 or 2 CVs, all defined";
        return WTMD_EINVAL;
    }
    int nco = 0, nrg = 0;
    for (int c = 0; c < h->d; ++c) {
        const CvDev& cv = h->cv[c];
        const bool co = cv.kind == WTMD_CV_COORDINATION && cv.n_a < 0 && cv.n_b < 0;
        const bool rg = cv.kind == WTMD_CV_RG && cv.n_a < 0;
        if (!(co || rg) || cv.period > 0.0) {
            h->err = "persistent walkers support coordination (all atoms) and Rg (all atoms)";
            return WTMD_EINVAL;
        }
        nco += co;
        nrg += rg;
    }
    if (nco > 1 || nrg > 1) {
        h->err = "at most one coordination and one Rg CV";
        return WTMD_EINVAL;
    }
    if (h->max_wn > 8192) {
        h->err = "walkers above 8192 atoms do not fit the staged-positions design";
        return WTMD_EINVAL;
    }
    if (surrogate_k0(h)) {
        h->err = "turn the surrogate off before the persistent walker step";
        return WTMD_EINVAL;
    }
    const int T = h->wk.T ? h->wk.T : 128, bps = h->wk.bps ? h->wk.bps : 2, hm = h->wk.hsplit_mult ? h->wk.hsplit_mult : 1;
    h->wk.hsplit_mult = hm;
    const int rc = wk_build(h, T, bps, hm);
    if (rc) return rc;
    h->persistent = true;
    return WTMD_OK;
}

int launch_walkers_step(wtmd_t* h, int mode)
{
    const WalkerPlan& k = h->wk;
    WkArgs a{};
    a.W = h->W;
    a.N = h->N;
    a.woff = h->woff;
    a.wn = h->wn;
    a.aw = h->atom_walker;
    a.tasks = k.tasks;
    a.ntasks = k.ntasks;
    a.T = k.T;
    a.tbase = k.tbase;
    a.tcount = k.tcount;
    a.tpart = k.tpart;
    a.ticket = k.ticket;
    a.rgc = k.rgc;
    a.x = (float4*)h->pos;
    a.v = (float4*)h->vel;
    a.f = (float4*)h->force;
    const wtmd_config& c = h->cfg;
    a.rc2 = (float)(c.lj_rc * c.lj_rc);
    a.sig2 = (float)(c.lj_sigma * c.lj_sigma);
    a.eps24 = (float)(24.0 * c.lj_eps);
    const double c1 = exp(-c.friction * c.dt);
    a.half = (float)(0.5 * c.dt);
    a.inv_m = (float)(1.0 / c.mass);
    a.c1 = (float)c1;
    a.c2 = (float)sqrt((1.0 - c1 * c1) * c.kT / c.mass);
    a.seed = c.seed;
    a.step = h->step;
    a.d = h->d;
    a.cv_coord = a.cv_rg = -1;
    for (int q = 0; q < h->d; ++q) {
        const CvDev& cv = h->cv[q];
        if (cv.kind == WTMD_CV_COORDINATION) {
            a.cv_coord = q;
            a.inv_r0sq = (float)(1.0 / (cv.r0 * cv.r0));
            a.hpow = cv.nn / 2;
            a.coord_scw = cv.scw;
        } else {
            a.cv_rg = q;
            a.rg_scale = cv.scale;
            a.rg_intensive = cv.flags & WTMD_CV_INTENSIVE;
        }
    }
    a.J = (float4*)h->J;
    a.xi = h->xi;
    a.hp = h->hills32;
    a.cnt = h->count;
    a.ctr = h->ctr;
    for (int q = 0; q < 3; ++q) {
        a.hprm.a[q] = h->a[q];
        a.hprm.per[q] = 0.f;
        a.hprm.iper[q] = 0.f;
    }
    a.hpart = (dbl4*)h->partial;
    a.hsplit = k.hsplit;
    a.hout.V = (float*)h->V;
    a.hout.dV = (float*)h->dV;
    a.hout.dvs = 4;
    a.hout.D = h->d;
    for (int q = 0; q < 3; ++q) {
        a.hout.gs[q] = -2.0 * 0.69314718055994530942 * h->a[q];
        a.hout.gsf[q] = (float)a.hout.gs[q];
    }
    a.hout.ticket = nullptr;
    a.hout.status = h->status;
    a.dep = dep_prm(h);  // harmonic windows deposit nothing
    a.count = h->count;
    a.depw = h->dep;
    a.ctrw = h->ctr;
    a.h64 = (dbl4*)h->hills64;
    a.h32 = (float*)h->hills32;
    a.bar = k.bar;
    a.status = h->status;
    a.max_wn = h->max_wn;
    a.wait_limit = h->wait_limit > 0 ? h->wait_limit : kWaitLimit;
    a.box = h->box;
    a.bias = h->bias_harm ? 1 : (h->bias_grid ? 2 : 0);
    a.hcen = h->harm_centre;
    a.hsum = h->harm_sum;
    for (int q = 0; q < 3; ++q) {
        a.hk[q] = h->harm_k[q];
        a.hper[q] = q < h->d ? h->cv[q].period : 0.0;
    }
    if (h->grid) a.g = grid_prm(h);
    a.grid = h->grid;
    // barrier counter, generation and task queue start clean on every launch
    // (a timed-out barrier would leave its counter dirty)
    WTMD_CUDA_TRY(h, cudaMemsetAsync(k.bar, 0, sizeof(unsigned) * 4, h->stream));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(k.grid);
    cfg.blockDim = dim3(WK_T);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, wk_kernel(h), a, mode);
    if (e != cudaSuccess) {
        h->err = std::string("persistent walker launch: ") + cudaGetErrorString(e);
        return WTMD_ECUDA;
    }
    mark(h, "walkers_step");
    if (mode == 0 && h->grid) return launch_grid_update(h);
    return WTMD_OK;
}

int walkers_retile(wtmd_t* h, int T, int bps, int hsplit_mult)
{
    h->wk.hsplit_mult = hsplit_mult;
    return wk_build(h, T, bps, hsplit_mult);
}

}  // namespace wtmd
