// Small systems in one CTA: whole MD steps of an FP64 handle whose walkers
// are a few particles on an analytic landscape (Mueller-Brown, three wells)
// with component CVs, many steps per launch.
//
// Such a step is a handful of tiny operations (a BAOAB half step and an
// analytic force per particle, one CV read per walker, the bias at each
// walker's CVs, the deposit, a kick), so the per-kernel step is a chain of
// launch latencies.  Here one CTA runs the steps in a loop with a barrier
// between the phases -- the same operations in the same order as the
// per-kernel step (Sec. 3.2.1 steps (a)-(f) with the metadynamics update of
// Sec. 2.1.5):
//   B-A-O-A for every particle (baoab_first_atom, the same Philox stream);
//   the engine force and the walkers' component CVs;
//   the bias at each walker's CVs from the handle's source: the FP64 hills
//   sum (threads stride the hills, a fixed-order block reduction per walker),
//   the FP64 grid read (grid_point) or the harmonic window (harmonic_point,
//   window sums accumulated);
//   deposition (deposit_block), the grid update after a deposit
//   (grid_factors, grid_add) and the bias force -J^T dV/dxi with the closing
//   half kick.
// No waits on other CTAs or kernels: the only synchronization is the CTA's
// own barrier.
#include "analytic_dev.cuh"
#include "step_dev.cuh"

namespace wtmd {

constexpr int SMS_T = 512;              // threads of the CTA
constexpr int SMS_MAX_N = SMS_T;        // particles of the handle (one per thread)
constexpr int SMS_MAX_W = 256;          // walkers
constexpr size_t SMS_NOISE_BYTES = 96 * 1024;  // deviates drawn ahead: K steps x N particles x 3 doubles
constexpr int SMS_MAX_W_HILLS = 16;     // walkers with the hills source (one block reduction each)
constexpr long long SMS_MAX_HILLS = 2048; // hill capacity with the hills source: one SM's FP64 pipe takes
                                         // ~13 cycles a hill, the per-kernel step is faster beyond ~3e3
constexpr long long SMS_CHUNK = 65536;  // steps per launch

struct SmallArgs {
    long long N;
    int W, d, dims, engine;
    const int64_t* woff;
    const int* aw;
    dbl4* x;
    dbl4* v;
    dbl4* f;
    uint64_t seed;
    double half, inv_m, c1, c2, hdm;  // hdm = dt / (2 m)
    long long* step;
    int cidx[3], caxis[3];
    double cscale[3];
    double* xi;  // [W][4]
    double* V;   // [W]
    double* dV;  // [W][4]
    int bias;    // 0 hills, 1 harmonic windows, 2 grid
    const dbl4* hills;
    double inv2s2[3], hper[3], gs[3];
    const double* hcen;
    double* hsum;
    double hk[3], wper[3];
    GridPrm g;
    double* grid;
    double* gfac;
    int gtot;
    long long ncell;
    DepPrm dep;
    long long* count;
    long long* depw;
    double* ctr;
    dbl4* h64;
    float* h32;
    unsigned* status;
};

// Each thread owns one particle (x, v, f stay in its registers for the whole
// launch); the walkers' CVs, V and dV/dxi, the hill count and the step live
// in shared memory, and the normal deviates of the next K steps are drawn
// ahead by all threads at once (the same Philox values the per-kernel step
// draws one at a time), so a step waits on no global memory round trip.
template <int D>
__global__ void __launch_bounds__(SMS_T) small_step_kernel(SmallArgs a, long long nsteps, int K)
{
    extern __shared__ double noise_s[];  // [K][N][3]
    __shared__ double xi_s[SMS_MAX_W * 4], V_s[SMS_MAX_W], dV_s[SMS_MAX_W * 4];
    __shared__ double red[SMS_T / 32][4];
    __shared__ double ctr_s[3];
    __shared__ long long cnt_s, dep_s[2];
    __shared__ int doit_s;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int N = (int)a.N;
    const bool own = tid < N;
    dbl4 x = dbl4{0.0, 0.0, 0.0, 0.0}, v = x, f = x;
    int w_own = 0, li = 0;
    if (own) {
        x = a.x[tid];
        v = a.v[tid];
        f = a.f[tid];
        w_own = a.aw[tid];
        li = tid - (int)a.woff[w_own];
    }
    const long long t0 = *a.step;
    if (tid == 0) {
        cnt_s = *a.count;
        for (int q = 0; q < 3; ++q) ctr_s[q] = a.ctr[q];
    }
    __syncthreads();
    for (long long s = 0; s < nsteps; ++s) {
        const long long t = t0 + s;
        const int ks = (int)(s % K);
        if (ks == 0) {  // deviates of steps t .. t + K - 1
            for (int q = tid; q < K * N; q += SMS_T) {
                const int k = q / N, i = q % N;
                const Normal3<double> n = noise3<double>(a.seed, t + k, (uint32_t)i);
                double* o = noise_s + 3 * (size_t)q;
                o[0] = n.g[0];
                o[1] = n.g[1];
                o[2] = n.g[2];
            }
            __syncthreads();
        }
        // B-A-O-A, the engine force and this particle's component CVs
        if (own) {
            baoa_update<double>(x, v, f, noise_s + 3 * ((size_t)ks * N + tid), a.half, a.inv_m, a.c1, a.c2, a.dims);
            f = a.engine == WTMD_ENGINE_MB ? mb_force<double>(x) : wells3_force<double>(x);
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (li == a.cidx[c]) xi_s[w_own * 4 + c] = a.cscale[c] * (a.caxis[c] == 0 ? x.x : (a.caxis[c] == 1 ? x.y : x.z));
        }
        __syncthreads();
        // the bias at every walker's CVs
        if (a.bias == 0) {
            const long long H = cnt_s;
            for (int w = 0; w < a.W; ++w) {
                double xw[D];
#pragma unroll
                for (int c = 0; c < D; ++c) xw[c] = xi_s[w * 4 + c];
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                for (long long k = tid; k < H; k += SMS_T) {
                    const dbl4 hk = a.hills[k];
                    const double sk[3] = {hk.x, hk.y, hk.z};
                    double dd[D], q = 0.0;
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        double di = xw[c] - sk[c];
                        if (a.hper[c] > 0.0) di -= a.hper[c] * rint(di / a.hper[c]);
                        dd[c] = di;
                        q += di * di * a.inv2s2[c];
                    }
                    const double e = hk.w * exp(-q);
                    acc[0] += e;
#pragma unroll
                    for (int c = 0; c < D; ++c) acc[1 + c] += e * dd[c];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                if (lane == 0)
                    for (int q = 0; q < 4; ++q) red[warp][q] = acc[q];
                __syncthreads();
                if (warp == 0) {  // the warps' sums by a fixed xor tree
                    double t4[4];
                    for (int q = 0; q < 4; ++q) t4[q] = lane < SMS_T / 32 ? red[lane][q] : 0.0;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        for (int o = SMS_T / 64; o > 0; o >>= 1) t4[q] += __shfl_xor_sync(0xffffffffu, t4[q], o);
                    if (lane == 0) {
                        bool ok = isfinite(t4[0]);
                        V_s[w] = t4[0];
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            const double g = a.gs[c] * t4[1 + c];
                            ok = ok && isfinite(g);
                            dV_s[w * 4 + c] = g;
                        }
                        if (!ok) atomicOr(a.status, ST_NUMERIC);
                    }
                }
                __syncthreads();  // red[] is refilled for the next walker
            }
        } else {
            for (int w = tid; w < a.W; w += SMS_T) {
                if (a.bias == 1) {
                    harmonic_point<double>(D, a.hk, a.wper, xi_s + w * 4, a.hcen + w * 4, V_s + w, dV_s + w * 4,
                                           a.hsum + w * 4);
                    if (w == 0) a.hsum[a.W * 4] += 1.0;
                } else {
                    double xw[D], vv = 0.0, gr[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) xw[c] = xi_s[w * 4 + c];
                    grid_point<D, false>(a.g, a.grid, xw, vv, gr);
                    V_s[w] = vv;
#pragma unroll
                    for (int c = 0; c < D; ++c) dV_s[w * 4 + c] = gr[c];
                }
            }
        }
        // deposition after steps t with (t + 1) % stride == 0 (as
        // deposit_block, with the count and the centre in shared memory)
        if (tid == 0) {
            int doit = a.dep.stride > 0 && (t + 1) % a.dep.stride == 0;
            const long long base = cnt_s;
            if (doit && base + a.W > a.dep.cap) {
                atomicOr(a.status, ST_CAPACITY);
                doit = 0;
            }
            dep_s[0] = base;
            dep_s[1] = doit ? a.W : 0;
            if (doit && isnan(ctr_s[0]))
                for (int q = 0; q < 3; ++q) a.ctr[q] = ctr_s[q] = q < D ? xi_s[q] : 0.0;
            doit_s = doit;
        }
        __syncthreads();
        if (doit_s) {
            const long long base = dep_s[0];
            for (int w = tid; w < a.W; w += SMS_T) {
                const long long k = base + w;
                double sv[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int c = 0; c < D; ++c) sv[c] = xi_s[w * 4 + c];
                const double hgt = a.dep.w0 * exp(-V_s[w] * a.dep.inv_dT);
                a.h64[k] = dbl4{sv[0], sv[1], sv[2], hgt};
                const long long b = (k >> 1) * 8 + (k & 1);
                a.h32[b + 0] = (float)(-(sv[0] - ctr_s[0]) * a.dep.a[0]);
                a.h32[b + 2] = (float)(-(sv[1] - ctr_s[1]) * a.dep.a[1]);
                a.h32[b + 4] = (float)(-(sv[2] - ctr_s[2]) * a.dep.a[2]);
                a.h32[b + 6] = (float)(-log2(hgt));
            }
            __syncthreads();
            if (a.grid) {
                grid_factors(a.g, dep_s, a.h64, a.gtot, a.gfac, tid, SMS_T);
                __syncthreads();
                grid_add(a.g, dep_s, a.h64, a.gtot, a.gfac, a.ncell, a.grid, tid, SMS_T);
            }
            if (tid == 0) cnt_s = dep_s[0] + a.W;
        }
        // bias force -J^T dV/dxi and the closing half kick
        if (own) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double g = dV_s[w_own * 4 + c];
                const bool mine = li == a.cidx[c];
                const double jx = mine && a.caxis[c] == 0 ? a.cscale[c] : 0.0;
                const double jy = mine && a.caxis[c] == 1 ? a.cscale[c] : 0.0;
                const double jz = mine && a.caxis[c] == 2 ? a.cscale[c] : 0.0;
                f.x -= g * jx;
                f.y -= g * jy;
                f.z -= g * jz;
            }
            v.x += a.hdm * f.x;
            v.y += a.hdm * f.y;
            if (a.dims > 2) v.z += a.hdm * f.z;
        }
        __syncthreads();  // xi_s, V_s, dV_s and the count are rewritten by the next step
    }
    // the state, the last step's CVs and bias, the counters
    if (own) {
        a.x[tid] = x;
        a.v[tid] = v;
        a.f[tid] = f;
    }
    for (int q = tid; q < a.W * 4; q += SMS_T) {
        if (q % 4 < D) {
            a.xi[q] = xi_s[q];
            a.dV[q] = dV_s[q];
        }
        if (q % 4 == 0) a.V[q / 4] = V_s[q / 4];
    }
    if (tid == 0) {
        *a.step = t0 + nsteps;
        *a.count = cnt_s;
        a.depw[0] = dep_s[0];
        a.depw[1] = dep_s[1];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool small_step_eligible(const wtmd_t* h)
{
    if (!h->small_on || h->prec != WTMD_F64 || h->persistent || surrogate_k0(h)) return false;
    if (h->cfg.engine != WTMD_ENGINE_MB && h->cfg.engine != WTMD_ENGINE_WELLS3) return false;
    if (h->N > SMS_MAX_N || h->W > SMS_MAX_W || h->ncv != h->d || h->d < 1 || h->d > 3) return false;
    for (int c = 0; c < h->d; ++c)
        if (h->cv[c].kind != WTMD_CV_COMPONENT) return false;
    if (!h->bias_harm && !h->bias_grid && (h->W > SMS_MAX_W_HILLS || h->cap > SMS_MAX_HILLS)) return false;
    return true;
}

int launch_small_steps(wtmd_t* h, int64_t n_steps)
{
    SmallArgs a{};
    const wtmd_config& c = h->cfg;
    a.N = h->N;
    a.W = h->W;
    a.d = h->d;
    a.dims = c.engine == WTMD_ENGINE_MB ? 2 : 3;
    a.engine = c.engine;
    a.woff = h->woff;
    a.aw = h->atom_walker;
    a.x = (dbl4*)h->pos;
    a.v = (dbl4*)h->vel;
    a.f = (dbl4*)h->force;
    a.seed = c.seed;
    const double c1 = exp(-c.friction * c.dt);
    a.half = 0.5 * c.dt;
    a.inv_m = 1.0 / c.mass;
    a.c1 = c1;
    a.c2 = sqrt((1.0 - c1 * c1) * c.kT / c.mass);
    a.hdm = 0.5 * c.dt / c.mass;
    a.step = h->step;
    for (int q = 0; q < h->d; ++q) {
        a.cidx[q] = h->cv[q].hidx[0];
        a.caxis[q] = h->cv[q].axis;
        a.cscale[q] = h->cv[q].scale != 0.0 ? h->cv[q].scale : 1.0;
    }
    a.xi = h->xi;
    a.V = (double*)h->V;
    a.dV = (double*)h->dV;
    a.bias = h->bias_harm ? 1 : (h->bias_grid ? 2 : 0);
    a.hills = (const dbl4*)h->hills64;
    for (int q = 0; q < 3; ++q) {
        const double sg = c.sigma[q] > 0 ? c.sigma[q] : 1.0;
        a.inv2s2[q] = 1.0 / (2.0 * sg * sg);
        a.gs[q] = -1.0 / (sg * sg);
        a.hper[q] = q < h->d ? h->cv[q].period : 0.0;
        a.hk[q] = h->harm_k[q];
        a.wper[q] = a.hper[q];
    }
    a.hcen = h->harm_centre;
    a.hsum = h->harm_sum;
    if (h->grid) {
        a.g = grid_prm(h);
        a.grid = h->grid;
        a.gfac = h->gfac;
        a.gtot = h->gbins_sum;
        a.ncell = h->ncell;
    }
    a.dep = dep_prm(h);
    a.count = h->count;
    a.depw = h->dep;
    a.ctr = h->ctr;
    a.h64 = (dbl4*)h->hills64;
    a.h32 = (float*)h->hills32;
    a.status = h->status;
    // steps whose deviates are drawn at once
    const int K = (int)std::max<long long>(1, std::min<long long>(256, SMS_NOISE_BYTES / (24 * (size_t)h->N)));
    const size_t smem = (size_t)K * h->N * 3 * sizeof(double);
    auto kern = h->d == 1 ? small_step_kernel<1> : (h->d == 2 ? small_step_kernel<2> : small_step_kernel<3>);
    static bool set[64][3] = {};
    int dev = 0;
    WTMD_CUDA_TRY(h, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        h->err = "device index";
        return WTMD_ECUDA;
    }
    if (!set[dev][h->d - 1]) {
        WTMD_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMS_NOISE_BYTES));
        set[dev][h->d - 1] = true;
    }
    for (int64_t done = 0; done < n_steps;) {
        const long long k = std::min<long long>(SMS_CHUNK, n_steps - done);
        kern<<<1, SMS_T, smem, h->stream>>>(a, k, K);
        WTMD_CUDA_TRY(h, cudaGetLastError());
        mark(h, "small_step");
        done += k;
    }
    return WTMD_OK;
}

}  // namespace wtmd
