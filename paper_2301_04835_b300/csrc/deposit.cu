// Hill deposition of metadynamics with optional grid storage of the bias, and
// the free-energy estimate (PySAGES paper, Sec. 2.1.5; Sec. 2 `analyze`;
// Sec. 2.1, Eq. (free-energy)).
//
// Every `stride` steps each walker appends one hill at its current CVs.  The
// height is w0 in standard metadynamics and, in the well-tempered variant,
// w0 exp(-V(s) / (kT (gamma - 1))) with V(s) the bias of the hills that
// existed before this step's deposits (the same V the force used); it is
// computed in FP64.  Walkers append in index order.  The FP64 grid holds the
// running bias at cell centres; each new Gaussian is added as a product of
// per-axis factors exp(-D_i^2/(2 sigma_i^2)) (periodic axes use the minimum
// image), which needs sum(bins) exponentials per hill instead of prod(bins).
#include <algorithm>

#include "step_dev.cuh"

namespace wtmd {

void store_hills32_range(wtmd_t* h, long long k0, long long k1);

template <typename R>
__global__ void __launch_bounds__(256) deposit_kernel(DepPrm p, const double* __restrict__ xi,
                                                      const R* __restrict__ V, long long* __restrict__ count,
                                                      long long* __restrict__ step, long long* __restrict__ dep,
                                                      double* __restrict__ ctr, dbl4* __restrict__ h64,
                                                      float* __restrict__ h32, unsigned* status)
{
    deposit_block<R>(p, xi, V, count, step, dep, ctr, h64, h32, status);
}

__global__ void grid_factor_kernel(GridPrm g, const long long* __restrict__ dep, const dbl4* __restrict__ h64,
                                   int tot, double* __restrict__ fac)
{
    grid_factors(g, dep, h64, tot, fac, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x);
}

__global__ void grid_add_kernel(GridPrm g, const long long* __restrict__ dep, const dbl4* __restrict__ h64, int tot,
                                const double* __restrict__ fac, long long ncell, double* __restrict__ grid)
{
    grid_add(g, dep, h64, tot, fac, ncell, grid, (long long)blockIdx.x * blockDim.x + threadIdx.x,
             (long long)gridDim.x * blockDim.x);
}

// Rebuild the grid from all hills (after a hill-list load).
__global__ void grid_rebuild_kernel(GridPrm g, const dbl4* __restrict__ h64, long long H, long long ncell,
                                    double* __restrict__ grid)
{
    for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < ncell;
         cidx += (long long)gridDim.x * blockDim.x) {
        double x[3] = {0, 0, 0};
        long long rem = cidx;
        for (int i = g.d - 1; i >= 0; --i) {
            const int k = (int)(rem % g.bins[i]);
            rem /= g.bins[i];
            x[i] = g.lo[i] + (k + 0.5) * g.dx[i];
        }
        double v = 0.0;
        for (long long n = 0; n < H; ++n) {
            const dbl4 h = h64[n];
            const double s[3] = {h.x, h.y, h.z};
            double e = h.w;
            for (int i = 0; i < g.d; ++i) {
                double D = x[i] - s[i];
                if (g.per[i] > 0.0) D -= g.per[i] * rint(D / g.per[i]);
                e *= exp(-D * D * g.inv2s2[i]);
            }
            v += e;
        }
        grid[cidx] = v;
    }
}

__global__ void __launch_bounds__(1024) grid_max_kernel(const double* __restrict__ grid, long long n,
                                                        double* __restrict__ out)
{
    __shared__ double sm[32];
    double m = -INFINITY;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, grid[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) sm[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmax(r, sm[w]);
        out[0] = r;
    }
}

__global__ void fes_kernel(const double* __restrict__ grid, long long n, double f, const double* __restrict__ vmax,
                           double* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // f < 0: the minimum of f*V is f*max(V)
    out[i] = f * grid[i] - f * vmax[0];
}

// Bias and gradient read from the grid at P points (grid_point, one thread
// per point, FP64 throughout; the result is rounded to R on the store).
// The point's corner nodes and their neighbours (at most 56 doubles) are
// L2-resident reads: the kernel is bound by its launch, not by memory.
template <int D, typename X, typename R>
__global__ void __launch_bounds__(128) grid_bias_kernel(GridPrm g, const double* __restrict__ grid,
                                                        const X* __restrict__ xi, int xs, long long P,
                                                        R* __restrict__ V, R* __restrict__ dV, int dvs)
{
    // launched as a programmatic dependent of the CV kernel in a step: every
    // read (xi, grid) comes after the wait; dependents may launch at once, as
    // their own wait covers this kernel's completion
    pdl_wait();
    pdl_trigger();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double x[D], v, gr[D];
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = (double)xi[p * xs + i];
    grid_point<D>(g, grid, x, v, gr);
    if (V) V[p] = (R)v;
    if (dV)
#pragma unroll
        for (int i = 0; i < D; ++i) dV[p * dvs + i] = (R)gr[i];
}

// ---------------------------------------------------------------------------
GridPrm grid_prm(const wtmd_t* h)
{
    GridPrm g{};
    g.d = h->d;
    int off = 0;
    for (int i = 0; i < 3; ++i) {
        g.bins[i] = i < h->d ? h->cfg.grid_bins[i] : 1;
        g.off[i] = off;
        if (i < h->d) off += h->cfg.grid_bins[i];
        g.lo[i] = h->cfg.grid_lo[i];
        g.dx[i] = i < h->d ? (h->cfg.grid_hi[i] - h->cfg.grid_lo[i]) / h->cfg.grid_bins[i] : 1.0;
        const double sg = h->cfg.sigma[i] > 0 ? h->cfg.sigma[i] : 1.0;
        g.inv2s2[i] = 1.0 / (2.0 * sg * sg);
        g.per[i] = i < h->d ? h->cv[i].period : 0.0;
    }
    return g;
}

static double fes_factor(const wtmd_config& c)
{
    return (c.gamma == 0.0 || isinf(c.gamma)) ? -1.0 : -c.gamma / (c.gamma - 1.0);
}

DepPrm dep_prm(const wtmd_t* h)
{
    DepPrm p{};
    p.stride = h->bias_harm ? 0 : h->cfg.stride;  // umbrella windows deposit no hills
    p.cap = h->cap;
    p.W = h->W;
    p.d = h->d;
    p.w0 = h->cfg.w0;
    p.inv_dT = (h->cfg.gamma == 0.0 || isinf(h->cfg.gamma)) ? 0.0 : 1.0 / (h->cfg.kT * (h->cfg.gamma - 1.0));
    for (int i = 0; i < 3; ++i) p.a[i] = h->a[i];
    return p;
}

int launch_deposit(wtmd_t* h)
{
    const DepPrm p = dep_prm(h);
    if (h->prec == WTMD_F32)
        deposit_kernel<float><<<1, 256, 0, h->stream>>>(p, h->xi, (const float*)h->V, h->count, h->step, h->dep,
                                                        h->ctr, (dbl4*)h->hills64, (float*)h->hills32, h->status);
    else
        deposit_kernel<double><<<1, 256, 0, h->stream>>>(p, h->xi, (const double*)h->V, h->count, h->step, h->dep,
                                                         h->ctr, (dbl4*)h->hills64, (float*)h->hills32, h->status);
    mark(h, "deposit");
    return launch_grid_update(h);
}

int launch_grid_update(wtmd_t* h)
{
    if (h->grid) {
        GridPrm g = grid_prm(h);
        const int tot = h->gbins_sum;
        const long long nf = (long long)h->W * tot;
        grid_factor_kernel<<<(unsigned)std::min<long long>((nf + 255) / 256, 4096), 256, 0, h->stream>>>(
            g, h->dep, (const dbl4*)h->hills64, tot, h->gfac);
        mark(h, "grid_factor");
        grid_add_kernel<<<(unsigned)std::min<long long>((h->ncell + 255) / 256, 8192), 256, 0, h->stream>>>(
            g, h->dep, (const dbl4*)h->hills64, tot, h->gfac, h->ncell, h->grid);
        mark(h, "grid_add");
    }
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

int launch_grid_rebuild(wtmd_t* h)
{
    if (!h->grid) return WTMD_OK;
    long long H = 0;
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(&H, h->count, sizeof(H), cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    GridPrm g = grid_prm(h);
    grid_rebuild_kernel<<<(unsigned)std::min<long long>((h->ncell + 255) / 256, 8192), 256, 0, h->stream>>>(
        g, (const dbl4*)h->hills64, H, h->ncell, h->grid);
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

int launch_fes(wtmd_t* h, double* out)
{
    double* vmax = (double*)h->gfac;  // any scratch double; the factor table is idle here
    grid_max_kernel<<<1, 1024, 0, h->stream>>>(h->grid, h->ncell, vmax);
    fes_kernel<<<(unsigned)((h->ncell + 255) / 256), 256, 0, h->stream>>>(h->grid, h->ncell, fes_factor(h->cfg), vmax,
                                                                          out);
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

// Harmonic biasing of every walker about its window centre (harmonic_point,
// Sec. 2.1.1 / 2.1.2).  In a step the kernel also adds each walker's xi to
// its window sums (FP64) and counts the sample.  One thread per walker.
struct HarmPrm {
    int W, d;
    double k[3], per[3];
};

template <typename R>
__global__ void harmonic_bias_kernel(HarmPrm hp, const double* __restrict__ xi, const double* __restrict__ centre,
                                     R* __restrict__ V, R* __restrict__ dV, double* __restrict__ sum)
{
    pdl_wait();  // xi comes from the CV kernel this launch depends on
    pdl_trigger();
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= hp.W) return;
    harmonic_point<R>(hp.d, hp.k, hp.per, xi + w * 4, centre + w * 4, V + w, dV + w * 4, sum ? sum + w * 4 : nullptr);
    if (sum && w == 0) sum[hp.W * 4] += 1.0;
}

int launch_harmonic(wtmd_t* h, bool accumulate)
{
    HarmPrm hp{};
    hp.W = h->W;
    hp.d = h->d;
    for (int c = 0; c < 3; ++c) {
        hp.k[c] = h->harm_k[c];
        hp.per[c] = c < h->d ? h->cv[c].period : 0.0;
    }
    double* sum = accumulate ? h->harm_sum : nullptr;
    const dim3 blocks((unsigned)((h->W + 127) / 128)), threads(128);
    cudaError_t e;
    if (h->prec == WTMD_F32)
        e = launch_pdl(harmonic_bias_kernel<float>, blocks, threads, 0, h->stream, hp, (const double*)h->xi,
                       (const double*)h->harm_centre, (float*)h->V, (float*)h->dV, sum);
    else
        e = launch_pdl(harmonic_bias_kernel<double>, blocks, threads, 0, h->stream, hp, (const double*)h->xi,
                       (const double*)h->harm_centre, (double*)h->V, (double*)h->dV, sum);
    mark(h, "harmonic_bias");
    WTMD_CUDA_TRY(h, e);
    return WTMD_OK;
}

template <typename X, typename R>
static cudaError_t grid_bias_go(wtmd_t* h, const GridPrm& g, const X* xi, int xs, long long P, R* V, R* dV, int dvs,
                                bool pdl)
{
    const dim3 blocks((unsigned)((P + 127) / 128)), threads(128);
    auto k = g.d == 1 ? grid_bias_kernel<1, X, R> : (g.d == 2 ? grid_bias_kernel<2, X, R> : grid_bias_kernel<3, X, R>);
    if (pdl) return launch_pdl(k, blocks, threads, 0, h->stream, g, (const double*)h->grid, xi, xs, P, V, dV, dvs);
    k<<<blocks, threads, 0, h->stream>>>(g, h->grid, xi, xs, P, V, dV, dvs);
    return cudaGetLastError();
}

int launch_grid_bias(wtmd_t* h, const void* xi, bool xi_f64, int xs, int64_t P, void* V, void* dV, int dvs, bool pdl)
{
    if (P <= 0) return WTMD_OK;
    const GridPrm g = grid_prm(h);
    cudaError_t e;
    if (h->prec == WTMD_F32) {
        if (xi_f64)
            e = grid_bias_go(h, g, (const double*)xi, xs, (long long)P, (float*)V, (float*)dV, dvs, pdl);
        else
            e = grid_bias_go(h, g, (const float*)xi, xs, (long long)P, (float*)V, (float*)dV, dvs, pdl);
    } else {
        e = grid_bias_go(h, g, (const double*)xi, xs, (long long)P, (double*)V, (double*)dV, dvs, pdl);
    }
    mark(h, "grid_bias");
    WTMD_CUDA_TRY(h, e);
    return WTMD_OK;
}

}  // namespace wtmd
