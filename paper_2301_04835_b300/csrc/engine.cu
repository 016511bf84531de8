// The minimal engine that drives the method: BAOAB Langevin integration with
// counter-based Philox noise, and three force fields (Mueller-Brown, 12-6
// Lennard-Jones with a cell list or all pairs, bead chain).  In the paper the
// backend (HOOMD-blue, OpenMM, ...) owns these steps: half-step integration,
// bonded and pair forces, second half-step (Sec. 3.2.1 steps (a), (b), (c), (f)).
//
// BAOAB (Leimkuhler & Matthews 2013): B v += dt/2 F/m; A x += dt/2 v;
// O v = c1 v + sqrt((1 - c1^2) kT/m) R, c1 = exp(-friction dt); A x += dt/2 v;
// forces; B.  The noise of particle i at step t is Philox4x32-10 with key
// (seed lo, seed hi) and counter (t lo, i, t hi, 0); its four words become
// uniforms u = (x + 1/2) 2^-32 and two Box-Muller pairs (first three normals
// used).  Positions are never wrapped; distances use the minimum image.
#include "step_dev.cuh"

namespace wtmd {

// First half of the step for every atom.  Launched as a programmatic
// dependent of the previous step's last kernel: it waits for that kernel,
// then lets the CV kernels launch.  It also zeroes the Jacobian rows given
// by jmask and the CV values given by xmask (CVs whose kernel accumulates
// them).
template <typename R>
__global__ void baoab_first_kernel(long long N, R4<R>* __restrict__ x, R4<R>* __restrict__ v,
                                   const R4<R>* __restrict__ f, const long long* __restrict__ step, uint64_t seed,
                                   R half, R inv_m, R c1, R c2, int dims, R4<R>* __restrict__ J, int jmask,
                                   double* __restrict__ xi, int xmask, int W)
{
    pdl_wait();
    pdl_trigger();  // the CV kernels that follow may launch; they wait for these positions
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < W)
        for (int c = 0; c < 3; ++c)
            if (xmask >> c & 1) xi[i * 4 + c] = 0.0;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c)
        if (jmask >> c & 1) J[(size_t)c * N + i] = mk4<R>(R(0), R(0), R(0), R(0));
    baoab_first_atom<R>(i, *step, x, v, f, seed, half, inv_m, c1, c2, dims);
}

// Mueller-Brown (Mueller & Brown 1979): sum of four anisotropic Gaussians.
__constant__ double kMB[6][4] = {
    {-200.0, -100.0, -170.0, 15.0},  // A
    {-1.0, -1.0, -6.5, 0.7},         // a
    {0.0, 0.0, 11.0, 0.6},           // b
    {-10.0, -10.0, -6.5, 0.7},       // c
    {1.0, 0.0, -0.5, -1.0},          // x0
    {0.0, 0.5, 1.5, 1.0},            // y0
};

// Three Gaussian wells in a harmonic confinement (3-D test landscape):
// U = -sum_m A_m exp(-|r - c_m|^2 / (2 s_m^2)) + (k/2) |r|^2, F = -grad U.
__constant__ double kW3[3][5] = {
    // A, s, c_x, c_y, c_z
    {8.0, 0.45, -1.0, 0.0, 0.0},
    {6.0, 0.40, 1.0, 0.2, -0.3},
    {7.0, 0.50, 0.1, 1.3, 0.6},
};
constexpr double kW3Conf = 1.5;

template <typename R>
__global__ void wells3_kernel(long long N, const R4<R>* __restrict__ x, R4<R>* __restrict__ f)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R4<R> p = x[i];
    R fx = -(R)kW3Conf * p.x, fy = -(R)kW3Conf * p.y, fz = -(R)kW3Conf * p.z;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const R dx = p.x - (R)kW3[m][2], dy = p.y - (R)kW3[m][3], dz = p.z - (R)kW3[m][4];
        const R is2 = (R)(1.0 / (kW3[m][1] * kW3[m][1]));
        const R e = (R)kW3[m][0] * exp(-(R)0.5 * (dx * dx + dy * dy + dz * dz) * is2);
        fx -= e * dx * is2;
        fy -= e * dy * is2;
        fz -= e * dz * is2;
    }
    f[i] = mk4<R>(fx, fy, fz, R(0));
}

template <typename R>
__global__ void mb_kernel(long long N, const R4<R>* __restrict__ x, R4<R>* __restrict__ f)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R4<R> p = x[i];
    R gx = 0, gy = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R dx = p.x - (R)kMB[4][k], dy = p.y - (R)kMB[5][k];
        const R a = (R)kMB[1][k], b = (R)kMB[2][k], c = (R)kMB[3][k];
        const R e = (R)kMB[0][k] * exp(a * dx * dx + b * dx * dy + c * dy * dy);
        gx += e * (R(2) * a * dx + b * dy);
        gy += e * (b * dx + R(2) * c * dy);
    }
    f[i] = mk4<R>(-gx, -gy, R(0), R(0));
}

// LJ pair force factor: F_t += fr * (r_t - r_s), fr = 24 eps (2 (s/r)^12 - (s/r)^6) / r^2.
template <typename R> __device__ __forceinline__ R inv(R x);
template <> __device__ __forceinline__ float inv<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double inv<double>(double x) { return 1.0 / x; }

template <typename R> __device__ __forceinline__ R lj_fr(R r2, R sig2, R eps24)
{
    const R ir2 = inv<R>(r2);
    const R sr2 = sig2 * ir2;
    const R sr6 = sr2 * sr2 * sr2;
    return eps24 * (R(2) * sr6 * sr6 - sr6) * ir2;
}

// All pairs within each walker; sources staged in shared memory.
template <typename R>
__global__ void __launch_bounds__(128) lj_allpairs_kernel(const R4<R>* __restrict__ x, const int64_t* __restrict__ woff,
                                                          const int* __restrict__ wn, Box box, R rc2, R sig2, R eps24,
                                                          R4<R>* __restrict__ f)
{
    __shared__ R4<R> src[128];
    const int w = blockIdx.y;
    const long long o = woff[w];
    const int n = wn[w];
    const int t = blockIdx.x * 128 + threadIdx.x;
    if (blockIdx.x * 128 >= n) return;
    R4<R> xt = t < n ? x[o + t] : mk4<R>(0, 0, 0, 0);
    R fx = 0, fy = 0, fz = 0;
    for (int s0 = 0; s0 < n; s0 += 128) {
        __syncthreads();
        if (s0 + threadIdx.x < n) src[threadIdx.x] = x[o + s0 + threadIdx.x];
        __syncthreads();
        const int m = min(128, n - s0);
        for (int j = 0; j < m; ++j) {
            if (s0 + j == t) continue;
            const R4<R> xs = src[j];
            const R dx = min_image<R>(xt.x - xs.x, box, 0);
            const R dy = min_image<R>(xt.y - xs.y, box, 1);
            const R dz = min_image<R>(xt.z - xs.z, box, 2);
            const R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2) {
                const R fr = lj_fr<R>(r2, sig2, eps24);
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
            }
        }
    }
    if (t < n) f[o + t] = mk4<R>(fx, fy, fz, R(0));
}

template <typename R> __device__ __forceinline__ R inv_box(const Box& b, int k);
template <> __device__ __forceinline__ float inv_box<float>(const Box& b, int k) { return b.invLf[k]; }
template <> __device__ __forceinline__ double inv_box<double>(const Box& b, int k) { return b.invL[k]; }

// x - m L for an integer m, with L as hi + lo floats in FP32.
template <typename R> __device__ __forceinline__ R shift_box(R x, R m, const Box& b, int k);
template <> __device__ __forceinline__ float shift_box<float>(float x, float m, const Box& b, int k)
{
    return fmaf(-m, b.Llo[k], fmaf(-m, b.Lf[k], x));
}
template <> __device__ __forceinline__ double shift_box<double>(double x, double m, const Box& b, int k)
{
    return x - m * b.L[k];
}

// Position of x in the periodic image of the home cell's frame: wrapped by
// floor(x / L) (the formula the binning uses), then moved by `img` boxes.
template <typename R> __device__ __forceinline__ R image_coord(R x, int img, const Box& b, int k)
{
    const R m = floor(x * inv_box<R>(b, k)) - (R)img;
    return shift_box<R>(x, m, b, k);
}

// Cell list (single periodic walker).  Binning with atomics, then each
// cell's list is sorted by atom index so the force sum order is fixed.
template <typename R>
__global__ void cell_bin_kernel(long long N, const R4<R>* __restrict__ x, Box box, int ncx, int ncy, int ncz,
                                int cap, int* __restrict__ cnt, int* __restrict__ atoms, unsigned* status)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R4<R> p = x[i];
    const R q[3] = {p.x, p.y, p.z};
    const int nc[3] = {ncx, ncy, ncz};
    int ci[3];
    for (int k = 0; k < 3; ++k) {
        R u = q[k] * inv_box<R>(box, k);
        u -= floor(u);  // fractional coordinate in [0, 1]
        int c = (int)(u * nc[k]);
        ci[k] = c >= nc[k] ? nc[k] - 1 : (c < 0 ? 0 : c);
    }
    const int cell = (ci[0] * ncy + ci[1]) * ncz + ci[2];
    const int slot = atomicAdd(&cnt[cell], 1);
    if (slot < cap) atoms[(size_t)cell * cap + slot] = (int)i;
    else atomicOr(status, ST_CELL);
}

// Each cell's atom list is put in increasing atom order once per step (one
// warp per cell: every entry's rank is the number of smaller entries; atom
// indices are distinct), so the binning atomics' order never reaches the
// force sums: the engine force is bitwise reproducible.
__global__ void __launch_bounds__(256) cell_sort_kernel(int ncells, int cap, const int* __restrict__ cnt,
                                                        int* __restrict__ atoms)
{
    extern __shared__ int cs_smem[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int c = blockIdx.x * 8 + warp;
    int* in = cs_smem + warp * 2 * cap;
    int* out = in + cap;
    const int n = c < ncells ? min(cnt[c], cap) : 0;
    int* a = atoms + (size_t)(c < ncells ? c : 0) * cap;
    for (int k = lane; k < n; k += 32) in[k] = a[k];
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
        const int v = in[k];
        int r = 0;
        for (int q = 0; q < n; ++q) r += in[q] < v;
        out[r] = v;
    }
    __syncwarp();
    for (int k = lane; k < n; k += 32) a[k] = out[k];
}

// Cell-tiled LJ forces.  One CTA per home cell gathers the (sorted) atom
// lists of the 27 neighbour cells and their positions into shared memory;
// one warp per target atom of the home cell; lane l takes candidates l,
// l+32, ... in (cell, atom) order; a fixed xor-shuffle tree reduces the lanes.
constexpr int LJ_T = 512;  // 16 warps: about one target atom per warp

template <typename R>
__global__ void __launch_bounds__(LJ_T) lj_tiled_kernel(const R4<R>* __restrict__ x, Box box, int ncx, int ncy,
                                                        int ncz, int cap, const int* __restrict__ cnt,
                                                        const int* __restrict__ atoms, R rc2, R sig2, R eps24,
                                                        R4<R>* __restrict__ f)
{
    extern __shared__ __align__(32) unsigned char lj_smem[];
    __shared__ int off[28];
    __shared__ int nbc[27];
    const int c = blockIdx.x;
    const int cz = c % ncz, cy = (c / ncz) % ncy, cx = c / (ncy * ncz);
    if (threadIdx.x < 27) {
        const int q = threadIdx.x;
        const int dx = q / 9 - 1, dy = (q / 3) % 3 - 1, dz = q % 3 - 1;
        const int nb = (((cx + dx + ncx) % ncx) * ncy + (cy + dy + ncy) % ncy) * ncz + (cz + dz + ncz) % ncz;
        nbc[q] = nb;
        off[q + 1] = min(cnt[nb], cap);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        off[0] = 0;
        for (int q = 0; q < 27; ++q) off[q + 1] += off[q];
    }
    __syncthreads();
    const int ncand = off[27];
    int* idx = reinterpret_cast<int*>(lj_smem);
    R4<R>* cp = reinterpret_cast<R4<R>*>(lj_smem + (((size_t)27 * cap * sizeof(int) + 31) / 32) * 32);
    // flat gather: candidate e lives in neighbour cell q with off[q] <= e <
    // off[q+1]; it is stored at its periodic image next to the home cell, so
    // the pair loop needs no minimum image
    const int hc[3] = {cx, cy, cz}, ncv[3] = {ncx, ncy, ncz};
    for (int e = threadIdx.x; e < ncand; e += LJ_T) {
        int q = 0;
        while (off[q + 1] <= e) ++q;
        const int j = atoms[(size_t)nbc[q] * cap + (e - off[q])];
        idx[e] = j;
        const int dq[3] = {q / 9 - 1, (q / 3) % 3 - 1, q % 3 - 1};
        int img[3];
        for (int k = 0; k < 3; ++k) {
            const int n = hc[k] + dq[k];
            img[k] = n < 0 ? -1 : (n >= ncv[k] ? 1 : 0);
        }
        const R4<R> sx = x[j];
        cp[e] = mk4<R>(image_coord<R>(sx.x, img[0], box, 0), image_coord<R>(sx.y, img[1], box, 1),
                       image_coord<R>(sx.z, img[2], box, 2), R(0));
    }
    __syncthreads();
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    const int nhome = min(cnt[c], cap);
    for (int t = warp; t < nhome; t += LJ_T / 32) {
        const int i = atoms[(size_t)c * cap + t];
        const R4<R> px = x[i];
        const R p[3] = {image_coord<R>(px.x, 0, box, 0), image_coord<R>(px.y, 0, box, 1),
                        image_coord<R>(px.z, 0, box, 2)};
        R fx = 0, fy = 0, fz = 0;
#pragma unroll 4
        for (int e = lane; e < ncand; e += 32) {
            const R4<R> s = cp[e];
            const R ddx = p[0] - s.x;
            const R ddy = p[1] - s.y;
            const R ddz = p[2] - s.z;
            const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 < rc2 && idx[e] != i) {
                const R fr = lj_fr<R>(r2, sig2, eps24);
                fx += fr * ddx;
                fy += fr * ddy;
                fz += fr * ddz;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane == 0) f[i] = mk4<R>(fx, fy, fz, R(0));
    }
}

template <typename R> static size_t lj_tiled_smem(int cap)
{
    return ((size_t)27 * cap * sizeof(int) + 31) / 32 * 32 + (size_t)27 * cap * sizeof(R4<R>);
}

// Bead chain: bonds kb/2 (r - r0)^2, angles ka/2 (theta - th0)^2, torsions
// kt (1 + cos 3 phi); each bead gathers the terms it takes part in.
template <typename R>
__device__ __forceinline__ void angle_grad(const R a[3], const R b[3], const R c[3], R ka, R th0, R ga[3], R gb[3],
                                           R gc[3])
{
    R u[3], v[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = a[k] - b[k];
        v[k] = c[k] - b[k];
    }
    const R nu2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], nv2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const R nu = sqrt(nu2), nv = sqrt(nv2);
    R cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (nu * nv);
    const R th = acos(cs);
    const R dU = ka * (th - th0) * (R(-1) / sin(th));  // dU/dcos
    for (int k = 0; k < 3; ++k) {
        const R du = v[k] / (nu * nv) - cs * u[k] / nu2;
        const R dv = u[k] / (nu * nv) - cs * v[k] / nv2;
        ga[k] = dU * du;
        gc[k] = dU * dv;
        gb[k] = -(ga[k] + gc[k]);
    }
}

template <typename R>
__global__ void chain_kernel(const R4<R>* __restrict__ x, const int64_t* __restrict__ woff, const int* __restrict__ wn,
                             R kb, R r0, R ka, R th0, R kt, R4<R>* __restrict__ f)
{
    const int w = blockIdx.y;
    const int n = wn[w];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long o = woff[w];
    auto P = [&](int j, R q[3]) {
        const R4<R> v = x[o + j];
        q[0] = v.x;
        q[1] = v.y;
        q[2] = v.z;
    };
    R gi[3] = {0, 0, 0};  // dU/dr_i
    R pi[3];
    P(i, pi);
    for (int j = i - 1; j <= i + 1; j += 2) {
        if (j < 0 || j >= n) continue;
        R pj[3];
        P(j, pj);
        const R d[3] = {pi[0] - pj[0], pi[1] - pj[1], pi[2] - pj[2]};
        const R r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const R c = kb * (r - r0) / r;
        for (int k = 0; k < 3; ++k) gi[k] += c * d[k];
    }
    for (int s = i - 2; s <= i; ++s) {  // angle (s, s+1, s+2)
        if (s < 0 || s + 2 >= n) continue;
        R a[3], b[3], c[3], ga[3], gb[3], gc[3];
        P(s, a);
        P(s + 1, b);
        P(s + 2, c);
        angle_grad<R>(a, b, c, ka, th0, ga, gb, gc);
        const R* g = (i == s) ? ga : (i == s + 1 ? gb : gc);
        for (int k = 0; k < 3; ++k) gi[k] += g[k];
    }
    for (int s = i - 3; s <= i; ++s) {  // torsion (s .. s+3)
        if (s < 0 || s + 3 >= n) continue;
        R p[4][3];
        for (int q = 0; q < 4; ++q) P(s + q, p[q]);
        R b1[3], b2[3], b3[3];
        for (int k = 0; k < 3; ++k) {
            b1[k] = p[1][k] - p[0][k];
            b2[k] = p[2][k] - p[1][k];
            b3[k] = p[3][k] - p[2][k];
        }
        const R n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
        const R n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
        const R b2sq = b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2], nb2 = sqrt(b2sq);
        const R phi = atan2(nb2 * (b1[0] * n2[0] + b1[1] * n2[1] + b1[2] * n2[2]),
                            n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
        const R dU = R(-3) * kt * sin(R(3) * phi);
        const R n1sq = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
        const R n2sq = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
        const R u = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / b2sq;
        const R v = (b3[0] * b2[0] + b3[1] * b2[1] + b3[2] * b2[2]) / b2sq;
        const int q = i - s;
        for (int k = 0; k < 3; ++k) {
            const R g0 = -nb2 / n1sq * n1[k], g3 = nb2 / n2sq * n2[k];
            R g = q == 0 ? g0 : (q == 3 ? g3 : (q == 1 ? -(R(1) + u) * g0 + v * g3 : -(R(1) + v) * g3 + u * g0));
            gi[k] += dU * g;
        }
    }
    f[o + i] = mk4<R>(-gi[0], -gi[1], -gi[2], R(0));
}

__global__ void philox_test_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* q = in + 6 * i;
    const U4 r = philox10(q[0], q[1], q[2], q[3], q[4], q[5]);
    for (int k = 0; k < 4; ++k) out[4 * i + k] = r.v[k];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int setup_cells(wtmd_t* h)
{
    h->ncells = 0;
    if (h->cfg.engine != WTMD_ENGINE_LJ || h->W != 1) return WTMD_OK;
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        if (!(h->cfg.box[k] > 0)) return WTMD_OK;  // open boundaries: all pairs
        nc[k] = (int)floor(h->cfg.box[k] / h->cfg.lj_rc);
        if (nc[k] < 3) return WTMD_OK;             // too small for a 27-cell stencil
    }
    h->nc[0] = nc[0];
    h->nc[1] = nc[1];
    h->nc[2] = nc[2];
    h->ncells = nc[0] * nc[1] * nc[2];
    // capacity: twice the mean occupancy plus 16 (a liquid cell exceeding it
    // is a many-sigma event; overflow is reported as WTMD_ECELL)
    const double mean = (double)h->N / h->ncells;
    int cap = (int)ceil(2.0 * mean + 16.0);
    h->cell_cap = (cap + 7) / 8 * 8;
    const size_t sm = h->prec == WTMD_F32 ? lj_tiled_smem<float>(h->cell_cap) : lj_tiled_smem<double>(h->cell_cap);
    if (sm > 200 * 1024) {
        h->ncells = 0;  // too dense for the tiled kernel: all pairs
        return WTMD_OK;
    }
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, cudaFuncSetAttribute(lj_tiled_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    else
        WTMD_CUDA_TRY(h, cudaFuncSetAttribute(lj_tiled_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->cell_count, sizeof(int) * h->ncells));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->cell_atoms, sizeof(int) * (size_t)h->ncells * h->cell_cap));
    return WTMD_OK;
}

template <typename R> static int launch_engine_t(wtmd_t* h)
{
    const auto* x = (const R4<R>*)h->pos;
    auto* f = (R4<R>*)h->force;
    const int nb = (int)((h->N + 255) / 256);
    cudaStream_t st = h->stream;
    const wtmd_config& c = h->cfg;
    switch (c.engine) {
    case WTMD_ENGINE_NONE:
        WTMD_CUDA_TRY(h, cudaMemsetAsync(f, 0, sizeof(R4<R>) * h->N, st));
        mark(h, "zero_force");
        break;
    case WTMD_ENGINE_MB:
        mb_kernel<R><<<nb, 256, 0, st>>>(h->N, x, f);
        mark(h, "mb_force");
        break;
    case WTMD_ENGINE_WELLS3:
        wells3_kernel<R><<<nb, 256, 0, st>>>(h->N, x, f);
        mark(h, "wells3_force");
        break;
    case WTMD_ENGINE_LJ: {
        const R rc2 = (R)(c.lj_rc * c.lj_rc), sig2 = (R)(c.lj_sigma * c.lj_sigma), e24 = (R)(24.0 * c.lj_eps);
        if (h->ncells > 0) {
            WTMD_CUDA_TRY(h, cudaMemsetAsync(h->cell_count, 0, sizeof(int) * h->ncells, st));
            cell_bin_kernel<R><<<nb, 256, 0, st>>>(h->N, x, h->box, h->nc[0], h->nc[1], h->nc[2], h->cell_cap,
                                                   h->cell_count, h->cell_atoms, h->status);
            mark(h, "lj_cell_bin");
            cell_sort_kernel<<<(h->ncells + 7) / 8, 256, 8 * 2 * h->cell_cap * sizeof(int), st>>>(
                h->ncells, h->cell_cap, h->cell_count, h->cell_atoms);
            mark(h, "lj_cell_sort");
            lj_tiled_kernel<R><<<h->ncells, LJ_T, lj_tiled_smem<R>(h->cell_cap), st>>>(
                x, h->box, h->nc[0], h->nc[1], h->nc[2], h->cell_cap, h->cell_count, h->cell_atoms, rc2, sig2, e24, f);
            mark(h, "lj_cell_force");
        } else {
            dim3 g((h->max_wn + 127) / 128, h->W);
            lj_allpairs_kernel<R><<<g, 128, 0, st>>>(x, h->woff, h->wn, h->box, rc2, sig2, e24, f);
            mark(h, "lj_allpairs");
        }
        break;
    }
    case WTMD_ENGINE_CHAIN: {
        dim3 g((h->max_wn + 127) / 128, h->W);
        chain_kernel<R><<<g, 128, 0, st>>>(x, h->woff, h->wn, (R)c.bond_k, (R)c.bond_r0, (R)c.angle_k,
                                           (R)c.angle_theta0, (R)c.torsion_k, f);
        mark(h, "chain_force");
        break;
    }
    default:
        h->err = "unknown engine";
        return WTMD_EINVAL;
    }
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

int launch_engine(wtmd_t* h)
{
    return h->prec == WTMD_F32 ? launch_engine_t<float>(h) : launch_engine_t<double>(h);
}

int launch_baoab_first(wtmd_t* h, int jmask, int xmask)
{
    const int nb = (int)((std::max<long long>(h->N, h->W) + 255) / 256);
    const wtmd_config& c = h->cfg;
    const double c1 = exp(-c.friction * c.dt);
    const double c2 = sqrt((1.0 - c1 * c1) * c.kT / c.mass);
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, launch_pdl(baoab_first_kernel<float>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N,
                                    (float4*)h->pos, (float4*)h->vel, (const float4*)h->force,
                                    (const long long*)h->step, c.seed, (float)(0.5 * c.dt), (float)(1.0 / c.mass),
                                    (float)c1, (float)c2, h->dims, (float4*)h->J, jmask, h->xi, xmask, h->W));
    else
        WTMD_CUDA_TRY(h, launch_pdl(baoab_first_kernel<double>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N,
                                    (dbl4*)h->pos, (dbl4*)h->vel, (const dbl4*)h->force, (const long long*)h->step,
                                    c.seed, 0.5 * c.dt, 1.0 / c.mass, c1, c2, h->dims, (dbl4*)h->J, jmask,
                                    h->xi, xmask, h->W));
    mark(h, "baoab_first");
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

}  // namespace wtmd

extern "C" int wtmd_philox(const uint32_t* in_host, uint32_t* out_host, int64_t n)
{
    if (n <= 0 || !in_host || !out_host) return WTMD_EINVAL;
    uint32_t *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, sizeof(uint32_t) * 6 * n) != cudaSuccess) return WTMD_ENOMEM;
    if (cudaMalloc(&dout, sizeof(uint32_t) * 4 * n) != cudaSuccess) {
        cudaFree(din);
        return WTMD_ENOMEM;
    }
    cudaMemcpy(din, in_host, sizeof(uint32_t) * 6 * n, cudaMemcpyHostToDevice);
    wtmd::philox_test_kernel<<<(unsigned)((n + 255) / 256), 256>>>(din, dout, n);
    cudaError_t e = cudaMemcpy(out_host, dout, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    return e == cudaSuccess ? WTMD_OK : WTMD_ECUDA;
}
