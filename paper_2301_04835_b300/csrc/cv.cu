// Collective variables and their Jacobians (PySAGES paper, Sec. 2.2; the paper
// differentiates them with jax.grad, Sec. 2 -- here the derivatives are
// written by hand), and the bias-force scatter F -= J^T dV/dxi that adds the
// biasing force to the engine's net force (Sec. 2, force-like object;
// Sec. 3.2.1 step (e)).
//
// Layout: positions/forces are [N][4] Real in HBM, walkers contiguous.  Every
// CV c writes xi[w][c] for every walker w and its dense Jacobian rows
// J[c][atom] (Real4) for the atoms it touches; rows of other atoms stay zero.
// Pair CVs (coordination) run as two deterministic gather passes over
// (target tile x source split) blocks with the sources staged in shared
// memory, followed by a fixed-order reduction over the splits: no atomics, so
// results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "step_dev.cuh"
#include "coord_dev.cuh"

namespace wtmd {

template <typename R> __device__ __forceinline__ void load3(const R4<R>* p, long long i, R& x, R& y, R& z)
{
    const R4<R> v = p[i];
    x = v.x;
    y = v.y;
    z = v.z;
}

template <typename R> __device__ __forceinline__ void delta(const Box& b, R ax, R ay, R az, R bx, R by, R bz, R d[3])
{
    d[0] = min_image<R>(ax - bx, b, 0);
    d[1] = min_image<R>(ay - by, b, 1);
    d[2] = min_image<R>(az - bz, b, 2);
}

// Deterministic block-wide sum of NV values (blockDim.x a multiple of 32,
// <= 1024); every thread gets the totals.
template <typename T, int NV> __device__ void block_sum(T v[NV])
{
    __shared__ T sm[32][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    __syncthreads();
    for (int k = 0; k < NV; ++k) {
        T s = 0;
        for (int w = 0; w < nw; ++w) s += sm[w][k];
        v[k] = s;
    }
}

// Deterministic block-wide compensated FP32 sum of NV values; every thread
// gets the totals.
template <int NV> __device__ void block_sum_cf(cf v[NV])
{
    __shared__ cf sm[32][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = cf_add(v[k], cf_shfl_xor(v[k], o));
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    __syncthreads();
    for (int k = 0; k < NV; ++k) {
        cf t = sm[0][k];
        for (int w = 1; w < nw; ++w) t = cf_add(t, sm[w][k]);
        v[k] = t;
    }
}

// ---------------------------------------------------------------------------
// Component (Sec. 2.2, AxisCV): xi = scale * x_axis of one atom.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void cv_component_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff, int W, int idx,
                                    int axis, R scale, double* __restrict__ xi, int col, R4<R>* __restrict__ J)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const long long i = woff[w] + idx;
    const R4<R> p = pos[i];
    const R v = axis == 0 ? p.x : (axis == 1 ? p.y : p.z);
    xi[w * 4 + col] = (double)(scale * v);
    J[i] = mk4<R>(axis == 0 ? scale : R(0), axis == 1 ? scale : R(0), axis == 2 ? scale : R(0), R(0));
}

// ---------------------------------------------------------------------------
// Dihedral angle (Sec. 2.2, FourPointCV), IUPAC sign:
//   b1 = p1-p0, b2 = p2-p1, b3 = p3-p2, n1 = b1 x b2, n2 = b2 x b3,
//   phi = atan2(|b2| b1.n2, n1.n2);
//   dphi/dp0 = -|b2|/|n1|^2 n1, dphi/dp3 = |b2|/|n2|^2 n2,
//   dphi/dp1 = -(1+u) dphi/dp0 + v dphi/dp3, dphi/dp2 = -(1+v) dphi/dp3 + u dphi/dp0,
//   u = b1.b2/|b2|^2, v = b3.b2/|b2|^2.
// ---------------------------------------------------------------------------
template <typename R> struct Dih {
    R phi;
    R g[4][3];
};

template <typename R>
__device__ __forceinline__ void dihedral_grad(const R p[4][3], const Box& box, Dih<R>& out, bool want_grad)
{
    R b1[3], b2[3], b3[3];
    delta<R>(box, p[1][0], p[1][1], p[1][2], p[0][0], p[0][1], p[0][2], b1);
    delta<R>(box, p[2][0], p[2][1], p[2][2], p[1][0], p[1][1], p[1][2], b2);
    delta<R>(box, p[3][0], p[3][1], p[3][2], p[2][0], p[2][1], p[2][2], b3);
    const R n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
    const R n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
    const R b2sq = b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2];
    const R nb2 = sqrt(b2sq);
    const R y = nb2 * (b1[0] * n2[0] + b1[1] * n2[1] + b1[2] * n2[2]);
    const R x = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
    out.phi = atan2(y, x);
    if (!want_grad) return;
    const R n1sq = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
    const R n2sq = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
    const R u = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / b2sq;
    const R v = (b3[0] * b2[0] + b3[1] * b2[1] + b3[2] * b2[2]) / b2sq;
    const R f0 = -nb2 / n1sq, f3 = nb2 / n2sq;
    for (int k = 0; k < 3; ++k) {
        const R g0 = f0 * n1[k], g3 = f3 * n2[k];
        out.g[0][k] = g0;
        out.g[3][k] = g3;
        out.g[1][k] = -(R(1) + u) * g0 + v * g3;
        out.g[2][k] = -(R(1) + v) * g3 + u * g0;
    }
}

template <typename R>
__global__ void cv_dihedral_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff, int W, int4 idx,
                                   Box box, R scale, double* __restrict__ xi, int col, R4<R>* __restrict__ J)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const long long o = woff[w];
    const long long ids[4] = {o + idx.x, o + idx.y, o + idx.z, o + idx.w};
    R p[4][3];
    for (int k = 0; k < 4; ++k) load3<R>(pos, ids[k], p[k][0], p[k][1], p[k][2]);
    Dih<R> dh;
    dihedral_grad<R>(p, box, dh, true);
    xi[w * 4 + col] = (double)(scale * dh.phi);
    for (int k = 0; k < 4; ++k) J[ids[k]] = mk4<R>(scale * dh.g[k][0], scale * dh.g[k][1], scale * dh.g[k][2], R(0));
}

// ---------------------------------------------------------------------------
// Radius of gyration (Sec. 2.2), equal masses.  Members are unwrapped by the
// minimum image relative to the group's first atom; Rg = sqrt(mean |u-c|^2),
// dRg/dr_k = (u_k - c) / (m Rg).  One block per walker.
// ---------------------------------------------------------------------------
constexpr int RG_CACHE = 1024;  // members whose unwrapped position stays in shared memory

// Rg of walker w by the whole CTA (u: RG_CACHE staged members in shared
// memory).  The member indices of the first round are read before wait()
// (the dependency wait of a programmatic launch), the positions after it.
// FP32 handles finish in FP32 (compensated sums; a dependent FP64 division
// or square root costs ~700 cycles on this GPU), FP64 handles in FP64.
template <typename R, class Wait>
__device__ void cv_rg_body(int w, const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff,
                           const int* __restrict__ wn, const int* __restrict__ A, int nA, const Box& box, double scale,
                           int intensive, double* __restrict__ xi, int col, R4<R>* __restrict__ J, R4<R>* u, Wait wait)
{
    __shared__ R bc[4];  // broadcast: centre (3) and the Jacobian factor
    const long long o = woff[w];
    const int m = A ? nA : wn[w];
    const int i0 = A ? A[0] : 0;
    const int ifirst = (int)threadIdx.x < m ? (A ? A[threadIdx.x] : (int)threadIdx.x) : 0;
    wait();
    R rx, ry, rz;
    load3<R>(pos, o + i0, rx, ry, rz);
    // unwrapped position of member p (minimum image relative to member 0)
    auto unwrap_i = [&](int i) {
        R x, y, z, d[3];
        load3<R>(pos, o + i, x, y, z);
        delta<R>(box, x, y, z, rx, ry, rz, d);
        return mk4<R>(rx + d[0], ry + d[1], rz + d[2], R(0));
    };
    auto member = [&](int p) { return p == (int)threadIdx.x ? ifirst : (A ? A[p] : p); };
    // FP32 handles sum in compensated FP32, FP64 handles in FP64
    cf s[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double sd[3] = {0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const R4<R> q = unwrap_i(member(p));
        if (p < RG_CACHE) u[p] = q;
        if constexpr (sizeof(R) == 4) {
            s[0] = cf_add(s[0], (float)q.x);
            s[1] = cf_add(s[1], (float)q.y);
            s[2] = cf_add(s[2], (float)q.z);
        } else {
            sd[0] += (double)q.x;
            sd[1] += (double)q.y;
            sd[2] += (double)q.z;
        }
    }
    if constexpr (sizeof(R) == 4) block_sum_cf<3>(s);
    else block_sum<double, 3>(sd);
    if (threadIdx.x == 0) {
        if constexpr (sizeof(R) == 4) {
            const float im = 1.f / (float)m;
            for (int k = 0; k < 3; ++k) bc[k] = (s[k].hi + s[k].lo) * im;
        } else {
            for (int k = 0; k < 3; ++k) bc[k] = (R)(sd[k] / m);
        }
    }
    __syncthreads();
    const R c[3] = {bc[0], bc[1], bc[2]};
    cf q2[1] = {{0.f, 0.f}};
    double q2d[1] = {0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const R4<R> q = p < RG_CACHE ? u[p] : unwrap_i(member(p));
        const R ux = q.x - c[0], uy = q.y - c[1], uz = q.z - c[2];
        if constexpr (sizeof(R) == 4) q2[0] = cf_add(q2[0], (float)(ux * ux + uy * uy + uz * uz));
        else q2d[0] += (double)(ux * ux + uy * uy + uz * uz);
    }
    if constexpr (sizeof(R) == 4) block_sum_cf<1>(q2);
    else block_sum<double, 1>(q2d);
    __shared__ double rg_s;
    if (threadIdx.x == 0) {
        if constexpr (sizeof(R) == 4) {
            const float rg = sqrtf((q2[0].hi + q2[0].lo) / (float)m);
            float sc = scale != 0.0 ? (float)scale : 1.f;
            if (intensive) sc /= cbrtf((float)m);
            bc[3] = sc / ((float)m * rg);
            rg_s = (double)(sc * rg);
        } else {
            const double rg = sqrt(q2d[0] / m);
            double sc = scale != 0.0 ? scale : 1.0;
            if (intensive) sc /= cbrt((double)m);
            bc[3] = (R)(sc / (m * rg));
            rg_s = sc * rg;
        }
    }
    __syncthreads();
    const R f = bc[3];
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = member(p);
        const R4<R> q = p < RG_CACHE ? u[p] : unwrap_i(i);
        J[o + i] = mk4<R>(f * (q.x - c[0]), f * (q.y - c[1]), f * (q.z - c[2]), R(0));
    }
    if (threadIdx.x == 0) xi[w * 4 + col] = rg_s;
}

// One block per walker.  A programmatic dependent of the kernel that moved
// the atoms: the kernels that need this CV (joined after it) may launch at
// once; the positions are waited for.
template <typename R>
__global__ void __launch_bounds__(256) cv_rg_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff,
                                                    const int* __restrict__ wn, const int* __restrict__ A, int nA,
                                                    Box box, double scale, int intensive, double* __restrict__ xi,
                                                    int col, R4<R>* __restrict__ J)
{
    __shared__ R4<R> u[RG_CACHE];
    pdl_trigger();
    cv_rg_body<R>((int)blockIdx.x, pos, woff, wn, A, nA, box, scale, intensive, xi, col, J, u, [] { pdl_wait(); });
}

// ---------------------------------------------------------------------------
// Equal-mass centre of a group (all atoms of the walker when A is null):
// members unwrapped by the minimum image relative to the first member, as
// for Rg; compensated FP32 sums on FP32 handles, FP64 sums on FP64 handles.
// Block-wide; every thread gets the centre.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R4<R> unwrap_member(const R4<R>* pos, long long o, const int* A, int p, const Box& box,
                                               R rx, R ry, R rz)
{
    const int i = A ? A[p] : p;
    R x, y, z, d[3];
    load3<R>(pos, o + i, x, y, z);
    delta<R>(box, x, y, z, rx, ry, rz, d);
    return mk4<R>(rx + d[0], ry + d[1], rz + d[2], R(0));
}

template <typename R>
__device__ void group_centre(const R4<R>* pos, long long o, const int* A, int m, const Box& box, R ref[3], R c[3])
{
    load3<R>(pos, o + (A ? A[0] : 0), ref[0], ref[1], ref[2]);
    cf s[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double sd[3] = {0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const R4<R> q = unwrap_member<R>(pos, o, A, p, box, ref[0], ref[1], ref[2]);
        if constexpr (sizeof(R) == 4) {
            s[0] = cf_add(s[0], (float)q.x);
            s[1] = cf_add(s[1], (float)q.y);
            s[2] = cf_add(s[2], (float)q.z);
        } else {
            sd[0] += (double)q.x;
            sd[1] += (double)q.y;
            sd[2] += (double)q.z;
        }
    }
    if constexpr (sizeof(R) == 4) {
        block_sum_cf<3>(s);
        for (int k = 0; k < 3; ++k) c[k] = (R)(cf_val(s[k]) / m);
    } else {
        block_sum<double, 3>(sd);
        for (int k = 0; k < 3; ++k) c[k] = (R)(sd[k] / m);
    }
}

// ---------------------------------------------------------------------------
// Distance between the centres of groups A and B (Sec. 2.2, TwoPointCV),
// the centre difference d = c_B - c_A by the minimum image; xi = scale |d|,
// dxi/dr = -scale d / (|d| |A|) on A and +scale d / (|d| |B|) on B (A and B
// disjoint).  One block per walker.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) cv_distance_kernel(const R4<R>* __restrict__ pos,
                                                          const int64_t* __restrict__ woff, const int* __restrict__ A,
                                                          int nA, const int* __restrict__ B, int nB, Box box, R scale,
                                                          double* __restrict__ xi, int col, R4<R>* __restrict__ J)
{
    const int w = blockIdx.x;
    const long long o = woff[w];
    R ra[3], rb[3], ca[3], cb[3], d[3];
    group_centre<R>(pos, o, A, nA, box, ra, ca);
    group_centre<R>(pos, o, B, nB, box, rb, cb);
    delta<R>(box, cb[0], cb[1], cb[2], ca[0], ca[1], ca[2], d);
    const R r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const R ga = -scale / (r * (R)nA), gb = scale / (r * (R)nB);
    for (int p = threadIdx.x; p < nA; p += blockDim.x) J[o + A[p]] = mk4<R>(ga * d[0], ga * d[1], ga * d[2], R(0));
    for (int p = threadIdx.x; p < nB; p += blockDim.x) J[o + B[p]] = mk4<R>(gb * d[0], gb * d[1], gb * d[2], R(0));
    if (threadIdx.x == 0) xi[w * 4 + col] = (double)(scale * r);
}

// ---------------------------------------------------------------------------
// Angle at the middle of three atoms (Sec. 2.2, ThreePointCV): u = p0 - p1,
// v = p2 - p1 (minimum image), w = u x v, theta = atan2(|w|, u.v) in [0, pi];
// with n = w / |w|:  dtheta/du = (u.v (v x n) - |w| v) / (|w|^2 + (u.v)^2),
// dtheta/dv = (u.v (n x u) - |w| u) / (...), dtheta/dp1 = -(dtheta/du +
// dtheta/dv); zero where |w| = 0 (theta = 0 or pi).  One thread per walker.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void cv_angle_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff, int W, int3 idx,
                                Box box, R scale, double* __restrict__ xi, int col, R4<R>* __restrict__ J)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const long long o = woff[w];
    const long long i0 = o + idx.x, i1 = o + idx.y, i2 = o + idx.z;
    R p0[3], p1[3], p2[3], u[3], v[3];
    load3<R>(pos, i0, p0[0], p0[1], p0[2]);
    load3<R>(pos, i1, p1[0], p1[1], p1[2]);
    load3<R>(pos, i2, p2[0], p2[1], p2[2]);
    delta<R>(box, p0[0], p0[1], p0[2], p1[0], p1[1], p1[2], u);
    delta<R>(box, p2[0], p2[1], p2[2], p1[0], p1[1], p1[2], v);
    const R wx = u[1] * v[2] - u[2] * v[1], wy = u[2] * v[0] - u[0] * v[2], wz = u[0] * v[1] - u[1] * v[0];
    const R sn = sqrt(wx * wx + wy * wy + wz * wz);
    const R cs = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    R gu[3] = {R(0), R(0), R(0)}, gv[3] = {R(0), R(0), R(0)};
    if (sn > R(0)) {
        const R nx = wx / sn, ny = wy / sn, nz = wz / sn;
        const R inv = scale / (sn * sn + cs * cs);
        const R vn[3] = {v[1] * nz - v[2] * ny, v[2] * nx - v[0] * nz, v[0] * ny - v[1] * nx};
        const R nu[3] = {ny * u[2] - nz * u[1], nz * u[0] - nx * u[2], nx * u[1] - ny * u[0]};
        for (int k = 0; k < 3; ++k) {
            gu[k] = inv * (cs * vn[k] - sn * v[k]);
            gv[k] = inv * (cs * nu[k] - sn * u[k]);
        }
    }
    xi[w * 4 + col] = (double)(scale * atan2(sn, cs));
    J[i0] = mk4<R>(gu[0], gu[1], gu[2], R(0));
    J[i2] = mk4<R>(gv[0], gv[1], gv[2], R(0));
    J[i1] = mk4<R>(-(gu[0] + gv[0]), -(gu[1] + gv[1]), -(gu[2] + gv[2]), R(0));
}

// ---------------------------------------------------------------------------
// Gyration-tensor CVs (Sec. 2.2: PrincipalMoment, Asphericity,
// Acylindricity, ShapeAnisotropy), equal masses.  S = (1/m) sum (u-c)(u-c)^T
// over the unwrapped members; eigenvalues l1 <= l2 <= l3 with unit vectors
// e1..e3.  quantity 0..2: l1..l3; 3: l3 - (l1+l2)/2; 4: l2 - l1;
// 5: 3/2 (l1^2+l2^2+l3^2)/(l1+l2+l3)^2 - 1/2.  For simple eigenvalues
// dl_j/dr_k = (2/m) (e_j . (u_k - c)) e_j; the quantity's gradient is
// sum_j (dq/dl_j) dl_j/dr_k.  One block per walker; the 3x3 eigenproblem is
// solved by thread 0 in FP64 with Jacobi rotations, each zeroing one
// off-diagonal element and updating the others in place.
// ---------------------------------------------------------------------------
__device__ void sym3_eigen(double a[3][3], double lam[3], double ev[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) ev[i][j] = i == j ? 1.0 : 0.0;
    for (int it = 0; it < 64; ++it) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double dia = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off == 0.0 || off <= 1e-18 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = a[p][q];
                if (apq == 0.0) continue;
                const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
                const double t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = rsqrt(t * t + 1.0), s = t * c;
                a[p][p] -= t * apq;
                a[q][q] += t * apq;
                a[p][q] = a[q][p] = 0.0;
                const int r = 3 - p - q;  // the remaining index
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = a[p][r] = c * arp - s * arq;
                a[r][q] = a[q][r] = s * arp + c * arq;
                for (int k = 0; k < 3; ++k) {
                    const double vp = ev[k][p], vq = ev[k][q];
                    ev[k][p] = c * vp - s * vq;
                    ev[k][q] = s * vp + c * vq;
                }
            }
    }
    int ord[3] = {0, 1, 2};
    if (a[ord[1]][ord[1]] < a[ord[0]][ord[0]]) { const int t = ord[0]; ord[0] = ord[1]; ord[1] = t; }
    if (a[ord[2]][ord[2]] < a[ord[1]][ord[1]]) { const int t = ord[1]; ord[1] = ord[2]; ord[2] = t; }
    if (a[ord[1]][ord[1]] < a[ord[0]][ord[0]]) { const int t = ord[0]; ord[0] = ord[1]; ord[1] = t; }
    double e2[3][3];
    for (int j = 0; j < 3; ++j) {
        lam[j] = a[ord[j]][ord[j]];
        for (int k = 0; k < 3; ++k) e2[k][j] = ev[k][ord[j]];
    }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) ev[k][j] = e2[k][j];
}

template <typename R>
__global__ void __launch_bounds__(256) cv_gyration_kernel(const R4<R>* __restrict__ pos,
                                                          const int64_t* __restrict__ woff, const int* __restrict__ wn,
                                                          const int* __restrict__ A, int nA, Box box, int quantity,
                                                          double scale, double* __restrict__ xi, int col,
                                                          R4<R>* __restrict__ J)
{
    __shared__ R sh_e[3][3], sh_g[3];  // unit eigenvectors e_j (sh_e[j]) and factors scale dq/dl_j 2/m
    const int w = blockIdx.x;
    const long long o = woff[w];
    const int m = A ? nA : wn[w];
    R ref[3], c[3];
    group_centre<R>(pos, o, A, m, box, ref, c);
    cf t[6] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double td[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const R4<R> q = unwrap_member<R>(pos, o, A, p, box, ref[0], ref[1], ref[2]);
        const R dx = q.x - c[0], dy = q.y - c[1], dz = q.z - c[2];
        const R prod[6] = {dx * dx, dy * dy, dz * dz, dx * dy, dx * dz, dy * dz};
        for (int k = 0; k < 6; ++k) {
            if constexpr (sizeof(R) == 4) t[k] = cf_add(t[k], (float)prod[k]);
            else td[k] += (double)prod[k];
        }
    }
    if constexpr (sizeof(R) == 4) {
        block_sum_cf<6>(t);
        for (int k = 0; k < 6; ++k) td[k] = cf_val(t[k]);
    } else {
        block_sum<double, 6>(td);
    }
    if (threadIdx.x == 0) {
        double S[3][3] = {{td[0] / m, td[3] / m, td[4] / m}, {td[3] / m, td[1] / m, td[5] / m},
                          {td[4] / m, td[5] / m, td[2] / m}};
        double l[3], ev[3][3];
        sym3_eigen(S, l, ev);
        const double T = l[0] + l[1] + l[2], Q = l[0] * l[0] + l[1] * l[1] + l[2] * l[2];
        double q = 0.0, g[3] = {0.0, 0.0, 0.0};
        if (quantity <= 2) {
            q = l[quantity];
            g[quantity] = 1.0;
        } else if (quantity == 3) {
            q = l[2] - 0.5 * (l[0] + l[1]);
            g[0] = g[1] = -0.5;
            g[2] = 1.0;
        } else if (quantity == 4) {
            q = l[1] - l[0];
            g[0] = -1.0;
            g[1] = 1.0;
        } else {
            q = 1.5 * Q / (T * T) - 0.5;
            for (int j = 0; j < 3; ++j) g[j] = 3.0 * (l[j] * T - Q) / (T * T * T);
        }
        for (int j = 0; j < 3; ++j) {
            sh_g[j] = (R)(scale * g[j] * 2.0 / m);
            for (int k = 0; k < 3; ++k) sh_e[j][k] = (R)ev[k][j];
        }
        xi[w * 4 + col] = scale * q;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const R4<R> q = unwrap_member<R>(pos, o, A, p, box, ref[0], ref[1], ref[2]);
        const R d[3] = {q.x - c[0], q.y - c[1], q.z - c[2]};
        R jr[3] = {R(0), R(0), R(0)};
        for (int j = 0; j < 3; ++j) {
            const R f = sh_g[j] * (sh_e[j][0] * d[0] + sh_e[j][1] * d[1] + sh_e[j][2] * d[2]);
            for (int k = 0; k < 3; ++k) jr[k] += f * sh_e[j][k];
        }
        J[o + (A ? A[p] : p)] = mk4<R>(jr[0], jr[1], jr[2], R(0));
    }
}

// ---------------------------------------------------------------------------
// Switching-function pair sums.  s(r) = 1/(1 + y^h), y = r^2/r0^2, h = n/2
// (the rational (1-x^n)/(1-x^m) with m = 2n, which equals this exactly), and
// ds/dr_t = -(n/r0^2) y^(h-1) s^2 (r_t - r_s).
//
// Coordination xi = scale sum_{i in A} sum_{j in B, j != i} s(r_ij) has
//   dxi/dr_k = scale ( [k in A] sum_{j in B, j != k} ds/dr_k(r_kj)
//                    + [k in B] sum_{i in A, i != k} ds/dr_k(r_ik) ).
// One warp per target atom k computes its whole Jacobian row: lane l takes
// partners l, l+32, ... (FP32 lane sums, FP64 xor-shuffle tree, fixed order),
// and, for k in A, the row sum of s.  The last CTA of each walker reduces the
// row sums of A in index order into xi.  No atomics on data: deterministic.
// ---------------------------------------------------------------------------
constexpr int CW_T = 256;  // threads per block (8 target warps)

// correctly rounded reciprocal (FP32: MUFU estimate + refinement, no IEEE
// division subroutine; unbiased, so sums of many terms do not drift)
template <typename R> __device__ __forceinline__ R rcp(R x);
// FP32: the PTX approximate reciprocal (1 ulp), far cheaper than the IEEE
// division sequence; the switching-function terms need no more
template <> __device__ __forceinline__ float rcp<float>(float x) { return rcp_approx(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

template <typename R>
__device__ __forceinline__ R ypow(R y, int h)
{
    R r = y;
    for (int k = 1; k < h; ++k) r *= y;
    return r;
}

constexpr int CW_CH = 512;  // source positions staged per chunk
constexpr int CW_GT = 64;   // threads per target in group mode
constexpr int CW_G = CW_T / CW_GT;

template <typename R>
__global__ void __launch_bounds__(CW_T) coord_warp_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff,
                                                          const int* __restrict__ wn, const int* __restrict__ A, int nA,
                                                          const int* __restrict__ B, int nB,
                                                          const int* __restrict__ inv_a, const int* __restrict__ inv_b,
                                                          const int* __restrict__ order, int n_order, int a_blocks,
                                                          int same_ab,
                                                          Box box, R inv_r0sq, int h, R gpref, double scale,
                                                          const double* __restrict__ scw,
                                                          double* __restrict__ rowval, int rv_stride,
                                                          unsigned* __restrict__ tickets, R4<R>* __restrict__ J,
                                                          double* __restrict__ xi, int col)
{
    __shared__ R4<R> src[CW_CH];
    __shared__ int sid[CW_CH];
    const int w = blockIdx.y;
    const int nw = wn[w];
    const long long o = woff[w];
    const int nAw = A ? nA : nw, nBw = B ? nB : nw;
    const int lane = threadIdx.x % 32;
    // group mode: the first a_blocks CTAs take CW_G targets (members of A)
    // each, one per 64-thread group, partners read straight from global
    // memory; the other CTAs take one target per warp with staged partners
    const bool bm = (int)blockIdx.x < a_blocks;
    const int gid = threadIdx.x / CW_GT, gl = threadIdx.x % CW_GT;
    const int ng = a_blocks > 0 ? nA : 0;  // targets handled by groups: the members of A
    int t = bm ? (int)blockIdx.x * CW_G + gid : ng + ((int)blockIdx.x - a_blocks) * (CW_T / 32) + threadIdx.x / 32;
    if (bm && t >= ng) t = 1 << 30;  // spare group of the last group CTA
    int k = -1, pa = -1, pb = -1;
    if (t < (order ? n_order : nw)) {
        k = order ? order[t] : t;
        if (k < nw) {
            pa = A ? inv_a[k] : k;
            pb = B ? inv_b[k] : k;
        } else {
            k = -1;
        }
    }
    R tx = 0, ty = 0, tz = 0;
    if (k >= 0) load3<R>(pos, o + k, tx, ty, tz);
    R gx = 0, gy = 0, gz = 0, sv = 0;
    // sweep 0: partners in B (targets in A, with the value); sweep 1:
    // partners in A (targets in B, gradient only; not needed when A == B)
    auto pair = [&](const R4<R> sp, int j, bool value) {
        R d[3];
        delta<R>(box, tx, ty, tz, sp.x, sp.y, sp.z, d);
        const R y = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * inv_r0sq;
        const R yh1 = ypow<R>(y, h - 1);
        R s = rcp<R>(R(1) + yh1 * y);
        if (j == k) s = R(0);  // no self pair
        if (value) sv += s;
        const R gr = gpref * yh1 * s * s;
        gx += gr * d[0];
        gy += gr * d[1];
        gz += gr * d[2];
    };
    if (bm) {
        if (pa >= 0) {
#pragma unroll 4
            for (int q = gl; q < nBw; q += CW_GT) {
                const int j = B ? B[q] : q;
                pair(pos[o + j], j, true);
            }
        }
        if (pb >= 0 && !same_ab) {
#pragma unroll 4
            for (int q = gl; q < nAw; q += CW_GT) {
                const int i = A ? A[q] : q;
                pair(pos[o + i], i, false);
            }
        }
    } else {
        // one target per warp: the CTA's 8 targets share staged partners
        for (int sweep = 0; sweep < 2; ++sweep) {
            const bool mine = sweep == 0 ? pa >= 0 : (pb >= 0 && !same_ab);
            if (!__syncthreads_or(mine)) continue;
            const int* list = sweep == 0 ? B : A;
            const int n = sweep == 0 ? nBw : nAw;
            for (int c0 = 0; c0 < n; c0 += CW_CH) {
                const int m = min(CW_CH, n - c0);
                __syncthreads();
                for (int q = threadIdx.x; q < m; q += CW_T) {
                    const int j = list ? list[c0 + q] : c0 + q;
                    src[q] = pos[o + j];
                    sid[q] = j;
                }
                __syncthreads();
                if (!mine) continue;
#pragma unroll 4
                for (int q = lane; q < m; q += 32) pair(src[q], sid[q], sweep == 0);
            }
        }
    }
    // gradient in FP32 (a fixed shuffle tree), the row sum of s in FP64 (it
    // is the CV value, which the hills sum amplifies by |xi|/sigma)
    double srow = (double)sv;
    for (int off = 16; off > 0; off >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, off);
        gy += __shfl_xor_sync(0xffffffffu, gy, off);
        gz += __shfl_xor_sync(0xffffffffu, gz, off);
        srow += __shfl_xor_sync(0xffffffffu, srow, off);
    }
    if (bm) {  // the two warps of each group, in order
        __shared__ R redg[CW_T / 32][3];
        __shared__ double reds[CW_T / 32];
        if (lane == 0) {
            redg[threadIdx.x / 32][0] = gx;
            redg[threadIdx.x / 32][1] = gy;
            redg[threadIdx.x / 32][2] = gz;
            reds[threadIdx.x / 32] = srow;
        }
        __syncthreads();
        if (gl == 0) {
            const int w0 = threadIdx.x / 32;
            gx = gy = gz = R(0);
            srow = 0.0;
            for (int w = w0; w < w0 + CW_GT / 32; ++w) {
                gx += redg[w][0];
                gy += redg[w][1];
                gz += redg[w][2];
                srow += reds[w];
            }
        }
    }
    if ((bm ? gl : lane) == 0 && k >= 0) {
        const R f = (R)((same_ab ? 2.0 : 1.0) * scw[w]);
        J[o + k] = mk4<R>(f * gx, f * gy, f * gz, R(0));
        if (pa >= 0) rowval[(size_t)w * rv_stride + pa] = srow;
    }
    // the last CTA of this walker sums the row values of A in order
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&tickets[w], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < nAw; q += CW_T) v[0] += __ldcg(rowval + (size_t)w * rv_stride + q);
    block_sum<double, 1>(v);
    if (threadIdx.x == 0) {
        xi[w * 4 + col] = scw[w] * v[0];
        tickets[w] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Coordination for a list A against a large partner group B, each ordered
// pair (i in A, j in B) evaluated once.  A CTA takes a tile of 32 members of
// A (lane l holds a_l) and a chunk of CT_B partners staged in shared memory;
// warp w sweeps partners w*32 ... w*32+31 of the chunk.  ds/dr for the row
// atom a_l accumulates in its lane; each partner's column sum -ds/dr travels
// once around the warp (one shuffle per component per pair).  Row partials
// [chunk][A] and column partials [tile][B] are written once each and summed
// in fixed order by the CTAs that complete a tile or a chunk (tickets), in
// the same launch: deterministic.
// ---------------------------------------------------------------------------
constexpr int FB = 4;      // partial sums loaded per batch in the finalization


// A partial written by another CTA of the same launch: read past L1.
template <typename R> __device__ __forceinline__ R4<R> ldcg_r4(const R4<R>* p);
template <> __device__ __forceinline__ R4<float> ldcg_r4<float>(const R4<float>* p) { return __ldcg(p); }
template <> __device__ __forceinline__ R4<double> ldcg_r4<double>(const R4<double>* p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    return dbl4{a.x, a.y, b.x, b.y};
}

template <typename R, int HC>
__global__ void __launch_bounds__(CT_T) coord_tile_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff,
                                                          const int* __restrict__ wn, const int* __restrict__ A, int nA,
                                                          const int* __restrict__ B, int nB, int nbchunk, Box box,
                                                          R inv_r0sq, int h, R gpref, R4<R>* __restrict__ rowpart,
                                                          R4<R>* __restrict__ colpart, int nB_stride,
                                                          const double* __restrict__ scw, double* __restrict__ rowval,
                                                          unsigned* __restrict__ tk, R4<R>* __restrict__ J,
                                                          double* __restrict__ xi, int col,
                                                          const int* __restrict__ inv_b)
{
    __shared__ R4<R> src[CT_B];
    __shared__ int sid[CT_B];
    __shared__ R4<R> rowred[CT_T / 32][32];
    pdl_trigger();  // the hills sum that follows may start its hill copies now
    const int w = blockIdx.y;
    const int nw = wn[w];
    const long long o = woff[w];
    const int nBw = B ? nB : nw;
    const int tile = blockIdx.x / nbchunk, chunk = blockIdx.x % nbchunk;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    const int b0 = chunk * CT_B;
    const int mb = min(CT_B, nBw - b0);
    // partners of the chunk; padding slots carry weight 0 (.w) so that they
    // contribute nothing without a branch in the pair loop.  The index lists
    // are constant: they are read before waiting for the kernel that wrote
    // the positions (programmatic dependent launch), the positions after.
    const int ia = tile * 32 + lane;
    const int a = ia < nA ? A[ia] : -1;
    int jq[CT_B / CT_T];
#pragma unroll
    for (int k = 0; k < CT_B / CT_T; ++k) {
        const int q = threadIdx.x + k * CT_T;
        jq[k] = q < mb ? (B ? B[b0 + q] : b0 + q) : -1;
    }
    pdl_wait();
#pragma unroll
    for (int k = 0; k < CT_B / CT_T; ++k) {
        const int q = threadIdx.x + k * CT_T;
        if (jq[k] >= 0) {
            const R4<R> p = pos[o + jq[k]];
            src[q] = mk4<R>(p.x, p.y, p.z, R(1));
        } else {
            src[q] = mk4<R>(R(0), R(0), R(0), R(0));
        }
        sid[q] = jq[k];
    }
    R tx = 0, ty = 0, tz = 0;
    if (a >= 0) load3<R>(pos, o + a, tx, ty, tz);
    const R gpl = a >= 0 ? gpref : R(0);  // an empty target lane adds nothing to the columns
    __syncthreads();
    // Warp `warp` sweeps partners warp*32 ... warp*32+31 in 32 rotation
    // steps: at step k lane l pairs its target with partner (l + k) mod 32
    // and carries that partner's column sum, which then moves to lane l - 1.
    // After the 32 steps lane l holds the full column sum of partner l.  The
    // pair of an atom with itself (d = 0) adds s(0) = 1 to the row sum and
    // nothing to the gradients; the row finalization removes it.
    R gx = 0, gy = 0, gz = 0, sv = 0;
    R cx = 0, cy = 0, cz = 0;
    const int base = warp * 32, from = (lane + 1) & 31;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        const R4<R> sp = src[base + ((lane + k) & 31)];
        R d[3];
        delta<R>(box, tx, ty, tz, sp.x, sp.y, sp.z, d);
        const R y = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * inv_r0sq;
        R yh1;  // y^(h-1); the exponent is a compile-time constant when HC > 0
        if constexpr (HC > 0) {
            yh1 = R(1);
#pragma unroll
            for (int e = 1; e < HC; ++e) yh1 *= y;
        } else {
            yh1 = ypow<R>(y, h - 1);
        }
        const R s = rcp<R>(R(1) + yh1 * y) * sp.w;
        sv += s;
        const R gr = gpl * yh1 * s * s;
        gx += gr * d[0];
        gy += gr * d[1];
        gz += gr * d[2];
        cx -= gr * d[0];
        cy -= gr * d[1];
        cz -= gr * d[2];
        cx = __shfl_sync(0xffffffffu, cx, from);
        cy = __shfl_sync(0xffffffffu, cy, from);
        cz = __shfl_sync(0xffffffffu, cz, from);
    }
    {
        const int q = base + lane;
        if (q < mb) colpart[((size_t)w * gridDim.x / nbchunk + tile) * nB_stride + b0 + q] = mk4<R>(cx, cy, cz, R(0));
    }
    // rows: the 8 warps hold partial sums over their partner slices
    rowred[warp][lane] = mk4<R>(gx, gy, gz, sv);
    __syncthreads();
    if (warp == 0 && a >= 0) {
        R4<R> t = rowred[0][lane];
        for (int k = 1; k < CT_T / 32; ++k) {
            const R4<R> u = rowred[k][lane];
            t.x += u.x;
            t.y += u.y;
            t.z += u.z;
            t.w += u.w;
        }
        rowpart[((size_t)w * nbchunk + chunk) * nA + ia] = t;
    }

    // Finalization without a second launch.  The CTA that completes a tile
    // (its last chunk) sums the tile's row partials over the chunks; the CTA
    // that completes a chunk (its last tile) sums the chunk's column
    // partials over the tiles; the CTA that completes the last tile sums the
    // row values into xi.  All sums run in a fixed order.  J was zeroed
    // before the launch and each atom receives at most one row and one
    // column contribution, so their two additions commute exactly.
    const int ntile = gridDim.x / nbchunk;
    const int ntk = ntile + nbchunk + 1;
    unsigned* tkw = tk + (size_t)w * ntk;
    __shared__ int last_row, last_col, last_x;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last_row = atomicAdd(&tkw[tile], 1u) == (unsigned)nbchunk - 1;
        last_col = atomicAdd(&tkw[ntile + chunk], 1u) == (unsigned)ntile - 1;
    }
    __syncthreads();
    const R f = (R)scw[w];
    if (last_row) {
        __threadfence();
        if (warp == 0 && a >= 0) {
            R sx = 0, sy = 0, sz = 0;
            cf sv{0.f, 0.f};
            double svd = 0.0;
            // loads issued in batches of FB before they are summed (in order):
            // a dependent load per partial would serialize L2 round trips
            for (int c0 = 0; c0 < nbchunk; c0 += FB) {
                R4<R> u[FB];
#pragma unroll
                for (int k = 0; k < FB; ++k)
                    if (c0 + k < nbchunk) u[k] = ldcg_r4<R>(rowpart + ((size_t)w * nbchunk + c0 + k) * nA + ia);
#pragma unroll
                for (int k = 0; k < FB; ++k)
                    if (c0 + k < nbchunk) {
                        sx += u[k].x;
                        sy += u[k].y;
                        sz += u[k].z;
                        if constexpr (sizeof(R) == 4) sv = cf_add(sv, (float)u[k].w);
                        else svd += (double)u[k].w;
                    }
            }
            atomicAdd(&J[o + a].x, f * sx);
            atomicAdd(&J[o + a].y, f * sy);
            atomicAdd(&J[o + a].z, f * sz);
            // the target's pair with itself, if it is a partner, added s(0)
            const bool self = inv_b ? inv_b[a] >= 0 : a < nw;
            const R s0 = self ? rcp<R>(R(1)) : R(0);
            if constexpr (sizeof(R) == 4) sv = cf_add(sv, -(float)s0);
            else svd -= (double)s0;
            rowval[(size_t)w * nA + ia] = sizeof(R) == 4 ? cf_val(sv) : svd;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            tkw[tile] = 0u;
            last_x = atomicAdd(&tkw[ntile + nbchunk], 1u) == (unsigned)ntile - 1;
        }
        __syncthreads();
        if (last_x) {
            __threadfence();
            double v[1] = {0.0};
            for (int q = threadIdx.x; q < nA; q += CT_T) v[0] += __ldcg(rowval + (size_t)w * nA + q);
            block_sum<double, 1>(v);
            if (threadIdx.x == 0) {
                xi[w * 4 + col] = scw[w] * v[0];
                tkw[ntile + nbchunk] = 0u;
            }
        }
    }
    if (last_col) {
        __threadfence();
        for (int q = threadIdx.x; q < mb; q += CT_T) {
            R sx = 0, sy = 0, sz = 0;
            for (int t0 = 0; t0 < ntile; t0 += FB) {
                R4<R> u[FB];
#pragma unroll
                for (int k = 0; k < FB; ++k)
                    if (t0 + k < ntile) u[k] = ldcg_r4<R>(colpart + ((size_t)w * ntile + t0 + k) * nB_stride + b0 + q);
#pragma unroll
                for (int k = 0; k < FB; ++k)
                    if (t0 + k < ntile) {
                        sx += u[k].x;
                        sy += u[k].y;
                        sz += u[k].z;
                    }
            }
            const int j = sid[q];
            atomicAdd(&J[o + j].x, f * sx);
            atomicAdd(&J[o + j].y, f * sy);
            atomicAdd(&J[o + j].z, f * sz);
        }
        if (threadIdx.x == 0) tkw[ntile + chunk] = 0u;
    }
}

template <int HC>
__global__ void __launch_bounds__(CT_T) coord_tile2_kernel(const float4* __restrict__ pos,
                                                           const int64_t* __restrict__ woff,
                                                           const int* __restrict__ wn, const int* __restrict__ A,
                                                           int nA, const int* __restrict__ B, int nB, int nbchunk,
                                                           Box box, float inv_r0sq, int h, float gpref,
                                                           float4* __restrict__ rowpart, float4* __restrict__ colpart,
                                                           int nB_stride, const double* __restrict__ scw,
                                                           double* __restrict__ xi, int col,
                                                           const int* __restrict__ inv_b, double xq, double ixq)
{
    __shared__ float4 srcA[CT_B], srcB[CT_B];
    __shared__ float4 rowred[CT_T / 32][C2_A];
    __shared__ double xred[2];
    pdl_trigger();  // the hills sum that follows may start its hill copies now
    const int w = blockIdx.y;
    const int ntile = gridDim.x / nbchunk;
    CoordTile2 t{pos + woff[w], wn[w], A, nA, B, nB, nbchunk, ntile, box, inv_r0sq, h, gpref,
                 rowpart + (size_t)w * nbchunk * nA, colpart + (size_t)w * ntile * nB_stride, nB_stride, scw[w],
                 xi + w * 4 + col, inv_b, xq, ixq};
    coord_tile2_body<HC>(t, (int)blockIdx.x / nbchunk, (int)blockIdx.x % nbchunk, (int)threadIdx.x, srcA, srcB, rowred,
                         xred, [] { pdl_wait(); }, [] { __syncthreads(); });
}

// Coordination tiles with the radius of gyration of another CV in the same
// launch: CTAs x < ntile * nbchunk take the tiles, CTA x = ntile * nbchunk of
// each walker the Rg group.  The hills sum, which needs both CVs, then
// depends on one launch, and that launch lets its dependents start at once.
constexpr size_t C2_SMEM = sizeof(float4) * (2 * CT_B + (CT_T / 32) * C2_A) + 2 * sizeof(double);
constexpr size_t C2RG_SMEM = C2_SMEM > sizeof(float4) * RG_CACHE ? C2_SMEM : sizeof(float4) * RG_CACHE;

template <int HC>
__global__ void __launch_bounds__(CT_T) coord_tile2_rg_kernel(const float4* __restrict__ pos,
                                                              const int64_t* __restrict__ woff,
                                                              const int* __restrict__ wn, const int* __restrict__ A,
                                                              int nA, const int* __restrict__ B, int nB, int nbchunk,
                                                              Box box, float inv_r0sq, int h, float gpref,
                                                              float4* __restrict__ rowpart,
                                                              float4* __restrict__ colpart, int nB_stride,
                                                              const double* __restrict__ scw, double* __restrict__ xi,
                                                              int col, const int* __restrict__ inv_b, double xq,
                                                              double ixq, const int* __restrict__ rA, int rnA,
                                                              double rscale, int rintensive, int rcol,
                                                              float4* __restrict__ rJ)
{
    __shared__ __align__(16) unsigned char sm[C2RG_SMEM];
    pdl_trigger();  // the hills sum that follows may start its hill copies now
    const int w = blockIdx.y;
    const int ntc = (int)gridDim.x - 1;  // tile CTAs of the walker
    if ((int)blockIdx.x == ntc) {
        cv_rg_body<float>(w, pos, woff, wn, rA, rnA, box, rscale, rintensive, xi, rcol, rJ, reinterpret_cast<float4*>(sm),
                          [] { pdl_wait(); });
        return;
    }
    float4* srcA = reinterpret_cast<float4*>(sm);
    float4* srcB = srcA + CT_B;
    float4(*rowred)[C2_A] = reinterpret_cast<float4(*)[C2_A]>(srcB + CT_B);
    double* xred = reinterpret_cast<double*>(rowred + CT_T / 32);
    const int ntile = ntc / nbchunk;
    CoordTile2 t{pos + woff[w], wn[w], A, nA, B, nB, nbchunk, ntile, box, inv_r0sq, h, gpref,
                 rowpart + (size_t)w * nbchunk * nA, colpart + (size_t)w * ntile * nB_stride, nB_stride, scw[w],
                 xi + w * 4 + col, inv_b, xq, ixq};
    coord_tile2_body<HC>(t, (int)blockIdx.x / nbchunk, (int)blockIdx.x % nbchunk, (int)threadIdx.x, srcA, srcB, rowred,
                         xred, [] { pdl_wait(); }, [] { __syncthreads(); });
}

// The Rg CV whose group rides along in the launch of the FP32 tile
// coordination CV 0 (coord_tile2_rg_kernel), or -1.
int folded_rg(const wtmd_t* h)
{
    if (h->ncv < 2 || !coord_factored(h, 0)) return -1;
    for (int c = 1; c < h->ncv; ++c)
        if (h->cv[c].kind == WTMD_CV_RG) return c;
    return -1;
}

// J rows of an FP32 tile coordination CV for every atom (0 for atoms in
// neither group).
// A programmatic dependent of the tile kernel: the atom's walker and local
// index are read first, then the partials are waited for.
__global__ void coord_jfin_kernel(long long N, const int* __restrict__ aw, const int64_t* __restrict__ woff,
                                  CoordParts p, float4* __restrict__ J)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    // the atom's walker, its positions in the two groups and the walker's
    // scale are constant: read before the wait
    int w = 0, pb = -1, ia = -1;
    float f = 0.f;
    if (i < N) {
        w = aw[i];
        const int li = (int)(i - woff[w]);
        pb = p.inv_b ? p.inv_b[li] : li;
        ia = p.inv_a[li];
        f = (float)p.scw[w];
    }
    pdl_wait();
    if (i < N) J[i] = coord_j_parts_at(p, w, pb, ia, f);
}

// J rows and the CV value from the tile partials.  Thread k sums the chunk
// partials of its row (k in A; also its row value of s, stored per member)
// and the tile partials of its column (k in B); the walker's last CTA sums
// the per-member row values in member order.

// ---------------------------------------------------------------------------
// Q-like pair count: xi = scale * sum_p s(r_{i_p j_p}) over a fixed list.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void qpair_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff, const int* __restrict__ pl,
                             int np, Box box, R inv_r0sq, int h, R gpref, R4<R>* __restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (p >= np) return;
    const long long o = woff[w];
    R ax, ay, az, bx, by, bz, d[3];
    load3<R>(pos, o + pl[2 * p], ax, ay, az);
    load3<R>(pos, o + pl[2 * p + 1], bx, by, bz);
    delta<R>(box, ax, ay, az, bx, by, bz, d);
    const R y = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * inv_r0sq;
    const R yh1 = ypow<R>(y, h - 1);
    const R sv = R(1) / (R(1) + yh1 * y);
    const R gr = gpref * yh1 * sv * sv;
    out[(size_t)w * np + p] = mk4<R>(gr * d[0], gr * d[1], gr * d[2], sv);
}

template <typename R>
__global__ void qpair_jac_kernel(const int64_t* __restrict__ woff, const int* __restrict__ wn,
                                 const int* __restrict__ rowptr, const int* __restrict__ items, int np,
                                 const R4<R>* __restrict__ pv, double sc, R4<R>* __restrict__ J)
{
    const int w = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= wn[w]) return;
    const int b = rowptr[k], e = rowptr[k + 1];
    if (b == e) return;
    double gx = 0, gy = 0, gz = 0;
    for (int q = b; q < e; ++q) {
        const int it = items[q];
        const R4<R> v = pv[(size_t)w * np + (it >> 1)];
        const double sg = (it & 1) ? -1.0 : 1.0;
        gx += sg * v.x;
        gy += sg * v.y;
        gz += sg * v.z;
    }
    J[woff[w] + k] = mk4<R>((R)(sc * gx), (R)(sc * gy), (R)(sc * gz), R(0));
}

template <typename R>
__global__ void __launch_bounds__(256) qpair_value_kernel(const R4<R>* __restrict__ pv, int np, double sc,
                                                          double* __restrict__ xi, int col)
{
    const int w = blockIdx.x;
    double v[1] = {0.0};
    for (int p = threadIdx.x; p < np; p += blockDim.x) v[0] += (double)pv[(size_t)w * np + p].w;
    block_sum<double, 1>(v);
    if (threadIdx.x == 0) xi[w * 4 + col] = sc * v[0];
}

// ---------------------------------------------------------------------------
// Bias-force scatter: F_i -= sum_c dV/dxi_c(w(i)) J_c[i]; optionally the
// closing half kick v += dt/2 F/m of BAOAB.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void scatter_atom(long long i, int d, const int* __restrict__ aw, const R* __restrict__ dV,
                                             const R4<R>* __restrict__ J, long long N, R4<R>* __restrict__ force,
                                             R4<R>* __restrict__ vel, R half_dt_over_m, int dims)
{
    const int w = aw[i];
    R4<R> f = force[i];
    for (int c = 0; c < d; ++c) {
        const R g = dV[w * 4 + c];
        const R4<R> j = J[(size_t)c * N + i];
        f.x -= g * j.x;
        f.y -= g * j.y;
        f.z -= g * j.z;
    }
    force[i] = f;
    if (vel) {
        R4<R> v = vel[i];
        v.x += half_dt_over_m * f.x;
        v.y += half_dt_over_m * f.y;
        if (dims > 2) v.z += half_dt_over_m * f.z;
        vel[i] = v;
    }
}

// Closing half-kick of the step fused with the deposition: the last block
// first deposits (reads xi and V, appends hills, advances the step counter),
// then every block scatters its atoms' bias forces and kicks.
template <typename R>
__global__ void __launch_bounds__(256) scatter_deposit_kernel(long long N, int d, const int* __restrict__ aw,
                                                              const R* __restrict__ dV, const R4<R>* __restrict__ J,
                                                              R4<R>* __restrict__ force, R4<R>* __restrict__ vel,
                                                              R half_dt_over_m, int dims, DepPrm dp,
                                                              const double* __restrict__ xi, const R* __restrict__ V,
                                                              long long* count, long long* step, long long* dep,
                                                              double* ctr, dbl4* h64, float* h32, unsigned* status,
                                                              int* __restrict__ ccount, int ncells,
                                                              unsigned* __restrict__ nl_ctl)
{
    // Launched as a programmatic dependent of the hills sum: the velocity
    // (written by the previous step) is loaded first; the force and the
    // Jacobian rows, which come from graph branches that this launch joins
    // (joined edges are programmatic too), and dV/dxi, V and xi after the
    // wait.
    // It also resets the engine's cell counts and neighbour-list rebuild
    // flag (the engine branch has joined).
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < N;
    int w = 0;
    R4<R> f = mk4<R>(0, 0, 0, 0), v = f, jr[3] = {f, f, f};
    if (act) {
        w = aw[i];
        v = vel[i];
    }
    // the deposit's step counter, hill count and layout centre change only
    // in this kernel (the previous step's launch has completed): read them
    // before the wait
    __shared__ long long dpre[2];
    __shared__ double dcpre[3];
    const bool dep_block = blockIdx.x == gridDim.x - 1;
    if (dep_block && threadIdx.x == 0) {
        dpre[0] = *step;
        dpre[1] = *count;
        for (int k = 0; k < 3; ++k) dcpre[k] = ctr[k];
    }
    pdl_wait();
    // every load of the update first (one round trip to L2 for all of them)
    R g[3] = {R(0), R(0), R(0)};
    if (act) {
        f = force[i];
        for (int c = 0; c < d && c < 3; ++c) {
            jr[c] = J[(size_t)c * N + i];
            g[c] = dV[w * 4 + c];
        }
    }
    // after the wait: the engine's list build may still be reading the
    // counts until then (a joined edge lets this launch start early)
    for (long long c = i; c < ncells; c += (long long)gridDim.x * blockDim.x) ccount[c] = 0;
    if (nl_ctl && i == 0) *nl_ctl = 0u;
    if (dep_block) deposit_block_at<R>(dp, dpre, dcpre, xi, V, count, step, dep, ctr, h64, h32, status);
    if (!act) return;
    for (int c = 0; c < d && c < 3; ++c) {
        f.x -= g[c] * jr[c].x;
        f.y -= g[c] * jr[c].y;
        f.z -= g[c] * jr[c].z;
    }
    force[i] = f;
    v.x += half_dt_over_m * f.x;
    v.y += half_dt_over_m * f.y;
    if (dims > 2) v.z += half_dt_over_m * f.z;
    vel[i] = v;
}

template <typename R>
__global__ void scatter_kernel(long long N, int d, const int* __restrict__ aw, const R* __restrict__ dV,
                               const R4<R>* __restrict__ J, R4<R>* __restrict__ force, R4<R>* __restrict__ vel,
                               R half_dt_over_m, int dims)
{
    pdl_wait();  // a programmatic dependent of the bias sum: everything it reads comes after the wait
    pdl_trigger();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) scatter_atom<R>(i, d, aw, dV, J, N, force, vel, half_dt_over_m, dims);
}

// ---------------------------------------------------------------------------
// Adjoint of the CV map (the paper differentiates CVs with jax.grad, Sec. 2):
// grad_r[i] = sum_c grad_xi[w(i)][c] J_c[i] for an arbitrary upstream
// grad_xi [W][d]; with grad_xi = -dV/dxi this is the bias force.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void cv_adjoint_kernel(long long N, int d, const int* __restrict__ aw, const R* __restrict__ gxi,
                                  const R4<R>* __restrict__ J, R4<R>* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int w = aw[i];
    R gx = 0, gy = 0, gz = 0;
    for (int c = 0; c < d; ++c) {
        const R g = gxi[(size_t)w * d + c];
        const R4<R> j = J[(size_t)c * N + i];
        gx += g * j.x;
        gy += g * j.y;
        gz += g * j.z;
    }
    out[i] = mk4<R>(gx, gy, gz, R(0));
}

int launch_adjoint(wtmd_t* h, const void* grad_xi, void* grad_pos)
{
    const int nb = (int)((h->N + 255) / 256);
    if (h->prec == WTMD_F32)
        cv_adjoint_kernel<float><<<nb, 256, 0, h->stream>>>(h->N, h->d, h->atom_walker, (const float*)grad_xi,
                                                            (const float4*)h->J, (float4*)grad_pos);
    else
        cv_adjoint_kernel<double><<<nb, 256, 0, h->stream>>>(h->N, h->d, h->atom_walker, (const double*)grad_xi,
                                                             (const dbl4*)h->J, (dbl4*)grad_pos);
    mark(h, "cv_adjoint");
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int cv_alloc_scratch(wtmd_t* h, CvDev& c)
{
    const size_t r4 = h->prec == WTMD_F32 ? sizeof(float4) : sizeof(dbl4);
    if (c.kind == WTMD_CV_COORDINATION) {
        const int nA = c.n_a < 0 ? h->max_wn : c.n_a;
        c.nT_row = nA;  // row-value stride per walker
        WTMD_CUDA_TRY(h, cudaMalloc(&c.part_row, sizeof(double) * (size_t)h->W * nA));
        WTMD_CUDA_TRY(h, cudaMalloc(&c.part_col, sizeof(unsigned) * (size_t)h->W));
        WTMD_CUDA_TRY(h, cudaMemset(c.part_col, 0, sizeof(unsigned) * (size_t)h->W));
        // per-walker CV scale (default 1/|A|, |A| = walker size for "all")
        std::vector<double> scw(h->W);
        for (int w = 0; w < h->W; ++w)
            scw[w] = c.scale != 0.0 ? c.scale : 1.0 / (double)(c.n_a < 0 ? h->wn_h[w] : c.n_a);
        WTMD_CUDA_TRY(h, cudaMalloc(&c.scw, sizeof(double) * (size_t)h->W));
        if (c.n_a > 0) {  // tile path: row partials [W][chunk][A], column partials [W][tile][B]
            const int nB = c.n_b < 0 ? h->max_wn : c.n_b;
            c.nbchunk = (nB + 255) / 256;
            c.ntile = (c.n_a + 31) / 32;
            c.nB_stride = nB;
            // bound of |xi| over the walkers (every s <= 1)
            c.xi_bound = 0.0;
            for (int w = 0; w < h->W; ++w)
                c.xi_bound = std::max(c.xi_bound, std::fabs(scw[w]) * c.n_a * (c.n_b < 0 ? h->wn_h[w] : c.n_b));
            WTMD_CUDA_TRY(h, cudaMalloc(&c.tile_row, r4 * (size_t)h->W * c.nbchunk * c.n_a));
            WTMD_CUDA_TRY(h, cudaMalloc(&c.tile_col, r4 * (size_t)h->W * c.ntile * nB));
            const size_t ntk = (size_t)h->W * (c.ntile + c.nbchunk + 1);
            WTMD_CUDA_TRY(h, cudaMalloc(&c.tile_tk, sizeof(unsigned) * ntk));
            WTMD_CUDA_TRY(h, cudaMemset(c.tile_tk, 0, sizeof(unsigned) * ntk));
        }
        WTMD_CUDA_TRY(h, cudaMemcpy(c.scw, scw.data(), sizeof(double) * (size_t)h->W, cudaMemcpyHostToDevice));
    } else if (c.kind == WTMD_CV_QPAIRS) {
        WTMD_CUDA_TRY(h, cudaMalloc(&c.part_row, r4 * (size_t)h->W * c.n_pairs));
    }
    return WTMD_OK;
}

static CoordParts coord_parts(const wtmd_t* h, const CvDev& cv)
{
    CoordParts p;
    p.rowpart = (const float4*)cv.tile_row;
    p.colpart = (const float4*)cv.tile_col;
    p.inv_a = cv.inv_a;
    p.inv_b = cv.n_b < 0 ? nullptr : cv.inv_b;
    p.scw = cv.scw;
    p.nA = cv.n_a;
    p.nbchunk = cv.nbchunk;
    p.ntile = (cv.n_a + C2_A - 1) / C2_A;
    p.nB_stride = cv.nB_stride;
    return p;
}

bool coord_factored(const wtmd_t* h, int c)
{
    return h->prec == WTMD_F32 && h->cv[c].kind == WTMD_CV_COORDINATION && h->cv[c].n_a > 0;
}

template <typename R> static int launch_cvs_t(wtmd_t* h, const void* pos_, int c_begin, int c_end)
{
    const R4<R>* pos = (const R4<R>*)pos_;
    double* xi = h->xi;
    R4<R>* J = (R4<R>*)h->J;
    const int W = h->W;
    cudaStream_t st = h->stream;
    for (int c = c_begin; c < c_end; ++c) {
        CvDev& cv = h->cv[c];
        R4<R>* Jc = J + (size_t)c * h->N;
        const R sc = (R)(cv.scale != 0.0 ? cv.scale : 1.0);
        switch (cv.kind) {
        case WTMD_CV_COMPONENT:
            cv_component_kernel<R><<<(W + 127) / 128, 128, 0, st>>>(pos, h->woff, W, cv.hidx[0], cv.axis, sc,
                                                                     xi, c, Jc);
            mark(h, "cv_component");
            break;
        case WTMD_CV_DIHEDRAL: {
            const int4 q = make_int4(cv.hidx[0], cv.hidx[1], cv.hidx[2], cv.hidx[3]);
            cv_dihedral_kernel<R><<<(W + 127) / 128, 128, 0, st>>>(pos, h->woff, W, q, h->box, sc, xi, c, Jc);
            mark(h, "cv_dihedral");
            break;
        }
        case WTMD_CV_DISTANCE:
            cv_distance_kernel<R><<<W, 256, 0, st>>>(pos, h->woff, cv.a, cv.n_a, cv.b, cv.n_b, h->box, sc, xi, c, Jc);
            mark(h, "cv_distance");
            break;
        case WTMD_CV_ANGLE:
            cv_angle_kernel<R><<<(W + 127) / 128, 128, 0, st>>>(
                pos, h->woff, W, make_int3(cv.hidx[0], cv.hidx[1], cv.hidx[2]), h->box, sc, xi, c, Jc);
            mark(h, "cv_angle");
            break;
        case WTMD_CV_GYRATION:
            cv_gyration_kernel<R><<<W, 256, 0, st>>>(pos, h->woff, h->wn, cv.n_a < 0 ? nullptr : cv.a, cv.n_a, h->box,
                                                     cv.axis, cv.scale != 0.0 ? cv.scale : 1.0, xi, c, Jc);
            mark(h, "cv_gyration");
            break;
        case WTMD_CV_RG:
            if (c == folded_rg(h)) break;  // computed by the launch of CV 0
            WTMD_CUDA_TRY(h, launch_pdl(cv_rg_kernel<R>, dim3(W), dim3(256), 0, st, pos, (const int64_t*)h->woff,
                                        (const int*)h->wn, (const int*)(cv.n_a < 0 ? nullptr : cv.a), (int)cv.n_a,
                                        h->box, cv.scale, (int)(cv.flags & WTMD_CV_INTENSIVE), xi, c, Jc));
            mark(h, "cv_rg");
            break;
        case WTMD_CV_COORDINATION: {
            const R inv = (R)(1.0 / (cv.r0 * cv.r0));
            const R gp = (R)(-(double)cv.nn / (cv.r0 * cv.r0));
            const int* A = cv.n_a < 0 ? nullptr : cv.a;
            const int* B = cv.n_b < 0 ? nullptr : cv.b;
            if (cv.n_a > 0) {
                if constexpr (sizeof(R) == 4) {
                    // FP32: the CV value accumulates in xi, which starts at 0
                    // (the step's BAOAB kernel zeroes it)
                    if (!h->jz_pre)
                        WTMD_CUDA_TRY(h, cudaMemset2DAsync(xi + c, 4 * sizeof(double), 0, sizeof(double), W, st));
                    // shares are multiples of 2^-q with |xi| < 2^(53-q) for every walker
                    const int q = 50 - std::max(0, (int)std::ceil(std::log2(std::max(cv.xi_bound, 1.0))));
                    dim3 g2(((cv.n_a + C2_A - 1) / C2_A) * cv.nbchunk, W);
                    const int rgc = c == 0 ? folded_rg(h) : -1;
                    if (rgc >= 0) {
                        const CvDev& rg = h->cv[rgc];
                        g2.x += 1;
                        auto k2 = cv.nn == 6 ? coord_tile2_rg_kernel<3> : coord_tile2_rg_kernel<0>;
                        WTMD_CUDA_TRY(h, launch_pdl(k2, g2, dim3(CT_T), 0, st, pos, (const int64_t*)h->woff,
                                                    (const int*)h->wn, A, cv.n_a, B, cv.n_b, cv.nbchunk, h->box, inv,
                                                    cv.nn / 2, gp, (float4*)cv.tile_row, (float4*)cv.tile_col,
                                                    cv.nB_stride, (const double*)cv.scw, xi, c,
                                                    (const int*)(cv.n_b < 0 ? nullptr : cv.inv_b), std::ldexp(1.0, q),
                                                    std::ldexp(1.0, -q), (const int*)(rg.n_a < 0 ? nullptr : rg.a),
                                                    (int)rg.n_a, rg.scale, (int)(rg.flags & WTMD_CV_INTENSIVE), rgc,
                                                    (float4*)(J + (size_t)rgc * h->N)));
                    } else {
                        auto k2 = cv.nn == 6 ? coord_tile2_kernel<3> : coord_tile2_kernel<0>;
                        WTMD_CUDA_TRY(h, launch_pdl(k2, g2, dim3(CT_T), 0, st, pos, (const int64_t*)h->woff,
                                                    (const int*)h->wn, A, cv.n_a, B, cv.n_b, cv.nbchunk, h->box, inv,
                                                    cv.nn / 2, gp, (float4*)cv.tile_row, (float4*)cv.tile_col,
                                                    cv.nB_stride, (const double*)cv.scw, xi, c,
                                                    (const int*)(cv.n_b < 0 ? nullptr : cv.inv_b), std::ldexp(1.0, q),
                                                    std::ldexp(1.0, -q)));
                    }
                    mark(h, "coord_tile");
                    // J rows from the partials.  In a captured step this is
                    // a graph branch of its own beside the hills sum, which
                    // needs only xi; the closing kick joins it.
                    cudaStream_t js = st;
                    const bool branch = (h->jz_pre || h->jbranch) && !h->prof;
                    if (branch) {
                        WTMD_CUDA_TRY(h, cudaEventRecord(h->ev_jfork[c], st));
                        WTMD_CUDA_TRY(h, cudaStreamWaitEvent(h->jf_stream[c], h->ev_jfork[c], 0));
                        js = h->jf_stream[c];
                    }
                    WTMD_CUDA_TRY(h, launch_pdl(coord_jfin_kernel, dim3((unsigned)((h->N + 255) / 256)), dim3(256), 0,
                                                js, (long long)h->N, (const int*)h->atom_walker,
                                                (const int64_t*)h->woff, coord_parts(h, cv), (float4*)Jc));
                    mark(h, "coord_jfin");
                    if (branch) {
                        WTMD_CUDA_TRY(h, cudaEventRecord(h->ev_jjoin[c], js));
                        h->jf_pending |= 1 << c;
                    }
                    break;
                }
                else {  // FP64: the generic tile kernel, finalized in-launch
                    if (!h->jz_pre) WTMD_CUDA_TRY(h, cudaMemsetAsync(Jc, 0, sizeof(R4<R>) * (size_t)h->N, st));
                    dim3 gt(cv.ntile * cv.nbchunk, W);
                    // programmatic dependent of the kernel that moved the positions
                    auto kern = cv.nn == 6 ? coord_tile_kernel<R, 3> : coord_tile_kernel<R, 0>;
                    WTMD_CUDA_TRY(h, launch_pdl(kern, gt, dim3(CT_T), 0, st, pos, (const int64_t*)h->woff,
                                                (const int*)h->wn, A, cv.n_a, B, cv.n_b, cv.nbchunk, h->box, inv,
                                                cv.nn / 2, gp, (R4<R>*)cv.tile_row, (R4<R>*)cv.tile_col,
                                                cv.nB_stride, (const double*)cv.scw, (double*)cv.part_row,
                                                cv.tile_tk, Jc, xi, c, (const int*)(cv.n_b < 0 ? nullptr : cv.inv_b)));
                    mark(h, "coord_tile");
                    break;
                }
            }
            const int nt = cv.order ? cv.n_order : h->max_wn;
            // a short list A against many partners: one CTA per member of A
            const int nBmax = cv.n_b < 0 ? h->max_wn : cv.n_b;
            const int ab = (cv.order && nBmax >= 1024) ? (cv.n_a + CW_G - 1) / CW_G : 0;
            const int nrest = nt - (ab > 0 ? cv.n_a : 0);
            dim3 g(ab + (nrest + CW_T / 32 - 1) / (CW_T / 32), W);
            coord_warp_kernel<R><<<g, CW_T, 0, st>>>(pos, h->woff, h->wn, A, cv.n_a, B, cv.n_b, cv.inv_a, cv.inv_b,
                                                     cv.order, cv.n_order, ab, cv.same_ab ? 1 : 0, h->box, inv,
                                                     cv.nn / 2, gp, cv.scale,
                                                     cv.scw, (double*)cv.part_row, cv.nT_row, (unsigned*)cv.part_col,
                                                     Jc, xi,
                                                     c);
            mark(h, "coord_warp");
            break;
        }
        case WTMD_CV_QPAIRS: {
            const R inv = (R)(1.0 / (cv.r0 * cv.r0));
            const R gp = (R)(-(double)cv.nn / (cv.r0 * cv.r0));
            const double sc2 = cv.scale != 0.0 ? cv.scale : 1.0 / cv.n_pairs;
            dim3 g1((cv.n_pairs + 127) / 128, W);
            qpair_kernel<R><<<g1, 128, 0, st>>>(pos, h->woff, cv.a, cv.n_pairs, h->box, inv, cv.nn / 2, gp,
                                                (R4<R>*)cv.part_row);
            mark(h, "qpair");
            dim3 g2((h->max_wn + 255) / 256, W);
            qpair_jac_kernel<R><<<g2, 256, 0, st>>>(h->woff, h->wn, cv.q_rowptr, cv.q_items, cv.n_pairs,
                                                    (const R4<R>*)cv.part_row, sc2, Jc);
            mark(h, "qpair_jac");
            qpair_value_kernel<R><<<W, 256, 0, st>>>((const R4<R>*)cv.part_row, cv.n_pairs, sc2, xi, c);
            mark(h, "qpair_value");
            break;
        }
        default:
            h->err = "unknown CV kind";
            return WTMD_EINVAL;
        }
    }
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

int launch_cv(wtmd_t* h, const void* pos, int c)
{
    return h->prec == WTMD_F32 ? launch_cvs_t<float>(h, pos, c, c + 1) : launch_cvs_t<double>(h, pos, c, c + 1);
}

int launch_cvs(wtmd_t* h, const void* pos)
{
    return h->prec == WTMD_F32 ? launch_cvs_t<float>(h, pos, 0, h->ncv) : launch_cvs_t<double>(h, pos, 0, h->ncv);
}

int join_jbranches(wtmd_t* h)
{
    for (int c = 0; c < 3; ++c)
        if (h->jf_pending >> c & 1) WTMD_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_jjoin[c], 0));
    h->jf_pending = 0;
    return WTMD_OK;
}

int launch_scatter_deposit(wtmd_t* h)
{
    const int nb = (int)((h->N + 255) / 256);
    // join the J branches of the FP32 coordination CVs
    int rc = join_jbranches(h);
    if (rc) return rc;
    const double hdm = 0.5 * h->cfg.dt / h->cfg.mass;
    const DepPrm dp = dep_prm(h);
    // programmatic dependent of the hills sum (or of the network's part)
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, launch_pdl(scatter_deposit_kernel<float>, dim3(nb), dim3(256), 0, h->stream, h->N, h->d,
                                    (const int*)h->atom_walker, (const float*)h->dV, (const float4*)h->J,
                                    (float4*)h->force, (float4*)h->vel, (float)hdm, h->dims, dp, (const double*)h->xi,
                                    (const float*)h->V, h->count, h->step, h->dep, h->ctr, (dbl4*)h->hills64,
                                    (float*)h->hills32, h->status, h->cell_count, h->ncells, h->nl_ctl));
    else
        WTMD_CUDA_TRY(h, launch_pdl(scatter_deposit_kernel<double>, dim3(nb), dim3(256), 0, h->stream, h->N, h->d,
                                    (const int*)h->atom_walker, (const double*)h->dV, (const dbl4*)h->J,
                                    (dbl4*)h->force, (dbl4*)h->vel, hdm, h->dims, dp, (const double*)h->xi,
                                    (const double*)h->V, h->count, h->step, h->dep, h->ctr, (dbl4*)h->hills64,
                                    (float*)h->hills32, h->status, h->cell_count, h->ncells, h->nl_ctl));
    mark(h, "scatter_kick_deposit");
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return launch_grid_update(h);
}

int launch_scatter(wtmd_t* h, void* force, const void* vel, bool kick)
{
    const int nb = (int)((h->N + 255) / 256);
    const double hdm = 0.5 * h->cfg.dt / h->cfg.mass;
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, launch_pdl(scatter_kernel<float>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N, h->d,
                                    (const int*)h->atom_walker, (const float*)h->dV, (const float4*)h->J,
                                    (float4*)force, kick ? (float4*)vel : (float4*)nullptr, (float)hdm, h->dims));
    else
        WTMD_CUDA_TRY(h, launch_pdl(scatter_kernel<double>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N, h->d,
                                    (const int*)h->atom_walker, (const double*)h->dV, (const dbl4*)h->J,
                                    (dbl4*)force, kick ? (dbl4*)vel : (dbl4*)nullptr, hdm, h->dims));
    mark(h, "scatter_kick");
    return WTMD_OK;
}

}  // namespace wtmd
