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
#include "wtmd_internal.cuh"

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
template <typename R>
__global__ void __launch_bounds__(256) cv_rg_kernel(const R4<R>* __restrict__ pos, const int64_t* __restrict__ woff,
                                                    const int* __restrict__ wn, const int* __restrict__ A, int nA,
                                                    Box box, double scale, int intensive, double* __restrict__ xi, int col,
                                                    R4<R>* __restrict__ J)
{
    const int w = blockIdx.x;
    const long long o = woff[w];
    const int m = A ? nA : wn[w];
    const int i0 = A ? A[0] : 0;
    R rx, ry, rz;
    load3<R>(pos, o + i0, rx, ry, rz);
    double s[3] = {0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = A ? A[p] : p;
        R x, y, z, d[3];
        load3<R>(pos, o + i, x, y, z);
        delta<R>(box, x, y, z, rx, ry, rz, d);
        s[0] += (double)(rx + d[0]);
        s[1] += (double)(ry + d[1]);
        s[2] += (double)(rz + d[2]);
    }
    block_sum<double, 3>(s);
    const R c[3] = {(R)(s[0] / m), (R)(s[1] / m), (R)(s[2] / m)};
    double q[1] = {0.0};
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = A ? A[p] : p;
        R x, y, z, d[3];
        load3<R>(pos, o + i, x, y, z);
        delta<R>(box, x, y, z, rx, ry, rz, d);
        const R ux = rx + d[0] - c[0], uy = ry + d[1] - c[1], uz = rz + d[2] - c[2];
        q[0] += (double)(ux * ux + uy * uy + uz * uz);
    }
    block_sum<double, 1>(q);
    const double rg = sqrt(q[0] / m);
    double sc = scale != 0.0 ? scale : 1.0;
    if (intensive) sc /= cbrt((double)m);
    const R f = (R)(sc / (m * rg));
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = A ? A[p] : p;
        R x, y, z, d[3];
        load3<R>(pos, o + i, x, y, z);
        delta<R>(box, x, y, z, rx, ry, rz, d);
        J[o + i] = mk4<R>(f * (rx + d[0] - c[0]), f * (ry + d[1] - c[1]), f * (rz + d[2] - c[2]), R(0));
    }
    if (threadIdx.x == 0) xi[w * 4 + col] = sc * rg;
}

// ---------------------------------------------------------------------------
// Switching-function pair sums.  s(r) = 1/(1 + y^h), y = r^2/r0^2, h = n/2
// (the rational (1-x^n)/(1-x^m) with m = 2n, which equals this exactly), and
// ds/dr_t = -(n/r0^2) y^(h-1) s^2 (r_t - r_s).
// pair_pass: for every target t of the walker, over one split of sources,
//   part = (sum_s ds/dr_t, sum_s s(r_ts)), self pairs excluded.
// ---------------------------------------------------------------------------
constexpr int PP_T = 128;  // targets per block
constexpr int PP_S = 128;  // sources per split

template <typename R>
__device__ __forceinline__ R ypow(R y, int h)
{
    R r = y;
    for (int k = 1; k < h; ++k) r *= y;
    return r;
}

template <typename R>
__global__ void __launch_bounds__(PP_T) pair_pass_kernel(const R4<R>* __restrict__ pos,
                                                         const int64_t* __restrict__ woff, const int* __restrict__ wn,
                                                         const int* __restrict__ T, int nT, const int* __restrict__ S,
                                                         int nS, Box box, R inv_r0sq, int h, R gpref,
                                                         R4<R>* __restrict__ part, int nT_stride)
{
    __shared__ R4<R> src[PP_S];
    __shared__ int sid[PP_S];
    const int w = blockIdx.z;
    const int W = gridDim.z;
    const long long o = woff[w];
    const int nw = wn[w];
    const int nTw = T ? nT : nw;
    const int nSw = S ? nS : nw;
    const int s0 = blockIdx.y * PP_S;
    const int s1 = min(s0 + PP_S, nSw);
    for (int j = threadIdx.x; j < s1 - s0; j += blockDim.x) {
        const int li = S ? S[s0 + j] : s0 + j;
        src[j] = pos[o + li];
        sid[j] = li;
    }
    __syncthreads();
    const int t = blockIdx.x * PP_T + threadIdx.x;
    if (t >= nTw) return;
    const int ti = T ? T[t] : t;
    R tx, ty, tz;
    load3<R>(pos, o + ti, tx, ty, tz);
    R gx = 0, gy = 0, gz = 0, ss = 0;
    for (int j = 0; j < s1 - s0; ++j) {
        if (sid[j] == ti) continue;
        const R4<R> sp = src[j];
        R d[3];
        delta<R>(box, tx, ty, tz, sp.x, sp.y, sp.z, d);
        const R y = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * inv_r0sq;
        const R yh1 = ypow<R>(y, h - 1);
        const R sv = R(1) / (R(1) + yh1 * y);
        ss += sv;
        const R gr = gpref * yh1 * sv * sv;
        gx += gr * d[0];
        gy += gr * d[1];
        gz += gr * d[2];
    }
    part[((size_t)blockIdx.y * W + w) * nT_stride + t] = mk4<R>(gx, gy, gz, ss);
}

// J rows of coordination for every atom of every walker.
template <typename R>
__global__ void coord_finalize_kernel(const int64_t* __restrict__ woff, const int* __restrict__ wn, int W,
                                      const int* __restrict__ inv_a, bool a_all, const int* __restrict__ inv_b,
                                      bool b_all, bool same_ab, const R4<R>* __restrict__ prow, int split_row,
                                      int nT_row, const R4<R>* __restrict__ pcol, int split_col, int nT_col,
                                      double scale, int nA, R4<R>* __restrict__ J)
{
    const int w = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= wn[w]) return;
    const int pa = a_all ? k : inv_a[k];
    const int pb = b_all ? k : inv_b[k];
    if (pa < 0 && pb < 0) return;
    double gx = 0, gy = 0, gz = 0;
    if (pa >= 0)
        for (int s = 0; s < split_row; ++s) {
            const R4<R> q = prow[((size_t)s * W + w) * nT_row + pa];
            gx += q.x;
            gy += q.y;
            gz += q.z;
        }
    if (same_ab) {
        gx *= 2.0;
        gy *= 2.0;
        gz *= 2.0;
    } else if (pb >= 0) {
        for (int s = 0; s < split_col; ++s) {
            const R4<R> q = pcol[((size_t)s * W + w) * nT_col + pb];
            gx += q.x;
            gy += q.y;
            gz += q.z;
        }
    }
    const double sc = scale != 0.0 ? scale : 1.0 / (a_all ? wn[w] : nA);
    J[woff[w] + k] = mk4<R>((R)(sc * gx), (R)(sc * gy), (R)(sc * gz), R(0));
}

// xi = scale * sum over targets of group A of the row sums of s.
template <typename R>
__global__ void __launch_bounds__(256) coord_value_kernel(const int* __restrict__ wn, bool a_all, int nA,
                                                          const R4<R>* __restrict__ prow, int split_row, int nT_row,
                                                          double scale, double* __restrict__ xi, int col)
{
    const int w = blockIdx.x;
    const int W = gridDim.x;
    const int na = a_all ? wn[w] : nA;
    double v[1] = {0.0};
    for (int t = threadIdx.x; t < na; t += blockDim.x) {
        double r = 0.0;
        for (int s = 0; s < split_row; ++s) r += prow[((size_t)s * W + w) * nT_row + t].w;
        v[0] += r;
    }
    block_sum<double, 1>(v);
    const double sc = scale != 0.0 ? scale : 1.0 / na;
    if (threadIdx.x == 0) xi[w * 4 + col] = sc * v[0];
}

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
__global__ void scatter_kernel(long long N, int d, const int* __restrict__ aw, const R* __restrict__ dV,
                               const R4<R>* __restrict__ J, R4<R>* __restrict__ force, R4<R>* __restrict__ vel,
                               R half_dt_over_m, int dims)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int cv_alloc_scratch(wtmd_t* h, CvDev& c)
{
    const size_t r4 = h->prec == WTMD_F32 ? sizeof(float4) : sizeof(dbl4);
    if (c.kind == WTMD_CV_COORDINATION) {
        const int nA = c.n_a < 0 ? h->max_wn : c.n_a;
        const int nB = c.n_b < 0 ? h->max_wn : c.n_b;
        c.nT_row = nA;
        c.split_row = (nB + PP_S - 1) / PP_S;
        WTMD_CUDA_TRY(h, cudaMalloc(&c.part_row, r4 * (size_t)c.split_row * h->W * c.nT_row));
        if (!c.same_ab) {
            c.nT_col = nB;
            c.split_col = (nA + PP_S - 1) / PP_S;
            WTMD_CUDA_TRY(h, cudaMalloc(&c.part_col, r4 * (size_t)c.split_col * h->W * c.nT_col));
        }
    } else if (c.kind == WTMD_CV_QPAIRS) {
        WTMD_CUDA_TRY(h, cudaMalloc(&c.part_row, r4 * (size_t)h->W * c.n_pairs));
    }
    return WTMD_OK;
}

template <typename R> static int launch_cvs_t(wtmd_t* h, const void* pos_)
{
    const R4<R>* pos = (const R4<R>*)pos_;
    double* xi = h->xi;
    R4<R>* J = (R4<R>*)h->J;
    const int W = h->W;
    cudaStream_t st = h->stream;
    for (int c = 0; c < h->ncv; ++c) {
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
        case WTMD_CV_RG:
            cv_rg_kernel<R><<<W, 256, 0, st>>>(pos, h->woff, h->wn, cv.n_a < 0 ? nullptr : cv.a, cv.n_a, h->box,
                                               cv.scale, cv.flags & WTMD_CV_INTENSIVE, xi, c, Jc);
            mark(h, "cv_rg");
            break;
        case WTMD_CV_COORDINATION: {
            const R inv = (R)(1.0 / (cv.r0 * cv.r0));
            const R gp = (R)(-(double)cv.nn / (cv.r0 * cv.r0));
            const int hh = cv.nn / 2;
            const int* A = cv.n_a < 0 ? nullptr : cv.a;
            const int* B = cv.n_b < 0 ? nullptr : cv.b;
            dim3 g1((cv.nT_row + PP_T - 1) / PP_T, cv.split_row, W);
            pair_pass_kernel<R><<<g1, PP_T, 0, st>>>(pos, h->woff, h->wn, A, cv.n_a, B, cv.n_b, h->box, inv, hh, gp,
                                                     (R4<R>*)cv.part_row, cv.nT_row);
            mark(h, "coord_pair_row");
            if (!cv.same_ab) {
                dim3 g2((cv.nT_col + PP_T - 1) / PP_T, cv.split_col, W);
                pair_pass_kernel<R><<<g2, PP_T, 0, st>>>(pos, h->woff, h->wn, B, cv.n_b, A, cv.n_a, h->box, inv, hh,
                                                         gp, (R4<R>*)cv.part_col, cv.nT_col);
                mark(h, "coord_pair_col");
            }
            dim3 g3((h->max_wn + 255) / 256, W);
            coord_finalize_kernel<R><<<g3, 256, 0, st>>>(h->woff, h->wn, W, cv.inv_a, cv.n_a < 0, cv.inv_b,
                                                         cv.n_b < 0, cv.same_ab, (const R4<R>*)cv.part_row,
                                                         cv.split_row, cv.nT_row, (const R4<R>*)cv.part_col,
                                                         cv.split_col, cv.nT_col, cv.scale, cv.n_a, Jc);
            mark(h, "coord_finalize");
            coord_value_kernel<R><<<W, 256, 0, st>>>(h->wn, cv.n_a < 0, cv.n_a, (const R4<R>*)cv.part_row,
                                                     cv.split_row, cv.nT_row, cv.scale, xi, c);
            mark(h, "coord_value");
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

int launch_cvs(wtmd_t* h, const void* pos)
{
    return h->prec == WTMD_F32 ? launch_cvs_t<float>(h, pos) : launch_cvs_t<double>(h, pos);
}

int launch_scatter(wtmd_t* h, void* force, const void* vel, bool kick)
{
    const int nb = (int)((h->N + 255) / 256);
    const double hdm = 0.5 * h->cfg.dt / h->cfg.mass;
    if (h->prec == WTMD_F32)
        scatter_kernel<float><<<nb, 256, 0, h->stream>>>(h->N, h->d, h->atom_walker, (const float*)h->dV,
                                                         (const float4*)h->J, (float4*)force,
                                                         kick ? (float4*)vel : nullptr, (float)hdm, h->dims);
    else
        scatter_kernel<double><<<nb, 256, 0, h->stream>>>(h->N, h->d, h->atom_walker, (const double*)h->dV,
                                                          (const dbl4*)h->J, (dbl4*)force,
                                                          kick ? (dbl4*)vel : nullptr, hdm, h->dims);
    mark(h, "scatter_kick");
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

}  // namespace wtmd
