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
#include "lj_dev.cuh"
#include "analytic_dev.cuh"

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
                                   double* __restrict__ xi, int xmask, int W, const R4<R>* __restrict__ xref,
                                   R half_skin2, unsigned* nl_flag)
{
    pdl_wait();
    pdl_trigger();  // the CV kernels that follow may launch; they wait for these positions
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // every load first (one round trip), then the zeroing stores and the update
    const bool act = i < N;
    R4<R> xa = mk4<R>(R(0), R(0), R(0), R(0)), va = xa, fa = xa, ra = xa;
    if (act) {
        xa = x[i];
        va = v[i];
        fa = f[i];
        if (nl_flag) ra = xref[i];
    }
    const long long t = *step;
    if (i < W)
        for (int c = 0; c < 3; ++c)
            if (xmask >> c & 1) xi[i * 4 + c] = 0.0;
    if (!act) return;
    for (int c = 0; c < 3; ++c)
        if (jmask >> c & 1) J[(size_t)c * N + i] = mk4<R>(R(0), R(0), R(0), R(0));
    const Normal3<R> n = noise3<R>(seed, t, (uint32_t)i);
    baoa_update<R>(xa, va, fa, n.g, half, inv_m, c1, c2, dims);
    x[i] = xa;
    v[i] = va;
    if (nl_flag) {  // moved more than half the skin since the neighbour lists were built
        const R dx = xa.x - ra.x, dy = xa.y - ra.y, dz = xa.z - ra.z;
        if (dx * dx + dy * dy + dz * dz > half_skin2) atomicOr(nl_flag, 1u);
    }
}

template <typename R>
__global__ void wells3_kernel(long long N, const R4<R>* __restrict__ x, R4<R>* __restrict__ f)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    f[i] = wells3_force<R>(x[i]);
}

template <typename R>
__global__ void mb_kernel(long long N, const R4<R>* __restrict__ x, R4<R>* __restrict__ f)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    f[i] = mb_force<R>(x[i]);
}

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

// Binning (atomics: the slot order within a cell is arbitrary and harmless,
// since the sub-lists are sorted).  Cell counts are zero on entry.
template <typename R>
__global__ void nl_bin_kernel(long long N, const R4<R>* __restrict__ x, Box box, int ncx, int ncy, int ncz, int ccap,
                              int* __restrict__ ccount, int* __restrict__ catoms, const unsigned* __restrict__ ctl,
                              unsigned* status)
{
    // a programmatic dependent of BAOAB (which sets the flag and moves the
    // atoms): wait first; the list build may start once every CTA is past
    // this wait (the flag it reads is then final)
    pdl_wait();
    pdl_trigger();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // the position is loaded with the flag (one round trip in a rebuild step)
    const R4<R> p = i < N ? x[i] : mk4<R>(R(0), R(0), R(0), R(0));
    if (*ctl == 0u) return;
    if (i >= N) return;
    const int cell = (cell_coord<R>(p.x, box_inv<R>(box, 0), ncx) * ncy + cell_coord<R>(p.y, box_inv<R>(box, 1), ncy)) *
                         ncz + cell_coord<R>(p.z, box_inv<R>(box, 2), ncz);
    const int slot = atomicAdd(&ccount[cell], 1);
    if (slot < ccap) catoms[(size_t)cell * ccap + slot] = (int)i;
    else atomicOr(status, ST_CELL);
}

// List build, one CTA per home cell (nl_build_cell).
template <typename R>
__global__ void __launch_bounds__(NL_T) nl_build_kernel(long long N, const R4<R>* __restrict__ x, Box box, int ncx,
                                                        int ncy, int ncz, int ccap, const int* __restrict__ ccount,
                                                        const int* __restrict__ catoms, int* __restrict__ nbr,
                                                        int* __restrict__ ncnt, R4<R>* __restrict__ xref,
                                                        const unsigned* __restrict__ ctl, int cap8, R rl2,
                                                        unsigned* status)
{
    pdl_trigger();
    if (*ctl == 0u) return;  // final: the binning triggers this launch only after its wait for BAOAB
    pdl_wait();              // the binning
    extern __shared__ __align__(32) unsigned char nl_smem[];
    nl_build_cell<R>((int)blockIdx.x, x, box, ncx, ncy, ncz, ccap, ccount, catoms, nbr, ncnt, xref, cap8, rl2, status,
                     nl_smem);
}

// Forces from the lists: NL_S lanes per atom (lj_list_lane), a fixed xor
// tree over them.  The cell counts and the rebuild flag are reset after the
// step's join (the closing kick), or by nl_reset.
template <typename R>
__global__ void __launch_bounds__(NL_T) lj_list_kernel(long long N, const R4<R>* __restrict__ x, Box box,
                                                       const int* __restrict__ nbr, const int* __restrict__ ncnt,
                                                       int cap8, const unsigned* __restrict__ ctl, R rc2, R sig2,
                                                       R eps24, R4<R>* __restrict__ f)
{
    const long long u = (long long)blockIdx.x * NL_T + threadIdx.x;
    // what follows may launch now: every kernel launched after this one
    // waits for it before reading the forces, and BAOAB, whose positions and
    // velocities they read before that wait, has completed (the binning
    // waited for it before the list build and this launch could start)
    pdl_trigger();
    // the flag is final when this launch starts (the list build before it
    // starts only after the binning's wait for BAOAB) and is cleared after
    // the step; without a rebuild the lists are those of an
    // earlier step and nothing is waited for
    if (*ctl != 0u) pdl_wait();  // the list build
    R fx = 0, fy = 0, fz = 0;
    if (u < N * NL_S) lj_list_lane<R>(u, x, box, nbr, ncnt, cap8, rc2, sig2, eps24, fx, fy, fz);
    lj_lanes_sum<R>(fx, fy, fz);
    if (u < N * NL_S && u % NL_S == 0) f[u / NL_S] = mk4<R>(fx, fy, fz, R(0));
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
    // skin 0.3 sigma; cells at least rc + skin wide hold every list partner
    // in the 27 around an atom's own
    h->nl_skin = 0.3 * h->cfg.lj_sigma;
    const double rl = h->cfg.lj_rc + h->nl_skin;
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        if (!(h->cfg.box[k] > 0)) return WTMD_OK;  // open boundaries: all pairs
        nc[k] = (int)floor(h->cfg.box[k] / rl);
        if (nc[k] < 3) return WTMD_OK;             // too small for a 27-cell stencil
    }
    h->nc[0] = nc[0];
    h->nc[1] = nc[1];
    h->nc[2] = nc[2];
    h->ncells = nc[0] * nc[1] * nc[2];
    // capacities: twice the mean occupancy plus a margin (a liquid exceeding
    // them is a many-sigma event; overflow is reported as WTMD_ECELL)
    const double vol = h->cfg.box[0] * h->cfg.box[1] * h->cfg.box[2];
    const double mean = (double)h->N / h->ncells;
    h->cell_cap = ((int)ceil(2.0 * mean + 16.0) + 7) / 8 * 8;
    const double nmean = (double)h->N / vol * 4.0 / 3.0 * 3.14159265358979323846 * rl * rl * rl / NL_S;
    h->nl_cap8 = std::max(NL_B, ((int)ceil(2.0 * nmean + 12.0) + 3) / 4 * 4);
    const size_t r4 = h->prec == WTMD_F32 ? sizeof(float4) : sizeof(dbl4);
    WTMD_CUDA_TRY(h, cudaMalloc(&h->cell_count, sizeof(int) * h->ncells));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->cell_atoms, sizeof(int) * (size_t)h->ncells * h->cell_cap));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->nl_nbr, sizeof(int) * (size_t)h->N * NL_S * h->nl_cap8));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->nl_cnt, sizeof(int) * (size_t)h->N * NL_S));
    // an atom whose cell overflowed is not given a list: it keeps the last
    // one it had, or none
    WTMD_CUDA_TRY(h, cudaMemset(h->nl_cnt, 0, sizeof(int) * (size_t)h->N * NL_S));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->nl_xref, r4 * (size_t)h->N));
    WTMD_CUDA_TRY(h, cudaMalloc(&h->nl_ctl, sizeof(unsigned)));
    const unsigned one = 1u;  // build before the first use
    WTMD_CUDA_TRY(h, cudaMemcpy(h->nl_ctl, &one, sizeof(one), cudaMemcpyHostToDevice));
    // the build kernel's shared memory
    const size_t sm = h->prec == WTMD_F32 ? nl_smem_bytes<float>(h->cell_cap, h->nl_cap8)
                                          : nl_smem_bytes<double>(h->cell_cap, h->nl_cap8);
    h->nl_smem = sm;
    if (sm > 200 * 1024) {  // too dense for the staged build: all pairs
        h->ncells = 0;
        return WTMD_OK;
    }
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, cudaFuncSetAttribute(nl_build_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    else
        WTMD_CUDA_TRY(h, cudaFuncSetAttribute(nl_build_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    WTMD_CUDA_TRY(h, cudaMemset(h->cell_count, 0, sizeof(int) * h->ncells));
    return WTMD_OK;
}

// The next engine evaluation rebuilds the neighbour lists (the caller may
// have moved the atoms since the last step).
int nl_request(wtmd_t* h)
{
    if (h->ncells > 0) WTMD_CUDA_TRY(h, cudaMemsetAsync(h->nl_ctl, 0xff, sizeof(unsigned), h->stream));
    return WTMD_OK;
}

// Zero cell counts and rebuild flag after an engine evaluation outside a
// step (a step's closing kick does it there).
int nl_reset(wtmd_t* h)
{
    if (h->ncells > 0) {
        WTMD_CUDA_TRY(h, cudaMemsetAsync(h->cell_count, 0, sizeof(int) * h->ncells, h->stream));
        WTMD_CUDA_TRY(h, cudaMemsetAsync(h->nl_ctl, 0, sizeof(unsigned), h->stream));
    }
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
            const double rl = c.lj_rc + h->nl_skin;
            // bin -> build -> forces as programmatic dependents: the first
            // two return at once unless a rebuild is flagged
            // binning: a programmatic dependent of BAOAB; the list build: a
            // programmatic dependent of the binning, which triggers it after
            // its own wait for BAOAB, so the flag that it and the force
            // sweep read is final (its large-shared-memory CTAs wait on an
            // SM only in a step with a rebuild)
            WTMD_CUDA_TRY(h, launch_pdl(nl_bin_kernel<R>, dim3(nb), dim3(256), 0, st, (long long)h->N, x, h->box,
                                        h->nc[0], h->nc[1], h->nc[2], h->cell_cap, h->cell_count, h->cell_atoms,
                                        (const unsigned*)h->nl_ctl, h->status));
            mark(h, "nl_bin");
            WTMD_CUDA_TRY(h, launch_pdl(nl_build_kernel<R>, dim3(h->ncells), dim3(NL_T), h->nl_smem, st,
                                        (long long)h->N, x, h->box, h->nc[0], h->nc[1], h->nc[2], h->cell_cap,
                                        (const int*)h->cell_count, (const int*)h->cell_atoms, h->nl_nbr, h->nl_cnt,
                                        (R4<R>*)h->nl_xref, (const unsigned*)h->nl_ctl, h->nl_cap8, (R)(rl * rl),
                                        h->status));
            mark(h, "nl_build");
            const unsigned nbl = (unsigned)((h->N * NL_S + NL_T - 1) / NL_T);
            WTMD_CUDA_TRY(h, launch_pdl(lj_list_kernel<R>, dim3(nbl), dim3(NL_T), 0, st, (long long)h->N, x, h->box,
                                        (const int*)h->nl_nbr, (const int*)h->nl_cnt, h->nl_cap8,
                                        (const unsigned*)h->nl_ctl, rc2, sig2, e24, f));
            mark(h, "lj_list");
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
    // rebuild threshold slightly under (skin / 2)^2 against rounding
    const double hs2 = 0.249 * h->nl_skin * h->nl_skin;
    unsigned* nlf = h->ncells > 0 ? h->nl_ctl : nullptr;
    if (h->prec == WTMD_F32)
        WTMD_CUDA_TRY(h, launch_pdl(baoab_first_kernel<float>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N,
                                    (float4*)h->pos, (float4*)h->vel, (const float4*)h->force,
                                    (const long long*)h->step, c.seed, (float)(0.5 * c.dt), (float)(1.0 / c.mass),
                                    (float)c1, (float)c2, h->dims, (float4*)h->J, jmask, h->xi, xmask, h->W,
                                    (const float4*)h->nl_xref, (float)hs2, nlf));
    else
        WTMD_CUDA_TRY(h, launch_pdl(baoab_first_kernel<double>, dim3(nb), dim3(256), 0, h->stream, (long long)h->N,
                                    (dbl4*)h->pos, (dbl4*)h->vel, (const dbl4*)h->force, (const long long*)h->step,
                                    c.seed, 0.5 * c.dt, 1.0 / c.mass, c1, c2, h->dims, (dbl4*)h->J, jmask,
                                    h->xi, xmask, h->W, (const dbl4*)h->nl_xref, hs2, nlf));
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
