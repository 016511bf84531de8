// Lennard-Jones pieces shared by the per-kernel engine (engine.cu) and the
// persistent single-system step (sys_step.cu): the pair force, the cell
// grid and the Verlet neighbour lists built on it.
#pragma once

#include "wtmd_internal.cuh"

namespace wtmd {

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
// Verlet neighbour lists on a cell list (single periodic walker).
//
// A list holds every partner within rl = rc + skin at its build; while no
// atom is further than skin / 2 from where it was then, every pair within
// rc is in it, so a step normally evaluates forces from the list alone.
// BAOAB compares each atom's new position with its build position and
// raises the rebuild flag past skin / 2 (whoever moved the atom); a force
// evaluation that no BAOAB precedes requests a rebuild.
//
// Each atom's partners are stored as NL_S sub-lists by a hash of j
// (nl_sub), each in increasing j.  Lane s of the atom's NL_S lanes sums the pairs of sub-list
// s within rc in that order and a fixed xor tree adds the lanes, so the force
// depends only on the pairs within rc, never on when the list was built.
// Sub-list u = NL_S i + s owns the cap8 contiguous slots from nbr[u * cap8]
// (written in one run by the list build, read as 16-byte vectors).
//
// In the per-kernel step, three launches per evaluation: binning and the
// list build return at once unless the rebuild flag is set; the force kernel
// always runs.  The persistent single-system step (sys_step.cu) runs the same
// pieces as phases of one launch.
constexpr int NL_S = 8;     // sub-lists (lanes) per atom (a power of two)
constexpr int NL_SHIFT = 29; // 32 - log2(NL_S)
static_assert((1 << (32 - NL_SHIFT)) == NL_S, "NL_SHIFT matches NL_S");

// Sub-list of partner j: the top bits of a multiplicative (Fibonacci) hash
// of j, so that the sub-lists stay balanced when atom indices follow
// positions (a lattice start numbers the atoms row by row: j mod NL_S would
// put a whole plane of neighbours into one sub-list).
__host__ __device__ __forceinline__ int nl_sub(int j) { return (int)(((unsigned)j * 2654435761u) >> NL_SHIFT); }
constexpr int NL_T = 256;   // threads per CTA of the standalone build and force kernels
constexpr int NL_B = 12;    // list entries a force lane loads together
static_assert(NL_B % 4 == 0, "list entries are read as 16-byte vectors");

template <typename R> __device__ __forceinline__ int cell_coord(R q, R invL, int nc)
{
    R u = q * invL;
    u -= floor(u);  // fractional coordinate in [0, 1]
    const int c = (int)(u * (R)nc);
    return c >= nc ? nc - 1 : (c < 0 ? 0 : c);
}

template <typename R> __device__ __forceinline__ R box_inv(const Box& b, int k)
{
    return sizeof(R) == 4 ? (R)b.invLf[k] : (R)b.invL[k];
}

// List build for home cell c by the whole CTA (any block size): the 27
// neighbour cells' atoms are staged in shared memory (smem, nl_smem_bytes of
// it), every (home atom, candidate) pair is tested, partners within rl go to
// the home atom's sub-list nl_sub(j), and each sub-list is sorted.
// Sub-lists in shared memory have an odd stride.
template <typename R>
__device__ void nl_build_cell(int c, const R4<R>* __restrict__ x, const Box& box, int ncx, int ncy, int ncz, int ccap,
                              const int* __restrict__ ccount, const int* __restrict__ catoms, int* __restrict__ nbr,
                              int* __restrict__ ncnt, R4<R>* __restrict__ xref, int cap8, R rl2, unsigned* status,
                              unsigned char* nl_smem)
{
    const int tid = threadIdx.x, T = blockDim.x;
    __syncthreads();  // a CTA building several cells: the previous cell's reads of the staging are done
    const int ls = cap8 + 1;
    R4<R>* cpos = reinterpret_cast<R4<R>*>(nl_smem);
    R4<R>* hpos = cpos + 27 * ccap;
    int* cidx = reinterpret_cast<int*>(hpos + ccap);
    int* hidx = cidx + 27 * ccap;
    int* hcnt = hidx + ccap;
    int* hlist = hcnt + ccap * NL_S;
    __shared__ int off[28], nbc[27];
    const int hz = c % ncz, hy = (c / ncz) % ncy, hx = c / (ncy * ncz);
    if (tid < 27) {
        const int q = tid;
        const int nb = (((hx + q / 9 - 1 + ncx) % ncx) * ncy + (hy + (q / 3) % 3 - 1 + ncy) % ncy) * ncz +
                       (hz + q % 3 - 1 + ncz) % ncz;
        nbc[q] = nb;
        off[q + 1] = min(ccount[nb], ccap);
    }
    __syncthreads();
    if (tid == 0) {
        off[0] = 0;
        for (int q = 0; q < 27; ++q) off[q + 1] += off[q];
    }
    __syncthreads();
    const int ncand = off[27], nh = min(ccount[c], ccap);
    for (int e = tid; e < ncand; e += T) {
        int q = 0;
        while (off[q + 1] <= e) ++q;
        const int j = catoms[(size_t)nbc[q] * ccap + (e - off[q])];
        cidx[e] = j;
        cpos[e] = x[j];
    }
    for (int t = tid; t < nh; t += T) {
        const int i = catoms[(size_t)c * ccap + t];
        hidx[t] = i;
        hpos[t] = x[i];
    }
    for (int k = tid; k < nh * NL_S; k += T) hcnt[k] = 0;
    __syncthreads();
    // each thread holds its candidates and sweeps the home atoms
    // (broadcast reads), four at a time
    for (int e = tid; e < ncand; e += T) {
        const int j = cidx[e];
        const R4<R> o = cpos[e];
        const int sj = nl_sub(j);
#pragma unroll 4
        for (int t = 0; t < nh; ++t) {
            const R4<R> p = hpos[t];
            const R dx = min_image<R>(p.x - o.x, box, 0), dy = min_image<R>(p.y - o.y, box, 1),
                    dz = min_image<R>(p.z - o.z, box, 2);
            if (dx * dx + dy * dy + dz * dz < rl2 && j != hidx[t]) {
                const int k = t * NL_S + sj;
                const int slot = atomicAdd(&hcnt[k], 1);
                if (slot < cap8) hlist[k * ls + slot] = j;
                else atomicOr(status, ST_CELL);
            }
        }
    }
    __syncthreads();
    for (int k = tid; k < nh * NL_S; k += T) {
        const int n = min(hcnt[k], cap8);
        int* l = hlist + k * ls;
        for (int a = 1; a < n; ++a) {  // insertion sort: increasing j
            const int v = l[a];
            int b = a;
            while (b > 0 && l[b - 1] > v) {
                l[b] = l[b - 1];
                --b;
            }
            l[b] = v;
        }
        const long long u = (long long)hidx[k / NL_S] * NL_S + k % NL_S;
        int* out = nbr + u * cap8;  // the sub-list's own contiguous slots
        for (int a = 0; a < n; ++a) out[a] = l[a];
        ncnt[u] = n;
    }
    for (int t = tid; t < nh; t += T) xref[hidx[t]] = hpos[t];
}

// Pairs of sub-list u = NL_S i + s of atom i: NL_B entries at a time, all
// their indices, then all their positions in flight together; the sum runs
// in list order and is added to (fx, fy, fz).  The first NL_B slots
// (NL_B <= cap8) are read with the count.
template <typename R>
__device__ __forceinline__ void lj_list_lane(long long u, const R4<R>* __restrict__ x, const Box& box,
                                             const int* __restrict__ nbr, const int* __restrict__ ncnt, int cap8,
                                             R rc2, R sig2, R eps24, R& fx, R& fy, R& fz)
{
    {
        const R4<R> p = x[u / NL_S];
        const int n = min(ncnt[u], cap8);
        // NL_B entries at a time: all their indices, then all their
        // positions are in flight together; the sum runs in list order.  The
        // first NL_B slots (NL_B <= cap8) are read with the count.
        const int* lst = nbr + u * cap8;  // 16-byte aligned (cap8 is a multiple of 4)
        int jj[NL_B];
#pragma unroll
        for (int q = 0; q < NL_B; q += 4) {
            const int4 v = *reinterpret_cast<const int4*>(lst + q);
            jj[q] = v.x;
            jj[q + 1] = v.y;
            jj[q + 2] = v.z;
            jj[q + 3] = v.w;
        }
        for (int k0 = 0; k0 < n; k0 += NL_B) {
            if (k0 > 0) {
#pragma unroll
                for (int q = 0; q < NL_B; ++q) jj[q] = k0 + q < n ? lst[k0 + q] : -1;
            } else {
#pragma unroll
                for (int q = 0; q < NL_B; ++q) jj[q] = q < n ? jj[q] : -1;
            }
            R4<R> o[NL_B];
#pragma unroll
            for (int q = 0; q < NL_B; ++q) o[q] = jj[q] >= 0 ? x[jj[q]] : p;
#pragma unroll
            for (int q = 0; q < NL_B; ++q) {
                const R dx = min_image<R>(p.x - o[q].x, box, 0), dy = min_image<R>(p.y - o[q].y, box, 1),
                        dz = min_image<R>(p.z - o[q].z, box, 2);
                const R r2 = dx * dx + dy * dy + dz * dz;
                if (jj[q] >= 0 && r2 < rc2) {
                    const R fr = lj_fr<R>(r2, sig2, eps24);
                    fx += fr * dx;
                    fy += fr * dy;
                    fz += fr * dz;
                }
            }
        }
    }
}

// Fixed xor tree over the NL_S lanes of an atom (all 32 lanes of the warp
// take part); the atom's first lane holds the total.
template <typename R> __device__ __forceinline__ void lj_lanes_sum(R& fx, R& fy, R& fz)
{
    for (int o = NL_S / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
}

// Shared memory of nl_build_cell.
template <typename R> inline size_t nl_smem_bytes(int ccap, int cap8)
{
    return sizeof(R4<R>) * 28 * (size_t)ccap + sizeof(int) * ((size_t)28 * ccap + (size_t)ccap * NL_S * (2 + cap8));
}

}  // namespace wtmd
