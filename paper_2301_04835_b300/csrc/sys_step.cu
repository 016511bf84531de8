// One MD step of a single periodic system in one persistent launch.
//
// The per-kernel step (api.cu) is a graph of about ten launches; at 4096
// atoms each does a few microseconds of work behind a launch and a memory
// round trip, and the early-launched CTAs of waiting kernels hold SM slots
// that the running ones need.  For the common single-system form -- one
// periodic walker, the Lennard-Jones engine on Verlet lists, FP32, CVs that
// are FP32 tile coordination numbers or radii of gyration, the exact hills
// sum -- this file runs the whole step as one cooperative kernel with one
// CTA per SM and bounded grid barriers between its phases (PySAGES paper,
// Sec. 3.2.1 steps (a)-(f), with the method's update of Sec. 2.1.5 inside):
//
//   A  B-A-O-A half of BAOAB for the CTA's atoms (the rebuild test of the
//      lists against their build positions); the CTA's share of the hill
//      records is copied into shared memory by one bulk copy, which lands
//      while the next phases run;
//   (rebuild steps only: the atoms are binned, then each CTA builds the
//      lists of its cells; two more barriers)
//   B  two warp groups side by side: warps 0-7 the LJ forces of the CTA's
//      atoms from their lists, warps 8-15 the CV tasks -- coordination
//      tiles (64 members x 256 partners each) and radius-of-gyration
//      groups -- spread over the CTAs;
//   C  the hills sum at the new CVs over the CTA's records (compensated
//      FP32 partial per CTA); the coordination J rows of the CTA's atoms
//      from the tile partials;
//   D  every CTA reduces the partials in the same fixed order (so every CTA
//      holds the same V and dV/dxi); CTA 0 deposits; the CTA's atoms get
//      the bias force -J^T dV/dxi and the closing half kick.
//
// The pieces are those of the per-kernel step (lj_dev.cuh, coord_dev.cuh,
// step_dev.cuh), so the forces, CVs and noise are the same functions; only
// the hills partial split and the reduction order of V differ.  Every
// reduction has a fixed order: the step is deterministic.
#include <algorithm>

#include "coord_dev.cuh"
#include "hills_dev.cuh"
#include "lj_dev.cuh"
#include "step_dev.cuh"

namespace wtmd {

constexpr int SS_T = 512;         // threads per CTA
constexpr int SS_GT = 256;        // threads of each warp group in phase B
constexpr int SS_RG_MAX = 1024;   // members of an Rg group kept in shared memory

enum { SS_CV_COORD = 1, SS_CV_RG = 2 };

struct SsCv {
    int kind = 0;
    int col = 0;
    int ntask = 0;      // CV-group tasks of this CV
    CoordTile2 ct{};    // coordination: the tile task (walker 0)
    CoordParts cp{};    // coordination: its factored J
    const int* rg_a = nullptr;  // Rg: walker-local members, or null = all atoms
    int rg_m = 0;
    double rg_scale = 0.0;
    int rg_intensive = 0;
};

struct SsArgs {
    long long N;
    int per;            // atoms per CTA
    float4* x;
    float4* v;
    float4* f;
    float4* J;          // [d][N]
    double* xi;         // [4]
    long long* step;
    uint64_t seed;
    float half, inv_m, c1, c2;
    int dims;
    Box box;
    // cells and lists
    int nc[3], ccap, ncells;
    int* ccount;
    int* catoms;
    int* nbr;
    int* ncnt;
    float4* xref;
    unsigned* ctl;
    int cap8;
    float rl2, half_skin2, rc2, sig2, eps24;
    // CVs
    int d;
    SsCv cv[3];
    int ntask;          // CV-group tasks of all CVs
    // hills
    const float4* hp;
    const long long* cnt;
    const double* ctr;
    HillPrmF32 hprm;
    int hpf;            // hill pairs a CTA keeps in shared memory
    dbl4* hpart;        // [grid] compensated partials
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
    long long wait_limit;  // grid-barrier wait bound (SM cycles)
};

// Barrier of one 256-thread warp group of the CTA (named barrier 1 + group).
__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(SS_GT) : "memory");
}

// Deterministic sum of NV compensated values over the 256 threads of group
// g (the same order as the block sum of the per-kernel Rg kernel); every
// thread of the group gets the totals.
template <int NV> __device__ __forceinline__ void group_sum_cf(cf v[NV], cf (*sm)[NV], int gtid, int g)
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = cf_add(v[k], cf_shfl_xor(v[k], o));
    const int warp = gtid / 32, lane = gtid % 32;
    group_sync(g);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    group_sync(g);
    for (int k = 0; k < NV; ++k) {
        cf t = sm[0][k];
        for (int w = 1; w < SS_GT / 32; ++w) t = cf_add(t, sm[w][k]);
        v[k] = t;
    }
}

// Radius of gyration of one group by a 256-thread warp group: members
// unwrapped by the minimum image relative to the first, equal masses,
// compensated FP32 sums; writes xi and the members' J rows.
__device__ void ss_rg_task(const SsArgs& a, const SsCv& c, int gtid, int g, float4* u, cf (*sm3)[3], cf (*sm1)[1])
{
    const int m = c.rg_a ? c.rg_m : (int)a.N;
    const int i0 = c.rg_a ? c.rg_a[0] : 0;
    const float4 r0 = a.x[i0];
    auto unwrap = [&](int p) {
        const int i = c.rg_a ? c.rg_a[p] : p;
        const float4 q = a.x[i];
        return make_float4(r0.x + min_image<float>(q.x - r0.x, a.box, 0), r0.y + min_image<float>(q.y - r0.y, a.box, 1),
                           r0.z + min_image<float>(q.z - r0.z, a.box, 2), 0.f);
    };
    cf s[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int p = gtid; p < m; p += SS_GT) {
        const float4 q = unwrap(p);
        u[p] = q;
        s[0] = cf_add(s[0], q.x);
        s[1] = cf_add(s[1], q.y);
        s[2] = cf_add(s[2], q.z);
    }
    group_sum_cf<3>(s, sm3, gtid, g);
    const float cx = (float)(cf_val(s[0]) / m), cy = (float)(cf_val(s[1]) / m), cz = (float)(cf_val(s[2]) / m);
    cf q2[1] = {{0.f, 0.f}};
    for (int p = gtid; p < m; p += SS_GT) {
        const float4 q = u[p];
        const float ux = q.x - cx, uy = q.y - cy, uz = q.z - cz;
        q2[0] = cf_add(q2[0], ux * ux + uy * uy + uz * uz);
    }
    group_sum_cf<1>(q2, sm1, gtid, g);
    const double rg = sqrt(cf_val(q2[0]) / m);
    double sc = c.rg_scale != 0.0 ? c.rg_scale : 1.0;
    if (c.rg_intensive) sc /= cbrt((double)m);
    const float fj = (float)(sc / (m * rg));
    float4* Jc = a.J + (size_t)c.col * a.N;
    for (int p = gtid; p < m; p += SS_GT) {
        const int i = c.rg_a ? c.rg_a[p] : p;
        const float4 q = u[p];
        Jc[i] = make_float4(fj * (q.x - cx), fj * (q.y - cy), fj * (q.z - cz), 0.f);
    }
    if (gtid == 0) a.xi[c.col] = sc * rg;
    group_sync(g);  // u and the sums are free for the next task
}

// Hill pairs [k0, k1) of the CTA's split (shared-memory records first, the
// rest from global memory) at the point X: per-thread packed sums.
template <int D, bool PER>
__device__ __forceinline__ void ss_hill_pairs(const float4* rec, const float4* hp, long long q0, int npf, long long nq,
                                              const float2 X[3], const HillPrmF32& prm, float2& v, float2& g0,
                                              float2& g1, float2& g2)
{
    for (long long k = threadIdx.x; k < nq; k += SS_T) {
        float4 A, B;
        if (k < npf) {
            A = rec[2 * k];
            B = rec[2 * k + 1];
        } else {
            A = __ldg(hp + 2 * (q0 + k));
            B = __ldg(hp + 2 * (q0 + k) + 1);
        }
        float2 d0 = __fadd2_rn(X[0], make_float2(A.x, A.y));
        if constexpr (PER) d0 = wrap2(d0, prm.per[0], prm.iper[0]);
        float2 t = __ffma2_rn(d0, d0, make_float2(B.z, B.w));
        float2 d1, d2;
        if constexpr (D >= 2) {
            d1 = __fadd2_rn(X[1], make_float2(A.z, A.w));
            if constexpr (PER) d1 = wrap2(d1, prm.per[1], prm.iper[1]);
            t = __ffma2_rn(d1, d1, t);
        }
        if constexpr (D >= 3) {
            d2 = __fadd2_rn(X[2], make_float2(B.x, B.y));
            if constexpr (PER) d2 = wrap2(d2, prm.per[2], prm.iper[2]);
            t = __ffma2_rn(d2, d2, t);
        }
        const float2 e = make_float2(ex2_approx(-t.x), ex2_approx(-t.y));
        v = __fadd2_rn(v, e);
        g0 = __ffma2_rn(e, d0, g0);
        if constexpr (D >= 2) g1 = __ffma2_rn(e, d1, g1);
        if constexpr (D >= 3) g2 = __ffma2_rn(e, d2, g2);
    }
}

template <int D, bool PER, int HC>
__global__ void __launch_bounds__(SS_T, 1) sys_step_kernel(SsArgs a)
{
    extern __shared__ __align__(128) unsigned char ss_smem[];
    float4* rec = reinterpret_cast<float4*>(ss_smem);  // [hpf][2] hill pair records
    unsigned char* work = ss_smem + (((size_t)a.hpf * 32 + 127) / 128) * 128;
    __shared__ __align__(8) uint64_t hbar;
    __shared__ CF4 hred[SS_T / 32];
    __shared__ float sdv[3];
    __shared__ int rebuild;
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x, b = blockIdx.x;
    const long long i0 = (long long)b * a.per;

    // ---- A: B-A-O-A for the CTA's atoms; the hill records of its split
    const long long t = *a.step;
    const long long count = *a.cnt;
    const long long npairs = (count + 1) >> 1;
    const long long hper = (npairs + G - 1) / G;
    const long long q0 = (long long)b * hper;
    const long long nq = q0 < npairs ? (hper < npairs - q0 ? hper : npairs - q0) : 0;
    const int npf = (int)(nq < a.hpf ? nq : a.hpf);
    if (tid == 0) {
        mbar_init(&hbar, 1);
        fence_mbar_init();
        if (npf > 0) {
            mbar_arrive_expect_tx(&hbar, (uint32_t)npf * 32u);
            bulk_g2s(rec, a.hp + 2 * q0, (uint32_t)npf * 32u, &hbar);
        }
    }
    if (b == 0 && tid == 0)
        for (int c = 0; c < a.d; ++c)
            if (a.cv[c].kind == SS_CV_COORD) a.xi[c] = 0.0;
    for (int q = tid; q < a.per; q += SS_T) {
        const long long i = i0 + q;
        if (i >= a.N) break;
        baoab_first_atom<float>(i, t, a.x, a.v, a.f, a.seed, a.half, a.inv_m, a.c1, a.c2, a.dims);
        const float4 p = a.x[i], r = a.xref[i];
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        if (dx * dx + dy * dy + dz * dz > a.half_skin2) atomicOr(a.ctl, 1u);
    }
    // a CTA that leaves on a timeout first lets its own bulk copy land
    auto leave = [&]() {
        if (npf > 0) mbar_wait_bounded(&hbar, 0, a.status);
    };
    if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return leave();

    // ---- rebuild of the neighbour lists, when an atom moved past half the skin
    if (tid == 0) rebuild = *(volatile unsigned*)a.ctl != 0u;
    __syncthreads();
    if (rebuild) {
        for (int q = tid; q < a.per; q += SS_T) {
            const long long i = i0 + q;
            if (i >= a.N) break;
            const float4 p = a.x[i];
            const int cell = (cell_coord<float>(p.x, a.box.invLf[0], a.nc[0]) * a.nc[1] +
                              cell_coord<float>(p.y, a.box.invLf[1], a.nc[1])) * a.nc[2] +
                             cell_coord<float>(p.z, a.box.invLf[2], a.nc[2]);
            const int slot = atomicAdd(&a.ccount[cell], 1);
            if (slot < a.ccap) a.catoms[(size_t)cell * a.ccap + slot] = (int)i;
            else atomicOr(a.status, ST_CELL);
        }
        if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return leave();
        for (int c = b; c < a.ncells; c += G)
            nl_build_cell<float>(c, a.x, a.box, a.nc[0], a.nc[1], a.nc[2], a.ccap, a.ccount, a.catoms, a.nbr, a.ncnt,
                                 a.xref, a.cap8, a.rl2, a.status, work);
        if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return leave();
    }

    // ---- B: LJ forces (warps 0-7) beside the CV tasks (warps 8-15)
    const int g = tid / SS_GT, gtid = tid % SS_GT;
    if (g == 0) {
        const int s = gtid % NL_S;
        for (int q0a = 0; q0a < a.per; q0a += SS_GT / NL_S) {  // uniform trip count: the shuffles below
            const long long i = i0 + q0a + gtid / NL_S;
            const bool act = q0a + gtid / NL_S < a.per && i < a.N;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            if (act) lj_list_lane<float>(i * NL_S + s, a.x, a.box, a.nbr, a.ncnt, a.cap8, a.rc2, a.sig2, a.eps24, fx, fy, fz);
            lj_lanes_sum<float>(fx, fy, fz);
            if (act && s == 0) a.f[i] = make_float4(fx, fy, fz, 0.f);
        }
    } else {
        float4* srcA = reinterpret_cast<float4*>(work);
        float4* srcB = srcA + CT_B;
        float4(*rowred)[C2_A] = reinterpret_cast<float4(*)[C2_A]>(srcB + CT_B);
        double* xred = reinterpret_cast<double*>(rowred + CT_T / 32);
        float4* ru = reinterpret_cast<float4*>(xred + 2);
        cf(*sm3)[3] = reinterpret_cast<cf(*)[3]>(ru + SS_RG_MAX);
        cf(*sm1)[1] = reinterpret_cast<cf(*)[1]>(sm3 + 32);
        for (int task = b; task < a.ntask; task += G) {
            int c = 0, k = task;
            while (k >= a.cv[c].ntask) k -= a.cv[c].ntask, ++c;
            const SsCv& cv = a.cv[c];
            if (cv.kind == SS_CV_COORD)
                coord_tile2_body<HC>(cv.ct, k / cv.ct.nbchunk, k % cv.ct.nbchunk, gtid, srcA, srcB, rowred, xred, [] {},
                                     [] { group_sync(1); });
            else
                ss_rg_task(a, cv, gtid, 1, ru, sm3, sm1);
        }
    }
    if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return leave();

    // ---- C: hills partial of the CTA's split; J rows of the coordination CVs
    {
        float2 X[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float v = 0.f;
            if (k < D) v = (float)((__ldcg(a.xi + k) - a.ctr[k]) * a.hprm.a[k]);
            X[k] = make_float2(v, v);
        }
        if (npf > 0 && !mbar_wait_bounded(&hbar, 0, a.status)) return;
        float2 v = make_float2(0.f, 0.f), g0 = v, g1 = v, g2 = v;
        ss_hill_pairs<D, PER>(rec, a.hp, q0, npf, nq, X, a.hprm, v, g0, g1, g2);
        CF4 acc{};
        acc.v[0] = cf_add(cf_add(acc.v[0], v.x), v.y);
        acc.v[1] = cf_add(cf_add(acc.v[1], g0.x), g0.y);
        acc.v[2] = cf_add(cf_add(acc.v[2], g1.x), g1.y);
        acc.v[3] = cf_add(cf_add(acc.v[3], g2.x), g2.y);
        cf4_lane_sum<32>(acc);
        if (tid % 32 == 0) hred[tid / 32] = acc;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < SS_T / 32; ++w) cf4_add(acc, hred[w]);
            store_cf4(a.hpart + b, acc);
            mbar_inval(&hbar);
        }
        for (int c = 0; c < a.d; ++c) {
            if (a.cv[c].kind != SS_CV_COORD) continue;
            float4* Jc = a.J + (size_t)c * a.N;
            for (int q = tid; q < a.per; q += SS_T) {
                const long long i = i0 + q;
                if (i >= a.N) break;
                Jc[i] = coord_j_parts(a.cv[c].cp, 0, (int)i);
            }
        }
    }
    if (!grid_barrier(a.bar, G, a.status, a.wait_limit)) return;

    // ---- D: V and dV/dxi (the same fixed order in every CTA), deposition,
    // bias force and closing kick
    if (tid < 32) {
        CF4 acc{};
        for (int s = tid; s < (int)G; s += 32) cf4_add(acc, load_cf4(a.hpart + s));
        cf4_lane_sum<32>(acc);
        if (tid == 0) {
            for (int k = 0; k < 3; ++k) sdv[k] = a.hout.gsf[k] * (acc.v[1 + k].hi + acc.v[1 + k].lo);  // as emit_cf
            if (b == 0) emit_cf(0, acc, a.hout);
        }
    }
    __syncthreads();
    if (b == 0) {
        deposit_block<float>(a.dep, a.xi, a.hout.V, a.count, a.step, a.depw, a.ctrw, a.h64, a.h32, a.status);
        if (rebuild) {
            for (int c = tid; c < a.ncells; c += SS_T) a.ccount[c] = 0;
            if (tid == 0) *a.ctl = 0u;
        }
    }
    for (int q = tid; q < a.per; q += SS_T) {
        const long long i = i0 + q;
        if (i >= a.N) break;
        float4 F = a.f[i];
        for (int c = 0; c < D; ++c) {
            const float4 j = __ldcg(a.J + (size_t)c * a.N + i);
            F.x -= sdv[c] * j.x;
            F.y -= sdv[c] * j.y;
            F.z -= sdv[c] * j.z;
        }
        a.f[i] = F;
        float4 v = a.v[i];
        v.x += a.half * a.inv_m * F.x;
        v.y += a.half * a.inv_m * F.y;
        if (a.dims > 2) v.z += a.half * a.inv_m * F.z;
        a.v[i] = v;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using SsKernel = void (*)(SsArgs);

static bool ss_any_periodic(const wtmd_t* h)
{
    for (int c = 0; c < h->d; ++c)
        if (h->cv[c].period > 0.0) return true;
    return false;
}

template <int D, bool PER> static SsKernel ss_kernel_d(int hc)
{
    return hc == 3 ? sys_step_kernel<D, PER, 3> : sys_step_kernel<D, PER, 0>;
}

static SsKernel ss_kernel(const wtmd_t* h)
{
    int hc = 3;
    for (int c = 0; c < h->d; ++c)
        if (h->cv[c].kind == WTMD_CV_COORDINATION && h->cv[c].nn != 6) hc = 0;
    const bool per = ss_any_periodic(h);
    switch (h->d * 2 + (per ? 1 : 0)) {
    case 2: return ss_kernel_d<1, false>(hc);
    case 3: return ss_kernel_d<1, true>(hc);
    case 4: return ss_kernel_d<2, false>(hc);
    case 5: return ss_kernel_d<2, true>(hc);
    case 6: return ss_kernel_d<3, false>(hc);
    default: return ss_kernel_d<3, true>(hc);
    }
}

// Shared memory of the CV group's tasks: tile staging, row sums, the share,
// the Rg members and the group sums.
static size_t ss_cv_smem() { return sizeof(float4) * (2 * CT_B + (CT_T / 32) * C2_A) + 2 * sizeof(double) +
                                    sizeof(float4) * SS_RG_MAX + sizeof(cf) * 32 * 4; }

bool sys_step_eligible(const wtmd_t* h, std::string* why)
{
    auto no = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (h->prec != WTMD_F32) return no("FP64 handle");
    if (h->W != 1 || h->ncells <= 0) return no("not a single periodic walker on the LJ cell lists");
    if (h->cfg.engine != WTMD_ENGINE_LJ) return no("engine is not LJ");
    if (h->persistent) return no("the persistent multi-walker step is on");
    if (h->bias_grid || h->bias_harm) return no("bias not read from the hills");
    if (surrogate_k0(h)) return no("surrogate on");
    if (h->ncv != h->d || h->d < 1 || h->d > 3) return no("CVs not all defined");
    if (h->grid) return no("an FP64 bias grid is configured");
    for (int c = 0; c < h->d; ++c) {
        const CvDev& cv = h->cv[c];
        if (cv.kind == WTMD_CV_COORDINATION && coord_factored(h, c)) continue;
        if (cv.kind == WTMD_CV_RG && (cv.n_a < 0 ? h->N : cv.n_a) <= SS_RG_MAX) continue;
        return no("a CV other than an FP32 tile coordination number or a radius of gyration");
    }
    return true;
}

int sys_step_setup(wtmd_t* h)
{
    SysStepPlan& k = h->ss;
    int dev = 0, sms = 0, maxsm = 0;
    WTMD_CUDA_TRY(h, cudaGetDevice(&dev));
    WTMD_CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WTMD_CUDA_TRY(h, cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t work = std::max(nl_smem_bytes<float>(h->cell_cap, h->nl_cap8), ss_cv_smem());
    const size_t stat = 8 * 1024;  // static shared memory of the kernel, with margin
    const long long cap_pairs_cta = (h->cap_pairs + sms - 1) / sms;
    const long long room = ((long long)maxsm - (long long)stat - (long long)work - 128) / 32;
    if (room < 0) {
        h->err = "persistent step: shared memory too small";
        return WTMD_EINVAL;
    }
    k.hpf = (int)std::min<long long>(cap_pairs_cta, room);
    k.smem = (((size_t)k.hpf * 32 + 127) / 128) * 128 + work;
    const void* fn = (const void*)ss_kernel(h);
    WTMD_CUDA_TRY(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    int occ = 0;
    WTMD_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, SS_T, k.smem));
    if (occ < 1) {
        h->err = "persistent step does not fit on an SM";
        return WTMD_EINVAL;
    }
    k.grid = sms;
    for (int q = 0; q < h->d; ++q) {
        k.scw[q] = 0.0;
        if (h->cv[q].kind == WTMD_CV_COORDINATION)
            WTMD_CUDA_TRY(h, cudaMemcpy(&k.scw[q], h->cv[q].scw, sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (!k.bar) {
        WTMD_CUDA_TRY(h, cudaMalloc(&k.bar, sizeof(unsigned) * 4));
        WTMD_CUDA_TRY(h, cudaMemset(k.bar, 0, sizeof(unsigned) * 4));
    }
    const size_t need = (size_t)k.grid * sizeof(dbl4);
    if (need > h->partial_bytes) {
        cudaFree(h->partial);
        h->partial = nullptr;
        h->partial_bytes = 0;
        WTMD_CUDA_TRY(h, cudaMalloc(&h->partial, need));
        h->partial_bytes = need;
    }
    k.ready = true;
    return WTMD_OK;
}

int launch_sys_step(wtmd_t* h)
{
    const SysStepPlan& k = h->ss;
    const wtmd_config& c = h->cfg;
    SsArgs a{};
    a.N = h->N;
    a.per = (int)((h->N + k.grid - 1) / k.grid);
    a.x = (float4*)h->pos;
    a.v = (float4*)h->vel;
    a.f = (float4*)h->force;
    a.J = (float4*)h->J;
    a.xi = h->xi;
    a.step = h->step;
    a.seed = c.seed;
    const double c1 = exp(-c.friction * c.dt);
    a.half = (float)(0.5 * c.dt);
    a.inv_m = (float)(1.0 / c.mass);
    a.c1 = (float)c1;
    a.c2 = (float)sqrt((1.0 - c1 * c1) * c.kT / c.mass);
    a.dims = h->dims;
    a.box = h->box;
    for (int q = 0; q < 3; ++q) a.nc[q] = h->nc[q];
    a.ccap = h->cell_cap;
    a.ncells = h->ncells;
    a.ccount = h->cell_count;
    a.catoms = h->cell_atoms;
    a.nbr = h->nl_nbr;
    a.ncnt = h->nl_cnt;
    a.xref = (float4*)h->nl_xref;
    a.ctl = h->nl_ctl;
    a.cap8 = h->nl_cap8;
    const double rl = c.lj_rc + h->nl_skin;
    a.rl2 = (float)(rl * rl);
    a.half_skin2 = (float)(0.249 * h->nl_skin * h->nl_skin);  // slightly under (skin / 2)^2 against rounding
    a.rc2 = (float)(c.lj_rc * c.lj_rc);
    a.sig2 = (float)(c.lj_sigma * c.lj_sigma);
    a.eps24 = (float)(24.0 * c.lj_eps);
    a.d = h->d;
    a.ntask = 0;
    for (int q = 0; q < h->d; ++q) {
        const CvDev& cv = h->cv[q];
        SsCv& s = a.cv[q];
        s.col = q;
        if (cv.kind == WTMD_CV_COORDINATION) {
            s.kind = SS_CV_COORD;
            const int ntile = (cv.n_a + C2_A - 1) / C2_A;
            const int qq = 50 - std::max(0, (int)std::ceil(std::log2(std::max(cv.xi_bound, 1.0))));
            const double scw = k.scw[q];
            s.ct = CoordTile2{(const float4*)h->pos, (int)h->N, cv.a, cv.n_a, cv.n_b < 0 ? nullptr : cv.b, cv.n_b,
                              cv.nbchunk, ntile, h->box, (float)(1.0 / (cv.r0 * cv.r0)), cv.nn / 2,
                              (float)(-(double)cv.nn / (cv.r0 * cv.r0)), (float4*)cv.tile_row, (float4*)cv.tile_col,
                              cv.nB_stride, scw, h->xi + q, cv.n_b < 0 ? nullptr : cv.inv_b, std::ldexp(1.0, qq),
                              std::ldexp(1.0, -qq)};
            s.cp.rowpart = (const float4*)cv.tile_row;
            s.cp.colpart = (const float4*)cv.tile_col;
            s.cp.inv_a = cv.inv_a;
            s.cp.inv_b = cv.n_b < 0 ? nullptr : cv.inv_b;
            s.cp.scw = cv.scw;
            s.cp.nA = cv.n_a;
            s.cp.nbchunk = cv.nbchunk;
            s.cp.ntile = ntile;
            s.cp.nB_stride = cv.nB_stride;
            s.ntask = ntile * cv.nbchunk;
        } else {
            s.kind = SS_CV_RG;
            s.rg_a = cv.n_a < 0 ? nullptr : cv.a;
            s.rg_m = cv.n_a < 0 ? (int)h->N : cv.n_a;
            s.rg_scale = cv.scale;
            s.rg_intensive = cv.flags & WTMD_CV_INTENSIVE;
            s.ntask = 1;
        }
        a.ntask += s.ntask;
    }
    a.hp = h->hills32;
    a.cnt = h->count;
    a.ctr = h->ctr;
    for (int q = 0; q < 3; ++q) {
        a.hprm.a[q] = h->a[q];
        const double pp = q < h->d ? h->cv[q].period * h->a[q] : 0.0;
        a.hprm.per[q] = (float)pp;
        a.hprm.iper[q] = pp > 0.0 ? (float)(1.0 / pp) : 0.f;
    }
    a.hpf = k.hpf;
    a.hpart = (dbl4*)h->partial;
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
    a.dep = dep_prm(h);
    a.count = h->count;
    a.depw = h->dep;
    a.ctrw = h->ctr;
    a.h64 = (dbl4*)h->hills64;
    a.h32 = (float*)h->hills32;
    a.bar = k.bar;
    a.status = h->status;
    a.wait_limit = h->wait_limit > 0 ? h->wait_limit : kWaitLimit;
    // a clean launch leaves the barrier counter at 0; after a timed-out
    // barrier wtmd_check clears it
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(k.grid);
    cfg.blockDim = dim3(SS_T);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, ss_kernel(h), a);
    if (e != cudaSuccess) {
        h->err = std::string("persistent step launch: ") + cudaGetErrorString(e);
        return WTMD_ECUDA;
    }
    mark(h, "sys_step");
    return WTMD_OK;
}

}  // namespace wtmd
