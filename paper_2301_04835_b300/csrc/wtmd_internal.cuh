// Internal declarations of libwtmd: device types, the handle, small device
// helpers (Philox, reductions, mbarrier/bulk-copy PTX) and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/wtmd.h"

namespace wtmd {

// ----------------------------------------------------------------------------
// status bits recorded by kernels (atomicOr into Handle::status)
// ----------------------------------------------------------------------------
enum : unsigned {
    ST_CAPACITY = 1u,
    ST_NUMERIC = 2u,
    ST_CELL = 4u,
    ST_TIMEOUT = 8u,
};

// 32-byte aligned 4-vector of doubles (positions/forces in FP64 mode).
struct __align__(32) dbl4 {
    double x, y, z, w;
};

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = dbl4; };
template <typename R> using R4 = typename Vec4<R>::T;

template <typename R> __host__ __device__ inline R4<R> mk4(R x, R y, R z, R w);
template <> __host__ __device__ inline float4 mk4<float>(float x, float y, float z, float w) { return make_float4(x, y, z, w); }
template <> __host__ __device__ inline dbl4 mk4<double>(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

// Periodic box: L[k] > 0 means periodic in k.  FP32 kernels use the edge as
// an unevaluated sum Lf + Llo of two floats (Llo = L - Lf): rounding L to one
// float would shift every boundary-crossing pair distance the same way, a
// systematic error that sums over all pairs of a CV.
struct Box {
    double L[3];
    double invL[3];
    float Lf[3];
    float Llo[3];
    float invLf[3];
};

template <typename R> __device__ __forceinline__ R min_image(R d, const Box& b, int k);
template <> __device__ __forceinline__ double min_image<double>(double d, const Box& b, int k)
{
    return b.L[k] > 0.0 ? d - b.L[k] * rint(d * b.invL[k]) : d;
}
template <> __device__ __forceinline__ float min_image<float>(float d, const Box& b, int k)
{
    if (!(b.Lf[k] > 0.f)) return d;
    const float n = rintf(d * b.invLf[k]);
    return fmaf(-n, b.Llo[k], fmaf(-n, b.Lf[k], d));
}

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Device version.
// ----------------------------------------------------------------------------
struct U4 {
    uint32_t v[4];
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
    const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(MA, c0), l0 = MA * c0;
        const uint32_t h1 = __umulhi(MB, c2), l1 = MB * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    U4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// ----------------------------------------------------------------------------
// shared-memory mbarrier + bulk-copy (TMA engine) wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared, completion counted on `bar` (bytes and both
// addresses must be multiples of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// The same test with acquire ordering at cluster scope: for a barrier whose
// transactions are stores of other CTAs of the cluster (st_async_f4).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^31 SM cycles (about a second), records
// ST_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Thread-block clusters: the CTA's rank and the cluster's size, a split
// barrier of all threads of the cluster, and an asynchronous store into the
// shared memory of another CTA of the cluster.
__device__ __forceinline__ unsigned cluster_ctarank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_nctarank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// The two halves of a cluster barrier, for one whose wait comes long after
// the arrival (every thread of the CTA calls both, in this order).  The
// arrival is relaxed: it orders nothing but the mbarrier initialisations
// that fence_mbar_init released before it, so no thread pays a memory
// barrier for it.
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Asynchronous 16-byte store into the shared memory of CTA `rank` of the
// cluster, at the address of the local variable `local` (16-byte aligned);
// its bytes complete transactions of the mbarrier at the address of `bar`
// in that CTA, which the receiver waits on (mbar_try_wait_cluster).  The
// value travels from registers: the storing CTA may exit before it lands.
__device__ __forceinline__ void st_async_f4(void* local, unsigned rank, float4 v, uint64_t* bar)
{
    uint32_t ra, rb;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(smem_addr(bar)), "r"(rank));
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     ra),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rb)
                 : "memory");
}

// Compensated FP32 sum (hi + lo, Knuth's TwoSum): about 48 significant bits
// from FP32 instructions only (FP64 throughput is very low on this part).
struct cf {
    float hi, lo;
};
__device__ __forceinline__ cf cf_add(cf a, float b)
{
    const float s = a.hi + b;
    const float bp = s - a.hi;
    return cf{s, a.lo + ((a.hi - (s - bp)) + (b - bp))};
}
__device__ __forceinline__ cf cf_add(cf a, cf b)
{
    cf r = cf_add(a, b.hi);
    r.lo += b.lo;
    return r;
}
__device__ __forceinline__ cf cf_shfl_xor(cf a, int off)
{
    return cf{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}
__device__ __forceinline__ double cf_val(cf a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor runs; pdl_wait() blocks until
// the predecessor grid has completed and its writes are visible (a no-op in
// a normal launch).  pdl_trigger() lets the dependent grid start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// 1/x from the PTX approximate reciprocal (max error 1 ulp; +-0 -> +-inf,
// +-inf -> +-0)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sense-reversing grid barrier for a cooperative launch.  Waits are bounded
// (limit SM cycles, by default 2^31, about a second); on a timeout the
// status word records it and false is returned, after which the CTA leaves
// the kernel.
constexpr long long kWaitLimit = 1ll << 31;
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* status,
                                             long long limit = kWaitLimit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (clock64() - t0 > limit) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}


// ----------------------------------------------------------------------------
// device-side CV description
// ----------------------------------------------------------------------------
struct CvDev {
    int kind = 0, axis = 0, nn = 6, flags = 0;
    int n_a = 0, n_b = 0;          // -1 = all atoms of the walker
    int hidx[4] = {0, 0, 0, 0};    // host copy of small index lists (COMPONENT, DIHEDRAL)
    int* a = nullptr;              // device, walker-local
    int* b = nullptr;
    int* inv_a = nullptr;          // device [max_wn]: position in A or -1
    int* inv_b = nullptr;
    double r0 = 1.0, scale = 0.0, period = 0.0;
    bool same_ab = false;          // A and B are the same set (one pair pass, factor 2)
    int* order = nullptr;          // device: coordination targets, members of A first, then B-only members
    double* scw = nullptr;         // device [W]: coordination scale per walker
    void* tile_row = nullptr;      // tile path (list A): row partials [W][chunk][|A|] R4
    void* tile_col = nullptr;      // column partials [W][tile][|B|] R4
    int nbchunk = 0, ntile = 0, nB_stride = 0;
    double xi_bound = 0.0;         // tile path: bound of |xi| (sets the FP32 share quantum)
    unsigned* tile_tk = nullptr;   // tile path tickets [W][ntile + nbchunk + 1]
    int n_order = 0;
    // QPAIRS: CSR from atom to (pair, sign)
    int n_pairs = 0;
    int* q_rowptr = nullptr;       // [max_wn + 1]
    int* q_items = nullptr;        // [2*n_pairs]: pair index * 2 + (0: atom is i, 1: atom is j)
    // scratch for pair passes
    void* part_row = nullptr;      // [split][W][nT] R4
    void* part_col = nullptr;
    int split_row = 0, split_col = 0;
    int nT_row = 0, nT_col = 0;    // per-walker target counts (max over walkers for "all")
};

// ----------------------------------------------------------------------------
// the handle
// ----------------------------------------------------------------------------
struct Tuned {
    int th = 0;       // hill lanes per point
    int split = 0;    // hill splits
};

struct Surrogate;  // MLP surrogate of the hills sum (mlp.cu)

// Plan of the persistent single-system step (sys_step.cu).
struct SysStepPlan {
    bool ready = false;   // set up for the current CVs and capacity
    int grid = 0;         // CTAs (one per SM)
    int hpf = 0;          // hill pairs a CTA keeps in shared memory
    size_t smem = 0;      // dynamic shared memory per CTA
    double scw[3] = {0.0, 0.0, 0.0};  // coordination scales of walker 0
    unsigned* bar = nullptr;          // grid-barrier counter and generation
};

// Plan of the persistent multi-walker step (walkers.cu).
struct WalkerPlan {
    int T = 0;             // targets per pair task
    int bps = 0;           // CTAs per SM
    int hsplit_mult = 0;   // hill splits per CTA
    int grid = 0, ntasks = 0, hsplit = 0;
    size_t smem = 0;
    int4* tasks = nullptr;
    int* tbase = nullptr;
    int* tcount = nullptr;
    double* tpart = nullptr;
    unsigned* ticket = nullptr;
    float4* rgc = nullptr;
    unsigned* bar = nullptr;
};

}  // namespace wtmd

struct wtmd_t {
    wtmd_config cfg{};
    int prec = 0;
    int d = 0;
    int dims = 3;
    int W = 1;
    int64_t N = 0;
    int max_wn = 0;
    bool walkers_from_bind = false;
    std::vector<int64_t> woff_h, wn_h;
    int64_t* woff = nullptr;   // device [W]
    int* wn = nullptr;         // device [W]
    int* atom_walker = nullptr;  // device [N]
    wtmd::CvDev cv[3];
    int ncv = 0;
    double a[3] = {0, 0, 0};   // sqrt(log2(e)/2)/sigma: scaled-CV factors of the FP32 hills sum
    wtmd::Box box{};
    // hills
    int64_t cap = 0;
    int64_t cap_pairs = 0;     // padded to a multiple of the chunk
    double* hills64 = nullptr;     // [cap][4]
    float4* hills32 = nullptr;     // [cap_pairs][2], pair-interleaved, pre-scaled, negated
    long long* count = nullptr;    // device hill count
    long long* step = nullptr;     // device step counter
    long long* dep = nullptr;      // device [2]: first new hill, number of new hills this step
    unsigned* status = nullptr;
    unsigned* ticket = nullptr;    // last-CTA ticket of the hills-sum launch (0 between launches)
    double* grid = nullptr;
    int64_t ncell = 0;
    double* gfac = nullptr;        // [W][sum bins] per-axis Gaussian factors of new hills
    int gbins_sum = 0;
    // per-evaluation scratch
    double* xi = nullptr;      // [W][4] CV values, FP64 in both precisions
    double* ctr = nullptr;     // device [3]: CV centre of the scaled FP32 hill layout (NaN = unset)
    void* V = nullptr;         // [W] R
    void* dV = nullptr;        // [W][4] R
    void* J = nullptr;         // [d][N] R4
    void* partial = nullptr;   // hills partial sums
    size_t partial_bytes = 0;
    void* hev_xi = nullptr;    // hills_eval staging
    size_t hev_bytes = 0;
    // LJ cell list and Verlet neighbour lists (single periodic walker)
    int nc[3] = {0, 0, 0};
    int ncells = 0;
    int cell_cap = 0;
    int* cell_count = nullptr;
    int* cell_atoms = nullptr;
    int* nl_nbr = nullptr;          // [nl_cap8][N][NL_S] partners by j mod NL_S, increasing j
    int* nl_cnt = nullptr;          // [N][NL_S]
    void* nl_xref = nullptr;        // [N] R4: positions at the last build
    unsigned* nl_ctl = nullptr;     // [0] rebuild flag
    int nl_cap8 = 0;
    size_t nl_smem = 0;             // shared memory of the list build
    double nl_skin = 0.0;
    // bound arrays
    void* pos = nullptr;
    void* vel = nullptr;
    void* force = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
    cudaStream_t side_stream = nullptr; // engine-force branch of a step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t cv_stream[3] = {nullptr, nullptr, nullptr};  // branches of CVs 1, 2
    cudaEvent_t ev_cv[3] = {nullptr, nullptr, nullptr};
    cudaStream_t jf_stream[3] = {nullptr, nullptr, nullptr};  // J branches of FP32 coordination CVs
    cudaEvent_t ev_jfork[3] = {nullptr, nullptr, nullptr}, ev_jjoin[3] = {nullptr, nullptr, nullptr};
    int jf_pending = 0;             // J branches the closing kick must join
    bool forces_valid = false;
    // graphs
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    cudaGraphExec_t graph1 = nullptr;
    cudaGraphExec_t graph_host = nullptr; // host state in -> one step -> host state out (wtmd_step_host)
    const void* gh_in = nullptr;          // the host buffers graph_host was captured with
    void* gh_out = nullptr;
    bool no_host_graph = false;           // its capture failed: copy around step_n instead
    bool persistent = false;        // multi-walker step as one persistent launch
    bool bias_grid = false;         // step/bias_eval read V, dV/dxi from the grid (WTMD_BIAS_GRID)
    bool bias_harm = false;         // harmonic bias about per-walker centres (WTMD_BIAS_HARMONIC)
    bool in_step = false;           // the bias being enqueued belongs to a step (window statistics count it)
    double harm_k[3] = {0.0, 0.0, 0.0};
    double* harm_centre = nullptr;  // device [W][4] window centres
    double* harm_sum = nullptr;     // device [W][4] sum of xi over steps, then [W*4] the sample count (as double)
    wtmd::WalkerPlan wk;
    bool no_graph = false;          // capture failed: replay eagerly
    bool jz_pre = false;            // the step zeroed the tile-path coordination J rows before BAOAB
    wtmd::Surrogate* sur = nullptr; // MLP surrogate state (null until used)
    wtmd::SysStepPlan ss;           // persistent single-system step
    bool fused_on = false;          // the caller allowed the persistent single-system step
    bool jbranch = false;           // bias_eval: the J rows of a tile CV on a branch beside the hills sum
    bool small_on = true;           // small FP64 analytic systems run many steps per single-CTA launch
    long long wait_limit = 0;       // grid-barrier wait bound of the persistent kernels (0: the default)
    // autotune cache: key = (P bucket, d) -> tile
    std::vector<std::pair<long long, wtmd::Tuned>> tuned;
    // profiling: when `prof` is set, mark() records a CUDA event on the
    // launching stream after each kernel (eager steps only, never in graphs)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::string> ev_names;
    int ev_n = 0;
    std::string err;
};

namespace wtmd {
inline void mark(wtmd_t* h, const char* name)
{
    if (!h->prof) return;
    if (h->ev_n >= (int)h->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->ev_pool.push_back(e);
        h->ev_names.emplace_back();
    }
    cudaEventRecord(h->ev_pool[h->ev_n], h->stream);
    h->ev_names[h->ev_n] = name;
    ++h->ev_n;
}
}  // namespace wtmd

namespace wtmd {

// launchers (defined in the .cu files); all enqueue on h->stream
int launch_cvs(wtmd_t* h, const void* pos);                       // xi, J for all CVs
int join_jbranches(wtmd_t* h);                                    // the main stream waits for the J-row branches
int launch_cv(wtmd_t* h, const void* pos, int c);               // xi, J of CV c
int launch_adjoint(wtmd_t* h, const void* grad_xi, void* grad_pos);  // J^T grad_xi
int launch_grid_update(wtmd_t* h);                              // FP64 grid += this step's new hills
// harmonic bias of every walker about its window centre (xi: h->xi)
int launch_harmonic(wtmd_t* h, bool accumulate);
// V, dV/dxi at P points read from the FP64 grid (xi: double if xi_f64, else Real)
int launch_grid_bias(wtmd_t* h, const void* xi, bool xi_f64, int xi_stride, int64_t P, void* V, void* dV,
                     int dV_stride, bool pdl);
int walkers_enable(wtmd_t* h);
int walkers_retile(wtmd_t* h, int T, int bps, int hsplit_mult);
int launch_walkers_step(wtmd_t* h, int mode);                   // 0: full step, 1: forces only
int launch_hills(wtmd_t* h, const void* xi, bool xi_f64, int xi_stride, int64_t P, void* V, void* dV, int dV_stride);
// hills [*k0p, *k1p) (k0p may be null: 0; *k0p a multiple of 256; FP32
// handles); max_hills > 0 bounds the range's length for the launch plan;
// pdl: programmatic dependent launch on the preceding kernel (which must not
// write the hill list, the counts or the centre; only the points)
int launch_hills_range(wtmd_t* h, const void* xi, bool xi_f64, int xi_stride, int64_t P, void* V, void* dV,
                       int dV_stride, const long long* k0p, const long long* k1p, long long max_hills, bool pdl);
long long surrogate_tail_bound(const wtmd_t* h);
int hills_tune(wtmd_t* h, int64_t P, int* th, int* split, double* ms);  // hills.cu
int hills_set_plan(wtmd_t* h, int64_t P, int lanes, int splits);       // hills.cu                // hills beyond k0 between refits (0: unbounded)
int launch_scatter(wtmd_t* h, void* force, const void* vel_or_null, bool kick);
int launch_scatter_deposit(wtmd_t* h);                          // kick + deposit (+ grid) of a step
// surrogate (mlp.cu)
void surrogate_free(Surrogate* s);
const long long* surrogate_k0(const wtmd_t* h);                 // first hill of the exact tail, or null
int launch_mlp_add(wtmd_t* h);                                   // V, dV += network part (if active)
int surrogate_segment(wtmd_t* h, int64_t n, int64_t* seg);       // refit if due; steps until the next refit
void surrogate_advanced(wtmd_t* h, int64_t n);
int surrogate_invalidate(wtmd_t* h);
void drop_step_graphs(wtmd_t* h);                                // api.cu
int launch_engine(wtmd_t* h);                                    // engine forces into h->force
int nl_request(wtmd_t* h);                                       // rebuild the LJ neighbour lists at the next use
int nl_reset(wtmd_t* h);                                         // cell counts and rebuild flag to 0
int launch_baoab_first(wtmd_t* h, int jmask, int xmask);         // Jacobian rows / CV values to zero
bool coord_factored(const wtmd_t* h, int c);  // CV c keeps J as FP32 tile partials (contracted by the kick)
int folded_rg(const wtmd_t* h);                                  // Rg CV computed in the launch of coordination CV 0, or -1
bool sys_step_eligible(const wtmd_t* h, std::string* why);       // the step can run as one persistent launch
int sys_step_setup(wtmd_t* h);                                   // its plan (outside graph capture)
int launch_sys_step(wtmd_t* h);                                  // one step as one cooperative launch
bool small_step_eligible(const wtmd_t* h);                       // small_step.cu: the handle's steps run in one CTA
int launch_small_steps(wtmd_t* h, int64_t n_steps);              // n steps, SMS_CHUNK per launch
int launch_deposit(wtmd_t* h);                                   // deposit + grid + step++
int launch_grid_rebuild(wtmd_t* h);
int launch_fes(wtmd_t* h, double* out);
void store_hills32(wtmd_t* h);                                   // rebuild FP32 layout from hills64
int setup_cells(wtmd_t* h);
int cv_alloc_scratch(wtmd_t* h, CvDev& c);

}  // namespace wtmd

namespace wtmd {
// Launch with programmatic stream serialization: the kernel may start while
// the preceding kernel on the stream runs; it must call pdl_wait() before it
// reads anything that kernel writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    // the largest shared-memory carveout: the kernels that a step runs side
    // by side then share one SM configuration, so a waiting dependent's CTAs
    // are not kept off an SM whose carveout another kernel chose smaller
    at[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    at[1].val.sharedMemCarveout = 100;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
}  // namespace wtmd

#define WTMD_CUDA_TRY(h, expr)                                                     \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            (h)->err = std::string(#expr) + ": " + cudaGetErrorString(_e);         \
            return WTMD_ECUDA;                                                     \
        }                                                                          \
    } while (0)
