// C ABI of libwtmd (declared in include/wtmd.h): handle lifetime, argument
// checks, and the per-step launch sequence captured once into a CUDA graph.
//
// One MD step (PySAGES paper, Sec. 3.2.1 steps (a)-(f), with the method's
// update inside the step as the paper's force-like object, Sec. 2):
//   (a) B-A-O-A half of BAOAB with Philox noise;
//   (b,c) engine forces at the new positions;
//   (d) CVs and their Jacobians;  hills sum V, dV/dxi;
//   (e) bias-force scatter F -= J^T dV/dxi, fused with (f) the closing B;
//   deposition every `stride` steps (Sec. 2.1.5), FP64 grid update, step++.
// The step counter and the hill count live in device memory, so one captured
// graph replays for the whole run while the hill list grows.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "wtmd_internal.cuh"

using namespace wtmd;

namespace wtmd {
void store_hills32_range(wtmd_t* h, long long k0, long long k1);
int launch_hills_partial_prealloc(wtmd_t* h, int64_t P);
}  // namespace wtmd

static const int kGraphSteps = 8;

#define FAIL(h, code, msg)    \
    do {                      \
        (h)->err = (msg);     \
        return (code);        \
    } while (0)

static double c_lo(const wtmd_config* c, int i) { return c->grid_lo[i]; }
static double c_hi(const wtmd_config* c, int i) { return c->grid_hi[i]; }

static size_t realsz(const wtmd_t* h) { return h->prec == WTMD_F32 ? sizeof(float) : sizeof(double); }
static size_t r4sz(const wtmd_t* h) { return h->prec == WTMD_F32 ? sizeof(float4) : sizeof(dbl4); }

__global__ static void pad_hills32_kernel(float4* p, long long npairs)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    p[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
    p[2 * i + 1] = make_float4(0.f, 0.f, INFINITY, INFINITY);
}

static void drop_graphs(wtmd_t* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph1) cudaGraphExecDestroy(h->graph1);
    if (h->graph_host) cudaGraphExecDestroy(h->graph_host);
    h->graph = nullptr;
    h->graph1 = nullptr;
    h->graph_host = nullptr;
    h->gh_in = nullptr;
    h->gh_out = nullptr;
    h->ss.ready = false;  // the persistent step's plan follows the CVs and bindings
}

namespace wtmd {
void drop_step_graphs(wtmd_t* h) { drop_graphs(h); }
}  // namespace wtmd

// Bias at the walkers' CVs: the exact hills sum, over [k0, count) plus the
// network's part when the surrogate is active, or the bias read from the grid
// (WTMD_BIAS_GRID).
static int launch_bias_sum(wtmd_t* h)
{
    if (h->bias_harm) return launch_harmonic(h, h->in_step);
    if (h->bias_grid) return launch_grid_bias(h, h->xi, true, 4, h->W, h->V, h->dV, 4, true);
    // the preceding kernel on this stream computes CVs (it writes xi only)
    int rc = launch_hills_range(h, h->xi, true, 4, h->W, h->V, h->dV, 4, surrogate_k0(h), h->count,
                                surrogate_tail_bound(h), true);
    if (rc) return rc;
    return launch_mlp_add(h);
}

static void free_cv(CvDev& c)
{
    cudaFree(c.a);
    cudaFree(c.b);
    cudaFree(c.inv_a);
    cudaFree(c.inv_b);
    cudaFree(c.q_rowptr);
    cudaFree(c.q_items);
    cudaFree(c.tile_tk);
    cudaFree(c.order);
    cudaFree(c.scw);
    cudaFree(c.tile_row);
    cudaFree(c.tile_col);
    cudaFree(c.part_row);
    cudaFree(c.part_col);
    c = CvDev();
}

extern "C" int wtmd_destroy(wtmd_t* h)
{
    if (!h) return WTMD_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaDeviceSynchronize();
    drop_graphs(h);
    for (int i = 0; i < h->ncv; ++i) free_cv(h->cv[i]);
    void* ptrs[] = {h->woff, h->wn, h->atom_walker, h->hills64, h->hills32, h->count, h->step, h->dep, h->status, h->ticket,
                    h->grid, h->gfac, h->xi, h->ctr, h->V, h->dV, h->J, h->partial, h->hev_xi, h->cell_count,
                    h->harm_centre, h->harm_sum,
                    h->cell_atoms, h->nl_nbr, h->nl_cnt, h->nl_xref, h->nl_ctl, h->ss.bar};
    for (void* p : ptrs) cudaFree(p);
    surrogate_free(h->sur);
    {
        WalkerPlan& k = h->wk;
        void* wp[] = {k.tasks, k.tbase, k.tcount, k.tpart, k.ticket, k.rgc, k.bar};
        for (void* p : wp) cudaFree(p);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (int c = 0; c < 3; ++c) {
        if (h->cv_stream[c]) cudaStreamDestroy(h->cv_stream[c]);
        if (h->ev_cv[c]) cudaEventDestroy(h->ev_cv[c]);
        if (h->jf_stream[c]) cudaStreamDestroy(h->jf_stream[c]);
        if (h->ev_jfork[c]) cudaEventDestroy(h->ev_jfork[c]);
        if (h->ev_jjoin[c]) cudaEventDestroy(h->ev_jjoin[c]);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return WTMD_OK;
}

extern "C" const char* wtmd_last_error(const wtmd_t* h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

extern "C" int wtmd_create(const wtmd_config* cfg, wtmd_t** out)
{
    if (!cfg || !out) return WTMD_EINVAL;
    *out = nullptr;
    const wtmd_config& c = *cfg;
    if (c.precision != WTMD_F32 && c.precision != WTMD_F64) return WTMD_EINVAL;
    if (c.n_cv < 1 || c.n_cv > 3) return WTMD_EINVAL;
    for (int i = 0; i < c.n_cv; ++i)
        if (!(c.sigma[i] > 0.0) || !isfinite(c.sigma[i])) return WTMD_EINVAL;
    if (!(c.w0 > 0.0) || !isfinite(c.w0)) return WTMD_EINVAL;
    if (!(c.gamma == 0.0 || isinf(c.gamma) || c.gamma > 1.0)) return WTMD_EINVAL;
    if (!(c.kT > 0.0)) return WTMD_EINVAL;
    if (c.stride < 0 || c.hill_capacity < 0) return WTMD_EINVAL;
    if (!(c.engine >= WTMD_ENGINE_NONE && c.engine <= WTMD_ENGINE_CHAIN) && c.engine != WTMD_ENGINE_WELLS3)
        return WTMD_EINVAL;
    if (c.n_walkers < 1 || !c.walker_size) return WTMD_EINVAL;
    if (!(c.dt > 0.0) || !(c.mass > 0.0) || c.friction < 0.0) return WTMD_EINVAL;
    const bool grid = c.grid_bins[0] > 0;
    for (int i = 0; i < c.n_cv; ++i) {
        if (grid != (c.grid_bins[i] > 0)) return WTMD_EINVAL;
        if (grid && !(c.grid_hi[i] > c.grid_lo[i])) return WTMD_EINVAL;
    }
    if (c.engine == WTMD_ENGINE_LJ && !(c.lj_rc > 0.0 && c.lj_sigma > 0.0)) return WTMD_EINVAL;

    wtmd_t* h = new (std::nothrow) wtmd_t();
    if (!h) return WTMD_ENOMEM;
    h->cfg = c;
    h->cfg.walker_size = nullptr;
    h->prec = c.precision;
    h->d = c.n_cv;
    h->dims = c.dims > 0 ? c.dims : (c.engine == WTMD_ENGINE_MB ? 2 : 3);
    if (h->dims < 2 || h->dims > 3) {
        delete h;
        return WTMD_EINVAL;
    }
    h->W = c.n_walkers;
    int64_t off = 0;
    for (int w = 0; w < h->W; ++w) {
        const int64_t n = c.walker_size[w];
        if (n < 1 || n > (1 << 30)) {
            delete h;
            return WTMD_EINVAL;
        }
        h->woff_h.push_back(off);
        h->wn_h.push_back(n);
        off += n;
        h->max_wn = std::max<int>(h->max_wn, (int)n);
    }
    h->N = off;
    const double log2e = 1.4426950408889634;
    for (int i = 0; i < 3; ++i) h->a[i] = i < h->d ? sqrt(log2e / 2.0) / c.sigma[i] : 0.0;
    for (int k = 0; k < 3; ++k) {
        h->box.L[k] = c.box[k] > 0.0 ? c.box[k] : 0.0;
        h->box.invL[k] = c.box[k] > 0.0 ? 1.0 / c.box[k] : 0.0;
        h->box.Lf[k] = (float)h->box.L[k];
        h->box.Llo[k] = (float)(h->box.L[k] - (double)h->box.Lf[k]);
        h->box.invLf[k] = (float)h->box.invL[k];
    }
    auto fail = [&](int code, const char* m) {
        h->err = m;
        wtmd_destroy(h);
        return code;
    };
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(WTMD_ECUDA, "streams");
    for (int c = 0; c < 3; ++c)
        if (cudaStreamCreateWithFlags(&h->cv_stream[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_cv[c], cudaEventDisableTiming) != cudaSuccess)
            return fail(WTMD_ECUDA, "streams");
    for (int c = 0; c < 3; ++c)
        if (cudaStreamCreateWithFlags(&h->jf_stream[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_jfork[c], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_jjoin[c], cudaEventDisableTiming) != cudaSuccess)
            return fail(WTMD_ECUDA, "streams");
    // walkers
    std::vector<int> aw(h->N), wn32(h->W);
    for (int w = 0; w < h->W; ++w) {
        wn32[w] = (int)h->wn_h[w];
        for (int64_t i = 0; i < h->wn_h[w]; ++i) aw[h->woff_h[w] + i] = w;
    }
    if (cudaMalloc(&h->woff, sizeof(int64_t) * h->W) || cudaMalloc(&h->wn, sizeof(int) * h->W) ||
        cudaMalloc(&h->atom_walker, sizeof(int) * h->N))
        return fail(WTMD_ENOMEM, "walker tables");
    cudaMemcpy(h->woff, h->woff_h.data(), sizeof(int64_t) * h->W, cudaMemcpyHostToDevice);
    cudaMemcpy(h->wn, wn32.data(), sizeof(int) * h->W, cudaMemcpyHostToDevice);
    cudaMemcpy(h->atom_walker, aw.data(), sizeof(int) * h->N, cudaMemcpyHostToDevice);
    // hills
    h->cap = c.hill_capacity;
    const int64_t CH = 128;  // chunk of the FP32 hills kernel (pairs)
    const int64_t pairs = (h->cap + 1) / 2;
    h->cap_pairs = std::max<int64_t>(CH, (pairs + CH - 1) / CH * CH);
    if (cudaMalloc(&h->hills64, 32 * (size_t)std::max<int64_t>(h->cap, 1)) ||
        cudaMalloc(&h->hills32, 32 * (size_t)h->cap_pairs))
        return fail(WTMD_ENOMEM, "hill list");
    cudaMemset(h->hills64, 0, 32 * (size_t)std::max<int64_t>(h->cap, 1));
    pad_hills32_kernel<<<(unsigned)((h->cap_pairs + 255) / 256), 256>>>(h->hills32, h->cap_pairs);
    if (cudaMalloc(&h->count, sizeof(long long)) || cudaMalloc(&h->step, sizeof(long long)) ||
        cudaMalloc(&h->dep, 2 * sizeof(long long)) || cudaMalloc(&h->status, sizeof(unsigned)) ||
        cudaMalloc(&h->ticket, sizeof(unsigned)))
        return fail(WTMD_ENOMEM, "counters");
    cudaMemset(h->count, 0, sizeof(long long));
    cudaMemset(h->step, 0, sizeof(long long));
    cudaMemset(h->dep, 0, 2 * sizeof(long long));
    cudaMemset(h->status, 0, sizeof(unsigned));
    cudaMemset(h->ticket, 0, sizeof(unsigned));
    // grid
    h->ncell = 0;
    h->gbins_sum = 0;
    if (grid) {
        h->ncell = 1;
        for (int i = 0; i < h->d; ++i) {
            h->ncell *= c.grid_bins[i];
            h->gbins_sum += c.grid_bins[i];
        }
        if (cudaMalloc(&h->grid, sizeof(double) * h->ncell)) return fail(WTMD_ENOMEM, "grid");
        cudaMemset(h->grid, 0, sizeof(double) * h->ncell);
    }
    if (cudaMalloc(&h->gfac, sizeof(double) * std::max<int64_t>(1, (int64_t)h->W * std::max(1, h->gbins_sum))))
        return fail(WTMD_ENOMEM, "grid factors");
    // per-walker and per-atom scratch
    if (cudaMalloc(&h->xi, sizeof(double) * 4 * h->W) || cudaMalloc(&h->ctr, sizeof(double) * 3) ||
        cudaMalloc(&h->V, realsz(h) * h->W) ||
        cudaMalloc(&h->dV, realsz(h) * 4 * h->W) || cudaMalloc(&h->J, r4sz(h) * h->d * (size_t)h->N))
        return fail(WTMD_ENOMEM, "scratch");
    cudaMemset(h->xi, 0, sizeof(double) * 4 * h->W);
    {
        // centre of the scaled FP32 hill layout: the grid's centre, else set
        // by the first loaded or deposited hills (NaN = not yet set)
        double c[3];
        for (int i = 0; i < 3; ++i)
            c[i] = i >= h->d ? 0.0 : (grid ? 0.5 * (c_lo(cfg, i) + c_hi(cfg, i)) : NAN);
        cudaMemcpy(h->ctr, c, sizeof(c), cudaMemcpyHostToDevice);
    }
    cudaMemset(h->dV, 0, realsz(h) * 4 * h->W);
    cudaMemset(h->J, 0, r4sz(h) * h->d * (size_t)h->N);
    if (setup_cells(h) != WTMD_OK) return fail(WTMD_ENOMEM, "cell list");
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(WTMD_ECUDA, "create");
    *out = h;
    return WTMD_OK;
}

extern "C" int wtmd_set_stream(wtmd_t* h, void* stream)
{
    if (!h) return WTMD_EINVAL;
    h->stream = (cudaStream_t)stream;
    return WTMD_OK;
}

static bool valid_list(const int32_t* a, int64_t n, int64_t limit, bool distinct)
{
    if (!a || n < 1) return false;
    std::vector<char> seen(distinct ? (size_t)limit : 0, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (a[i] < 0 || a[i] >= limit) return false;
        if (distinct) {
            if (seen[a[i]]) return false;
            seen[a[i]] = 1;
        }
    }
    return true;
}

extern "C" int cv_define(wtmd_t* h, const wtmd_cv_desc* d, int32_t* cv_id)
{
    if (!h) return WTMD_EINVAL;
    if (!d) FAIL(h, WTMD_EINVAL, "null CV description");
    if (h->ncv >= h->d) FAIL(h, WTMD_EINVAL, "all n_cv CVs are already defined");
    int64_t minw = h->wn_h[0];
    for (auto n : h->wn_h) minw = std::min(minw, n);
    CvDev c;
    c.kind = d->kind;
    c.axis = d->axis;
    c.nn = d->nn;
    c.flags = d->flags;
    c.r0 = d->r0;
    c.scale = d->scale;
    c.period = d->period;
    if (!(d->period >= 0.0) || !isfinite(d->period)) FAIL(h, WTMD_EINVAL, "bad period");
    if (!isfinite(d->scale)) FAIL(h, WTMD_EINVAL, "bad scale");
    auto upload = [&](const int32_t* src, int64_t n, int** dst) -> int {
        if (cudaMalloc(dst, sizeof(int) * n) != cudaSuccess) return WTMD_ENOMEM;
        cudaMemcpy(*dst, src, sizeof(int) * n, cudaMemcpyHostToDevice);
        return WTMD_OK;
    };
    switch (d->kind) {
    case WTMD_CV_COMPONENT:
        if (d->n_a != 1 || !valid_list(d->a, 1, minw, true)) FAIL(h, WTMD_EINVAL, "COMPONENT needs 1 atom index");
        if (d->axis < 0 || d->axis > 2) FAIL(h, WTMD_EINVAL, "COMPONENT axis must be 0, 1 or 2");
        c.hidx[0] = d->a[0];
        c.n_a = 1;
        break;
    case WTMD_CV_DIHEDRAL:
        if (d->n_a != 4 || !valid_list(d->a, 4, minw, true)) FAIL(h, WTMD_EINVAL, "DIHEDRAL needs 4 distinct atoms");
        for (int k = 0; k < 4; ++k) c.hidx[k] = d->a[k];
        c.n_a = 4;
        break;
    case WTMD_CV_ANGLE:
        if (d->n_a != 3 || !valid_list(d->a, 3, minw, true)) FAIL(h, WTMD_EINVAL, "ANGLE needs 3 distinct atoms");
        for (int k = 0; k < 3; ++k) c.hidx[k] = d->a[k];
        c.n_a = 3;
        break;
    case WTMD_CV_DISTANCE: {
        if (d->n_a < 1 || d->n_b < 1 || !valid_list(d->a, d->n_a, minw, true) || !valid_list(d->b, d->n_b, minw, true))
            FAIL(h, WTMD_EINVAL, "DISTANCE needs two non-empty groups of distinct atoms");
        std::vector<char> inA(minw, 0);
        for (int64_t p = 0; p < d->n_a; ++p) inA[d->a[p]] = 1;
        for (int64_t p = 0; p < d->n_b; ++p)
            if (inA[d->b[p]]) FAIL(h, WTMD_EINVAL, "DISTANCE groups must be disjoint");
        c.n_a = (int)d->n_a;
        c.n_b = (int)d->n_b;
        if (upload(d->a, d->n_a, &c.a) || upload(d->b, d->n_b, &c.b)) FAIL(h, WTMD_ENOMEM, "DISTANCE groups");
        break;
    }
    case WTMD_CV_GYRATION:
        if (d->axis < 0 || d->axis > 5) FAIL(h, WTMD_EINVAL, "GYRATION quantity (axis) must be 0..5");
        [[fallthrough]];
    case WTMD_CV_RG:
        c.n_a = (int)d->n_a;
        if (d->n_a == -1) {
            if (minw < 2) FAIL(h, WTMD_EINVAL, "RG / GYRATION needs at least 2 atoms");
        } else {
            if (d->n_a < 2 || !valid_list(d->a, d->n_a, minw, true)) FAIL(h, WTMD_EINVAL, "bad RG / GYRATION group");
            if (upload(d->a, d->n_a, &c.a)) FAIL(h, WTMD_ENOMEM, "RG / GYRATION group");
        }
        break;
    case WTMD_CV_COORDINATION:
    case WTMD_CV_QPAIRS: {
        if (!(d->r0 > 0.0)) FAIL(h, WTMD_EINVAL, "r0 must be > 0");
        if (d->nn < 2 || d->nn > 16 || d->nn % 2 || d->mm != 2 * d->nn)
            FAIL(h, WTMD_EINVAL, "switching exponents: nn even in 2..16 and mm = 2 nn");
        if (d->kind == WTMD_CV_QPAIRS) {
            if (d->n_a < 2 || d->n_a % 2 || !valid_list(d->a, d->n_a, minw, false))
                FAIL(h, WTMD_EINVAL, "QPAIRS needs 2*npairs indices");
            for (int64_t p = 0; p < d->n_a / 2; ++p)
                if (d->a[2 * p] == d->a[2 * p + 1]) FAIL(h, WTMD_EINVAL, "QPAIRS pair of one atom");
            c.n_pairs = (int)(d->n_a / 2);
            c.n_a = (int)d->n_a;
            if (upload(d->a, d->n_a, &c.a)) FAIL(h, WTMD_ENOMEM, "pairs");
            std::vector<int> cntv(h->max_wn + 1, 0), items(d->n_a);
            for (int64_t q = 0; q < d->n_a; ++q) cntv[d->a[q] + 1]++;
            for (int k = 0; k < h->max_wn; ++k) cntv[k + 1] += cntv[k];
            std::vector<int> fill(cntv.begin(), cntv.end() - 1);
            for (int64_t q = 0; q < d->n_a; ++q) items[fill[d->a[q]]++] = (int)((q / 2) * 2 + (q & 1));
            if (upload(cntv.data(), h->max_wn + 1, &c.q_rowptr) || upload(items.data(), d->n_a, &c.q_items))
                FAIL(h, WTMD_ENOMEM, "pair CSR");
            break;
        }
        c.n_a = (int)d->n_a;
        c.n_b = (int)d->n_b;
        if (d->n_a != -1 && !valid_list(d->a, d->n_a, minw, true)) FAIL(h, WTMD_EINVAL, "bad group A");
        if (d->n_b != -1 && !valid_list(d->b, d->n_b, minw, true)) FAIL(h, WTMD_EINVAL, "bad group B");
        if (d->n_a == -1 && d->n_b == -1) c.same_ab = true;
        if (d->n_a > 0 && d->n_a == d->n_b && !memcmp(d->a, d->b, sizeof(int32_t) * d->n_a)) c.same_ab = true;
        std::vector<int> inv(h->max_wn, -1);
        if (d->n_a > 0) {
            for (int64_t p = 0; p < d->n_a; ++p) inv[d->a[p]] = (int)p;
            if (upload(d->a, d->n_a, &c.a) || upload(inv.data(), h->max_wn, &c.inv_a)) FAIL(h, WTMD_ENOMEM, "A");
        }
        if (d->n_b > 0) {
            std::fill(inv.begin(), inv.end(), -1);
            for (int64_t p = 0; p < d->n_b; ++p) inv[d->b[p]] = (int)p;
            if (upload(d->b, d->n_b, &c.b) || upload(inv.data(), h->max_wn, &c.inv_b)) FAIL(h, WTMD_ENOMEM, "B");
        }
        // target order: members of A (in A's order), then members of B not in
        // A (increasing); "all" means every atom index below the largest
        // walker size (kernels skip indices beyond a walker's own size)
        if (!(d->n_a == -1)) {
            std::vector<char> inA(h->max_wn, 0);
            for (int64_t p = 0; p < d->n_a; ++p) inA[d->a[p]] = 1;
            std::vector<int> ord(d->a, d->a + d->n_a);
            for (int k = 0; k < h->max_wn; ++k) {
                bool inB = d->n_b == -1;
                if (!inB) inB = std::find(d->b, d->b + d->n_b, k) != d->b + d->n_b;
                if (inB && !inA[k]) ord.push_back(k);
            }
            c.n_order = (int)ord.size();
            if (upload(ord.data(), (int64_t)ord.size(), &c.order)) FAIL(h, WTMD_ENOMEM, "target order");
        }
        break;
    }
    default:
        FAIL(h, WTMD_EINVAL, "unknown CV kind");
    }
    const int rc = cv_alloc_scratch(h, c);
    if (rc != WTMD_OK) {
        free_cv(c);
        return rc;
    }
    h->cv[h->ncv] = c;
    if (cv_id) *cv_id = h->ncv;
    h->ncv++;
    drop_graphs(h);
    return WTMD_OK;
}

extern "C" int wtmd_bind(wtmd_t* h, void* pos, void* vel, void* force, int64_t n_atoms)
{
    if (!h) return WTMD_EINVAL;
    if (n_atoms != h->N) FAIL(h, WTMD_EINVAL, "n_atoms differs from the sum of walker sizes");
    if (!pos || !force) FAIL(h, WTMD_EINVAL, "positions and forces are required");
    const uintptr_t al = h->prec == WTMD_F32 ? 16 : 32;
    if ((uintptr_t)pos % al || (uintptr_t)force % al || (vel && (uintptr_t)vel % al))
        FAIL(h, WTMD_EINVAL, "particle arrays must be 16-byte (F32) / 32-byte (F64) aligned");
    h->pos = pos;
    h->vel = vel;
    h->force = force;
    h->forces_valid = false;
    drop_graphs(h);
    return WTMD_OK;
}

// Total force at the bound positions (engine + bias), no kick, no deposit.
static int enqueue_forces(wtmd_t* h)
{
    if (h->persistent) return launch_walkers_step(h, 1);
    int rc;
    if ((rc = nl_request(h)) || (rc = launch_engine(h)) || (rc = nl_reset(h))) return rc;
    if ((rc = launch_cvs(h, h->pos))) return rc;
    if ((rc = launch_bias_sum(h))) return rc;
    return launch_scatter(h, h->force, nullptr, false);
}

// Engine force and bias (CVs -> hills sum) both only read the positions, so
// they run as parallel branches of the captured graph: the engine on the
// main stream, the bias chain forked from it and joined back before the
// closing kick.  While profiling, the two run in sequence so that each
// kernel's event interval is its own.
static int enqueue_engine_and_bias(wtmd_t* h)
{
    int rc;
    const bool fork = !h->prof;
    if (!fork) {
        if ((rc = launch_engine(h)) || (rc = launch_cvs(h, h->pos))) return rc;
        return launch_bias_sum(h);
    }
    // the bias chain (CV 0 -> hills sum) on its own branch, CVs 1 and 2 on
    // theirs, the engine on the main stream; the closing kick joins them
    WTMD_CUDA_TRY(h, cudaEventRecord(h->ev_fork, h->stream));
    cudaStream_t main_stream = h->stream;
    const int folded = folded_rg(h);  // computed by CV 0's launch: no branch of its own
    for (int c = 1; c < h->ncv; ++c) {
        if (c == folded) continue;
        WTMD_CUDA_TRY(h, cudaStreamWaitEvent(h->cv_stream[c], h->ev_fork, 0));
        h->stream = h->cv_stream[c];
        rc = launch_cv(h, h->pos, c);
        h->stream = main_stream;
        if (rc) return rc;
        WTMD_CUDA_TRY(h, cudaEventRecord(h->ev_cv[c], h->cv_stream[c]));
    }
    WTMD_CUDA_TRY(h, cudaStreamWaitEvent(h->cv_stream[0], h->ev_fork, 0));
    h->stream = h->cv_stream[0];
    rc = launch_cv(h, h->pos, 0);
    for (int c = 1; c < h->ncv && !rc; ++c)
        if (c != folded && cudaStreamWaitEvent(h->stream, h->ev_cv[c], 0) != cudaSuccess) rc = WTMD_ECUDA;
    if (!rc) rc = launch_bias_sum(h);
    if (!rc && cudaEventRecord(h->ev_join, h->stream) != cudaSuccess) rc = WTMD_ECUDA;
    h->stream = main_stream;
    if (rc) return rc;
    if ((rc = launch_engine(h))) return rc;
    WTMD_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    return WTMD_OK;
}

// The step as one persistent launch when the handle's form allows it and
// its plan is set up (sys_step.cu), else as the per-kernel sequence.
static bool use_sys_step(const wtmd_t* h)
{
    return h->fused_on && h->ss.ready && sys_step_eligible(h, nullptr);
}

// Set up the persistent step's plan outside graph capture (a no-op when it
// is ready, switched off or not applicable).
static int prepare_sys_step(wtmd_t* h)
{
    if (!h->fused_on || h->ss.ready || !sys_step_eligible(h, nullptr)) return WTMD_OK;
    return sys_step_setup(h);
}

static int enqueue_step(wtmd_t* h)
{
    if (h->persistent) return launch_walkers_step(h, 0);
    if (small_step_eligible(h)) return launch_small_steps(h, 1);
    if (use_sys_step(h)) return launch_sys_step(h);
    int rc;
    h->jf_pending = 0;
    // BAOAB zeroes what the coordination tile kernels accumulate (the FP64
    // kernel's Jacobian rows, the FP32 kernel's CV value), so that the CV
    // kernels directly follow it (programmatic dependent launches: previous
    // step -> BAOAB -> CVs)
    int jmask = 0, xmask = 0;
    for (int c = 0; c < h->ncv; ++c) {
        if (coord_factored(h, c)) xmask |= 1 << c;
        else if (h->cv[c].kind == WTMD_CV_COORDINATION && h->cv[c].n_a > 0) jmask |= 1 << c;
    }
    if ((rc = launch_baoab_first(h, jmask, xmask))) return rc;
    h->jz_pre = true;
    h->in_step = true;
    rc = enqueue_engine_and_bias(h);
    h->jz_pre = false;
    h->in_step = false;
    if (rc) return rc;
    return launch_scatter_deposit(h);
}

static int capture(wtmd_t* h, int nsteps, cudaGraphExec_t* out)
{
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->stream = user;
        FAIL(h, WTMD_ECUDA, "begin capture");
    }
    int rc = WTMD_OK;
    for (int s = 0; s < nsteps && rc == WTMD_OK; ++s) rc = enqueue_step(h);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    h->stream = user;
    if (rc != WTMD_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) FAIL(h, WTMD_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) FAIL(h, WTMD_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return WTMD_OK;
}

static int ready(wtmd_t* h)
{
    if (h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs first");
    return WTMD_OK;
}

static int run_steps(wtmd_t* h, int64_t n_steps)
{
    int rc;
    if (small_step_eligible(h)) return launch_small_steps(h, n_steps);  // many steps per launch, no graph
    if (!h->graph && !h->no_graph) {
        if (capture(h, kGraphSteps, &h->graph) != WTMD_OK || capture(h, 1, &h->graph1) != WTMD_OK) {
            // this launch sequence cannot be captured here: replay eagerly
            cudaGetLastError();
            drop_graphs(h);
            h->no_graph = true;
        }
    }
    if (h->no_graph) {
        for (int64_t i = 0; i < n_steps; ++i)
            if ((rc = enqueue_step(h))) return rc;
        return WTMD_OK;
    }
    const int64_t full = n_steps / kGraphSteps, rest = n_steps % kGraphSteps;
    for (int64_t i = 0; i < full; ++i) WTMD_CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
    for (int64_t i = 0; i < rest; ++i) WTMD_CUDA_TRY(h, cudaGraphLaunch(h->graph1, h->stream));
    return WTMD_OK;
}

extern "C" int step_n(wtmd_t* h, int64_t n_steps)
{
    if (!h) return WTMD_EINVAL;
    if (n_steps < 0) FAIL(h, WTMD_EINVAL, "negative step count");
    int rc = ready(h);
    if (rc) return rc;
    if (!h->pos || !h->vel || !h->force) FAIL(h, WTMD_EINVAL, "bind positions, velocities and forces first");
    if (n_steps == 0) return WTMD_OK;
    if ((rc = launch_hills_partial_prealloc(h, h->W))) return rc;
    if ((rc = prepare_sys_step(h))) return rc;
    if (!h->forces_valid) {
        if ((rc = enqueue_forces(h))) return rc;
        h->forces_valid = true;
    }
    // with the surrogate on, the run is cut where a refit is due
    for (int64_t left = n_steps; left > 0;) {
        int64_t seg = left;
        if ((rc = surrogate_segment(h, left, &seg))) return rc;
        if ((rc = run_steps(h, seg))) return rc;
        surrogate_advanced(h, seg);
        left -= seg;
    }
    return WTMD_OK;
}

// One captured graph: the packed state [3][N][4] in from pinned host memory,
// one step, the state out to pinned host memory.
static int capture_host(wtmd_t* h, const void* in, void* out, size_t bytes)
{
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->stream = user;
        FAIL(h, WTMD_ECUDA, "begin capture");
    }
    int rc = WTMD_OK;
    if (cudaMemcpyAsync(h->pos, in, bytes, cudaMemcpyHostToDevice, h->cap_stream) != cudaSuccess) rc = WTMD_ECUDA;
    if (!rc) rc = enqueue_step(h);
    if (!rc && cudaMemcpyAsync(out, h->pos, bytes, cudaMemcpyDeviceToHost, h->cap_stream) != cudaSuccess)
        rc = WTMD_ECUDA;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    h->stream = user;
    if (rc != WTMD_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        FAIL(h, rc ? rc : WTMD_ECUDA, "capture of the host-buffer step");
    }
    e = cudaGraphInstantiate(&h->graph_host, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph_host = nullptr;
        FAIL(h, WTMD_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    h->gh_in = in;
    h->gh_out = out;
    return WTMD_OK;
}

static bool pinned(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

extern "C" int wtmd_step_host(wtmd_t* h, const void* in_host, void* out_host, int64_t n_steps, int32_t wait)
{
    if (!h) return WTMD_EINVAL;
    if (n_steps < 1 || !in_host || !out_host) FAIL(h, WTMD_EINVAL, "need n_steps >= 1 and host buffers");
    int rc = ready(h);
    if (rc) return rc;
    if (!h->pos || !h->vel || !h->force) FAIL(h, WTMD_EINVAL, "bind positions, velocities and forces first");
    const size_t pb = r4sz(h) * (size_t)h->N;
    const bool packed = (char*)h->vel == (char*)h->pos + pb && (char*)h->force == (char*)h->vel + pb;
    const bool one_graph = packed && n_steps == 1 && h->forces_valid && !h->persistent && !surrogate_k0(h) &&
                           !h->no_graph && !h->no_host_graph && !h->prof && pinned(in_host) && pinned(out_host);
    if (one_graph) {
        if ((rc = launch_hills_partial_prealloc(h, h->W))) return rc;
        if ((rc = prepare_sys_step(h))) return rc;
        if (!h->graph_host || h->gh_in != in_host || h->gh_out != out_host) {
            if (h->graph_host) cudaGraphExecDestroy(h->graph_host);
            h->graph_host = nullptr;
            if (capture_host(h, in_host, out_host, 3 * pb) != WTMD_OK) {
                cudaGetLastError();
                h->no_host_graph = true;  // this launch sequence cannot be captured here
            }
        }
        if (h->graph_host) {
            WTMD_CUDA_TRY(h, cudaGraphLaunch(h->graph_host, h->stream));
            if (wait) WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            return WTMD_OK;
        }
    }
    const char* src = (const char*)in_host;
    void* dev[3] = {h->pos, h->vel, h->force};
    for (int k = 0; k < 3; ++k)
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(dev[k], src + k * pb, pb, cudaMemcpyHostToDevice, h->stream));
    if ((rc = step_n(h, n_steps))) return rc;
    char* dst = (char*)out_host;
    for (int k = 0; k < 3; ++k)
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(dst + k * pb, dev[k], pb, cudaMemcpyDeviceToHost, h->stream));
    if (wait) WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return WTMD_OK;
}

extern "C" int wtmd_check(wtmd_t* h)
{
    if (!h) return WTMD_EINVAL;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    WTMD_CUDA_TRY(h, cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
    WTMD_CUDA_TRY(h, cudaMemset(h->status, 0, sizeof(unsigned)));
    if (st & ST_TIMEOUT) {
        // a barrier that gave up leaves its arrival counter dirty
        if (h->ss.bar) WTMD_CUDA_TRY(h, cudaMemset(h->ss.bar, 0, sizeof(unsigned) * 4));
        FAIL(h, WTMD_ETIMEOUT, "a bounded device wait gave up");
    }
    if (st & ST_NUMERIC) FAIL(h, WTMD_ENUMERIC, "non-finite CV, bias or gradient");
    if (st & ST_CELL) FAIL(h, WTMD_ECELL, "cell list overflow");
    if (st & ST_CAPACITY) FAIL(h, WTMD_ECAPACITY, "hill capacity reached; deposits skipped");
    return WTMD_OK;
}

template <typename S, typename D>
__global__ static void copy_cols_kernel(const S* __restrict__ src, D* __restrict__ dst, int W, int cols)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * cols) return;
    dst[i] = (D)src[(i / cols) * 4 + i % cols];
}

// [W][4] (double CV values or Real gradients) -> [W][cols] Real
static int copy_cols(wtmd_t* h, void* dst, const void* src, bool src_f64, int cols)
{
    const int n = h->W * cols, nb = (n + 255) / 256;
    if (h->prec == WTMD_F64)
        copy_cols_kernel<double, double><<<nb, 256, 0, h->stream>>>((const double*)src, (double*)dst, h->W, cols);
    else if (src_f64)
        copy_cols_kernel<double, float><<<nb, 256, 0, h->stream>>>((const double*)src, (float*)dst, h->W, cols);
    else
        copy_cols_kernel<float, float><<<nb, 256, 0, h->stream>>>((const float*)src, (float*)dst, h->W, cols);
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

// bias_eval's outputs in one launch: V [W] and the [W][4] CV values (double)
// and gradients (Real) as [W][d] Real, any of them optional
template <typename R>
__global__ static void bias_out_kernel(const R* __restrict__ V, const double* __restrict__ xi,
                                       const R* __restrict__ dV, R* __restrict__ V_out, R* __restrict__ xi_out,
                                       R* __restrict__ dV_out, int W, int d)
{
    pdl_wait();  // a programmatic dependent of the bias force kernel
    pdl_trigger();
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    if (V_out) V_out[w] = V[w];
    for (int c = 0; c < d; ++c) {
        if (xi_out) xi_out[w * d + c] = (R)xi[w * 4 + c];
        if (dV_out) dV_out[w * d + c] = dV[w * 4 + c];
    }
}

extern "C" int bias_eval(wtmd_t* h, const void* pos, void* force_inout, void* V_out, void* xi_out, void* dV_out)
{
    if (!h) return WTMD_EINVAL;
    int rc = ready(h);
    if (rc) return rc;
    if (!pos) FAIL(h, WTMD_EINVAL, "null positions");
    if ((rc = launch_hills_partial_prealloc(h, h->W))) return rc;
    // the J rows of a tile coordination CV go on a branch beside the hills
    // sum (which needs only xi); the scatter joins it
    h->jbranch = true;
    rc = launch_cvs(h, pos);
    h->jbranch = false;
    if (rc) return rc;
    if ((rc = launch_bias_sum(h))) return rc;
    if ((rc = join_jbranches(h))) return rc;
    if (force_inout && (rc = launch_scatter(h, force_inout, nullptr, false))) return rc;
    if (V_out || xi_out || dV_out) {
        const int nb = (h->W + 127) / 128;
        if (h->prec == WTMD_F32)
            WTMD_CUDA_TRY(h, launch_pdl(bias_out_kernel<float>, dim3(nb), dim3(128), 0, h->stream, (const float*)h->V,
                                        (const double*)h->xi, (const float*)h->dV, (float*)V_out, (float*)xi_out,
                                        (float*)dV_out, h->W, h->d));
        else
            WTMD_CUDA_TRY(h, launch_pdl(bias_out_kernel<double>, dim3(nb), dim3(128), 0, h->stream,
                                        (const double*)h->V, (const double*)h->xi, (const double*)h->dV,
                                        (double*)V_out, (double*)xi_out, (double*)dV_out, h->W, h->d));
    }
    return WTMD_OK;
}

extern "C" int wtmd_cv_forward(wtmd_t* h, const void* pos, void* xi_out)
{
    if (!h) return WTMD_EINVAL;
    int rc = ready(h);
    if (rc) return rc;
    if (!pos || !xi_out) FAIL(h, WTMD_EINVAL, "null positions or output");
    if ((rc = launch_cvs(h, pos))) return rc;
    return copy_cols(h, xi_out, h->xi, true, h->d);
}

extern "C" int wtmd_cv_adjoint(wtmd_t* h, const void* grad_xi, void* grad_pos)
{
    if (!h) return WTMD_EINVAL;
    int rc = ready(h);
    if (rc) return rc;
    if (!grad_xi || !grad_pos) FAIL(h, WTMD_EINVAL, "null gradient");
    return launch_adjoint(h, grad_xi, grad_pos);
}

extern "C" int hills_eval(wtmd_t* h, const void* xi, int64_t P, void* V_out, void* dV_out)
{
    if (!h) return WTMD_EINVAL;
    if (P < 0 || (P > 0 && !xi)) FAIL(h, WTMD_EINVAL, "bad points");
    if (h->ncv > 0 && h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs (or none) first");
    return launch_hills(h, xi, h->prec == WTMD_F64, h->d, P, V_out, dV_out, h->d);
}

extern "C" int wtmd_grid_eval(wtmd_t* h, const void* xi, int64_t P, void* V_out, void* dV_out)
{
    if (!h) return WTMD_EINVAL;
    if (!h->grid) FAIL(h, WTMD_EINVAL, "the handle has no grid");
    for (int i = 0; i < h->d; ++i)
        if (h->cfg.grid_bins[i] < 2) FAIL(h, WTMD_EINVAL, "every grid axis needs at least 2 cells");
    if (P < 0 || (P > 0 && !xi)) FAIL(h, WTMD_EINVAL, "bad points");
    if (P > (1ll << 40)) FAIL(h, WTMD_EINVAL, "too many points");
    if (h->ncv > 0 && h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs (or none) first");
    return launch_grid_bias(h, xi, h->prec == WTMD_F64, h->d, P, V_out, dV_out, h->d, false);
}

extern "C" int wtmd_bias_source(wtmd_t* h, int32_t source)
{
    if (!h) return WTMD_EINVAL;
    if (source != WTMD_BIAS_HILLS && source != WTMD_BIAS_GRID && source != WTMD_BIAS_HARMONIC)
        FAIL(h, WTMD_EINVAL, "unknown bias source");
    if (source == WTMD_BIAS_HARMONIC) {
        if (!h->harm_centre) FAIL(h, WTMD_EINVAL, "set the windows with wtmd_harmonic first");
        if (!h->bias_harm) {
            h->bias_harm = true;
            h->bias_grid = false;
            drop_graphs(h);
        }
        return WTMD_OK;
    }
    if (h->bias_harm) {
        h->bias_harm = false;
        drop_graphs(h);
    }
    const bool grid = source == WTMD_BIAS_GRID;
    if (grid) {
        if (!h->grid) FAIL(h, WTMD_EINVAL, "the handle has no grid");
        if (h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs first");
        for (int i = 0; i < h->d; ++i) {
            if (h->cfg.grid_bins[i] < 2) FAIL(h, WTMD_EINVAL, "every grid axis needs at least 2 cells");
            const double per = h->cv[i].period, span = h->cfg.grid_hi[i] - h->cfg.grid_lo[i];
            if (per > 0.0 && fabs(span - per) > 1e-9 * per)
                FAIL(h, WTMD_EINVAL, "the grid of a periodic CV must span exactly one period");
        }
        if (surrogate_k0(h)) FAIL(h, WTMD_EINVAL, "turn the surrogate off first");
    }
    if (grid != h->bias_grid) {
        h->bias_grid = grid;
        drop_graphs(h);
    }
    return WTMD_OK;
}

extern "C" int wtmd_harmonic(wtmd_t* h, const double* k, const double* centres)
{
    if (!h) return WTMD_EINVAL;
    if (!k || !centres) FAIL(h, WTMD_EINVAL, "null spring constants or centres");
    if (h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs first");
    if (surrogate_k0(h)) FAIL(h, WTMD_EINVAL, "turn the surrogate off first");
    for (int c = 0; c < h->d; ++c)
        if (!(k[c] > 0.0) || !isfinite(k[c])) FAIL(h, WTMD_EINVAL, "spring constants must be finite and > 0");
    std::vector<double> cen(4 * (size_t)h->W, 0.0);
    for (int w = 0; w < h->W; ++w)
        for (int c = 0; c < h->d; ++c) {
            const double v = centres[(size_t)w * h->d + c];
            if (!isfinite(v)) FAIL(h, WTMD_EINVAL, "non-finite window centre");
            cen[4 * (size_t)w + c] = v;
        }
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (!h->harm_centre) {
        WTMD_CUDA_TRY(h, cudaMalloc(&h->harm_centre, sizeof(double) * 4 * h->W));
        WTMD_CUDA_TRY(h, cudaMalloc(&h->harm_sum, sizeof(double) * (4 * h->W + 1)));
    }
    WTMD_CUDA_TRY(h, cudaMemcpy(h->harm_centre, cen.data(), sizeof(double) * 4 * h->W, cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemset(h->harm_sum, 0, sizeof(double) * (4 * h->W + 1)));
    for (int c = 0; c < 3; ++c) h->harm_k[c] = c < h->d ? k[c] : 0.0;
    h->bias_harm = true;
    h->bias_grid = false;
    drop_graphs(h);
    return WTMD_OK;
}

extern "C" int wtmd_umbrella_stats(wtmd_t* h, double* mean_out, int64_t* n_samples, int32_t reset)
{
    if (!h) return WTMD_EINVAL;
    if (!h->harm_sum) FAIL(h, WTMD_EINVAL, "no windows (wtmd_harmonic)");
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    std::vector<double> sum(4 * (size_t)h->W + 1);
    WTMD_CUDA_TRY(h, cudaMemcpy(sum.data(), h->harm_sum, sizeof(double) * sum.size(), cudaMemcpyDeviceToHost));
    const double n = sum[4 * (size_t)h->W];
    if (n_samples) *n_samples = (int64_t)n;
    if (mean_out)
        for (int w = 0; w < h->W; ++w)
            for (int c = 0; c < h->d; ++c) mean_out[(size_t)w * h->d + c] = n > 0 ? sum[4 * (size_t)w + c] / n : 0.0;
    if (reset) WTMD_CUDA_TRY(h, cudaMemset(h->harm_sum, 0, sizeof(double) * sum.size()));
    return WTMD_OK;
}

// Umbrella integration (Sec. 2.1.2) on the host from the windows' mean CVs:
// a few W x d numbers, no device work beyond reading the sums.
extern "C" int wtmd_umbrella_integrate(wtmd_t* h, double* mean_force_out, double* A_out)
{
    if (!h) return WTMD_EINVAL;
    std::vector<double> mean((size_t)h->W * h->d), cen(4 * (size_t)h->W);
    int64_t n = 0;
    int rc = wtmd_umbrella_stats(h, mean.data(), &n, 0);
    if (rc) return rc;
    if (n < 1) FAIL(h, WTMD_EINVAL, "no samples yet (run steps with the harmonic bias)");
    WTMD_CUDA_TRY(h, cudaMemcpy(cen.data(), h->harm_centre, sizeof(double) * cen.size(), cudaMemcpyDeviceToHost));
    const int d = h->d;
    std::vector<double> g((size_t)h->W * d);
    auto wrap = [&](double D, int c) {
        const double per = h->cv[c].period;
        return per > 0.0 ? D - per * std::nearbyint(D / per) : D;
    };
    for (int w = 0; w < h->W; ++w)
        for (int c = 0; c < d; ++c)
            g[(size_t)w * d + c] = -h->harm_k[c] * wrap(mean[(size_t)w * d + c] - cen[4 * (size_t)w + c], c);
    if (mean_force_out) std::memcpy(mean_force_out, g.data(), sizeof(double) * g.size());
    if (A_out) {
        A_out[0] = 0.0;
        for (int w = 0; w + 1 < h->W; ++w) {
            double dA = 0.0;
            for (int c = 0; c < d; ++c)
                dA += 0.5 * (g[(size_t)w * d + c] + g[(size_t)(w + 1) * d + c]) *
                      wrap(mean[(size_t)(w + 1) * d + c] - mean[(size_t)w * d + c], c);
            A_out[w + 1] = A_out[w] + dA;
        }
    }
    return WTMD_OK;
}

extern "C" int wtmd_hills_tune(wtmd_t* h, int64_t P, int32_t* choice, double* ms)
{
    if (!h) return WTMD_EINVAL;
    if (h->ncv != h->d) FAIL(h, WTMD_EINVAL, "define all n_cv CVs first");
    int th = 0, sp = 0;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const int rc = hills_tune(h, P, &th, &sp, ms);
    if (rc) return rc;
    drop_graphs(h);  // recapture with the tuned plan
    if (choice) {
        choice[0] = th;
        choice[1] = sp;
    }
    return WTMD_OK;
}

extern "C" int wtmd_hills_plan(wtmd_t* h, int64_t P, int32_t lanes, int32_t splits)
{
    if (!h) return WTMD_EINVAL;
    const int rc = hills_set_plan(h, P, lanes, splits);
    if (rc) return rc;
    drop_graphs(h);  // recapture with the plan
    return WTMD_OK;
}

extern "C" int fes_grid(wtmd_t* h, double* out, int64_t n_out)
{
    if (!h) return WTMD_EINVAL;
    if (!h->grid) FAIL(h, WTMD_EINVAL, "no grid configured");
    if (!out || n_out < h->ncell) FAIL(h, WTMD_EINVAL, "output smaller than the grid");
    return launch_fes(h, out);
}

extern "C" int wtmd_hills_load(wtmd_t* h, const double* hills, int64_t count)
{
    if (!h) return WTMD_EINVAL;
    if (count < 0 || count > h->cap || (count > 0 && !hills)) FAIL(h, WTMD_EINVAL, "count outside 0..capacity");
    for (int64_t k = 0; k < count; ++k) {
        const double w = hills[4 * k + 3];
        if (!(w > 0.0) || !isfinite(w)) FAIL(h, WTMD_EINVAL, "hill heights must be finite and > 0");
        for (int i = 0; i < 3; ++i)
            if (!isfinite(hills[4 * k + i])) FAIL(h, WTMD_EINVAL, "non-finite hill centre");
    }
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (count) WTMD_CUDA_TRY(h, cudaMemcpy(h->hills64, hills, 32 * (size_t)count, cudaMemcpyHostToDevice));
    long long c = count;
    WTMD_CUDA_TRY(h, cudaMemcpy(h->count, &c, sizeof(c), cudaMemcpyHostToDevice));
    double ctr[3];
    WTMD_CUDA_TRY(h, cudaMemcpy(ctr, h->ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
    if (isnan(ctr[0]) && count > 0) {
        for (int i = 0; i < 3; ++i) {
            double m = 0.0;
            for (int64_t k = 0; k < count; ++k) m += hills[4 * k + i];
            ctr[i] = i < h->d ? m / count : 0.0;
        }
        WTMD_CUDA_TRY(h, cudaMemcpy(h->ctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice));
    }
    pad_hills32_kernel<<<(unsigned)((h->cap_pairs + 255) / 256), 256, 0, h->stream>>>(h->hills32, h->cap_pairs);
    store_hills32_range(h, 0, count);
    int rc = launch_grid_rebuild(h);
    if (rc) return rc;
    if ((rc = surrogate_invalidate(h))) return rc;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return WTMD_OK;
}

extern "C" int wtmd_hills_read(wtmd_t* h, double* out, int64_t cap_out, int64_t* count)
{
    if (!h) return WTMD_EINVAL;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    long long c = 0;
    WTMD_CUDA_TRY(h, cudaMemcpy(&c, h->count, sizeof(c), cudaMemcpyDeviceToHost));
    if (count) *count = c;
    const int64_t n = std::min<int64_t>(c, cap_out);
    if (n > 0 && out) WTMD_CUDA_TRY(h, cudaMemcpy(out, h->hills64, 32 * (size_t)n, cudaMemcpyDeviceToHost));
    return WTMD_OK;
}

extern "C" int wtmd_counters(wtmd_t* h, int64_t* step, int64_t* n_hills)
{
    if (!h) return WTMD_EINVAL;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    long long s = 0, c = 0;
    WTMD_CUDA_TRY(h, cudaMemcpy(&s, h->step, sizeof(s), cudaMemcpyDeviceToHost));
    WTMD_CUDA_TRY(h, cudaMemcpy(&c, h->count, sizeof(c), cudaMemcpyDeviceToHost));
    if (step) *step = s;
    if (n_hills) *n_hills = c;
    return WTMD_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / restart.  The blob is the raw bytes of everything a step reads
// that the handle owns -- hill count, step counter, the centre of the scaled
// FP32 hill layout, both hill layouts, the FP64 grid -- and of the bound
// particle arrays.  Because the thermostat noise is a counter-based stream
// keyed by (seed, step, particle), restoring these bytes resumes the run
// bitwise.  Layout: CkHeader, then hills64 [count][4] double, hills32
// [cap_pairs][2] float4, grid [ncell] double, positions, velocities, forces
// [N][4] Real.
struct CkHeader {
    uint64_t magic;  // "WTMDCKP1"
    int32_t version, prec, d, W;
    int64_t N, cap, cap_pairs, ncell, count, step;
    double ctr[3];
    int64_t total;  // bytes of the whole blob
};
static const uint64_t kCkMagic = 0x31504b43444d5457ull;  // "WTMDCKP1" little-endian

static int ck_layout(wtmd_t* h, int64_t count, int64_t* total)
{
    const int64_t pb = (int64_t)r4sz(h) * h->N;
    *total = (int64_t)sizeof(CkHeader) + 32 * count + 32 * h->cap_pairs + 8 * h->ncell + 3 * pb;
    return WTMD_OK;
}

static int ck_check_handle(wtmd_t* h)
{
    if (!h->pos || !h->vel || !h->force) FAIL(h, WTMD_EINVAL, "bind positions, velocities and forces first");
    if (surrogate_k0(h)) FAIL(h, WTMD_EINVAL, "turn the surrogate off first (save its network with wtmd_mlp_params)");
    return WTMD_OK;
}

extern "C" int wtmd_checkpoint_size(wtmd_t* h, int64_t* bytes)
{
    if (!h || !bytes) return WTMD_EINVAL;
    int rc;
    if ((rc = ck_check_handle(h))) return rc;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    long long c = 0;
    WTMD_CUDA_TRY(h, cudaMemcpy(&c, h->count, sizeof(c), cudaMemcpyDeviceToHost));
    return ck_layout(h, c, bytes);
}

extern "C" int wtmd_checkpoint_save(wtmd_t* h, void* out, int64_t cap_bytes)
{
    if (!h) return WTMD_EINVAL;
    int rc;
    if ((rc = ck_check_handle(h))) return rc;
    if (!out) FAIL(h, WTMD_EINVAL, "null buffer");
    if (!h->forces_valid) {  // the forces at the bound positions are part of the state
        if ((rc = enqueue_forces(h))) return rc;
        h->forces_valid = true;
    }
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CkHeader hd{};
    hd.magic = kCkMagic;
    hd.version = 1;
    hd.prec = h->prec;
    hd.d = h->d;
    hd.W = h->W;
    hd.N = h->N;
    hd.cap = h->cap;
    hd.cap_pairs = h->cap_pairs;
    hd.ncell = h->ncell;
    long long c = 0, st = 0;
    WTMD_CUDA_TRY(h, cudaMemcpy(&c, h->count, sizeof(c), cudaMemcpyDeviceToHost));
    WTMD_CUDA_TRY(h, cudaMemcpy(&st, h->step, sizeof(st), cudaMemcpyDeviceToHost));
    WTMD_CUDA_TRY(h, cudaMemcpy(hd.ctr, h->ctr, sizeof(hd.ctr), cudaMemcpyDeviceToHost));
    hd.count = c;
    hd.step = st;
    ck_layout(h, c, &hd.total);
    if (cap_bytes < hd.total) FAIL(h, WTMD_EINVAL, "buffer smaller than wtmd_checkpoint_size");
    char* p = (char*)out;
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    if (c) WTMD_CUDA_TRY(h, cudaMemcpy(p, h->hills64, 32 * (size_t)c, cudaMemcpyDeviceToHost));
    p += 32 * c;
    WTMD_CUDA_TRY(h, cudaMemcpy(p, h->hills32, 32 * (size_t)h->cap_pairs, cudaMemcpyDeviceToHost));
    p += 32 * h->cap_pairs;
    if (h->ncell) WTMD_CUDA_TRY(h, cudaMemcpy(p, h->grid, 8 * (size_t)h->ncell, cudaMemcpyDeviceToHost));
    p += 8 * h->ncell;
    const size_t pb = r4sz(h) * (size_t)h->N;
    for (void* a : {h->pos, h->vel, h->force}) {
        WTMD_CUDA_TRY(h, cudaMemcpy(p, a, pb, cudaMemcpyDeviceToHost));
        p += pb;
    }
    return WTMD_OK;
}

extern "C" int wtmd_checkpoint_load(wtmd_t* h, const void* in, int64_t n_bytes)
{
    if (!h) return WTMD_EINVAL;
    int rc;
    if ((rc = ck_check_handle(h))) return rc;
    if (!in || n_bytes < (int64_t)sizeof(CkHeader)) FAIL(h, WTMD_EINVAL, "buffer too small for a checkpoint");
    CkHeader hd;
    std::memcpy(&hd, in, sizeof(hd));
    if (hd.magic != kCkMagic || hd.version != 1) FAIL(h, WTMD_EINVAL, "not a checkpoint of this library");
    if (hd.prec != h->prec || hd.d != h->d || hd.W != h->W || hd.N != h->N || hd.cap != h->cap ||
        hd.cap_pairs != h->cap_pairs || hd.ncell != h->ncell)
        FAIL(h, WTMD_EINVAL, "checkpoint of a handle with another precision, CV count, walkers, atoms, capacity "
                             "or grid");
    if (hd.count < 0 || hd.count > h->cap || hd.step < 0) FAIL(h, WTMD_EINVAL, "corrupt checkpoint counters");
    int64_t total = 0;
    ck_layout(h, hd.count, &total);
    if (hd.total != total || n_bytes < total) FAIL(h, WTMD_EINVAL, "truncated or corrupt checkpoint");
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const char* p = (const char*)in + sizeof(hd);
    if (hd.count) WTMD_CUDA_TRY(h, cudaMemcpy(h->hills64, p, 32 * (size_t)hd.count, cudaMemcpyHostToDevice));
    p += 32 * hd.count;
    WTMD_CUDA_TRY(h, cudaMemcpy(h->hills32, p, 32 * (size_t)h->cap_pairs, cudaMemcpyHostToDevice));
    p += 32 * h->cap_pairs;
    if (h->ncell) WTMD_CUDA_TRY(h, cudaMemcpy(h->grid, p, 8 * (size_t)h->ncell, cudaMemcpyHostToDevice));
    p += 8 * h->ncell;
    const size_t pb = r4sz(h) * (size_t)h->N;
    for (void* a : {h->pos, h->vel, h->force}) {
        WTMD_CUDA_TRY(h, cudaMemcpy(a, p, pb, cudaMemcpyHostToDevice));
        p += pb;
    }
    long long c = hd.count, st = hd.step;
    WTMD_CUDA_TRY(h, cudaMemcpy(h->count, &c, sizeof(c), cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemcpy(h->step, &st, sizeof(st), cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemcpy(h->ctr, hd.ctr, sizeof(hd.ctr), cudaMemcpyHostToDevice));
    // the restored forces belong to the restored positions; the neighbour
    // lists were built for other positions and are rebuilt by the next step
    // (from clean cell counts: a step that gave up may have left them)
    h->forces_valid = true;
    if ((rc = nl_reset(h)) || (rc = nl_request(h))) return rc;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return WTMD_OK;
}

extern "C" int wtmd_grid_read(wtmd_t* h, double* out, int64_t n_out)
{
    if (!h) return WTMD_EINVAL;
    if (!h->grid) FAIL(h, WTMD_EINVAL, "no grid configured");
    if (!out || n_out < h->ncell) FAIL(h, WTMD_EINVAL, "output smaller than the grid");
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpy(out, h->grid, sizeof(double) * h->ncell, cudaMemcpyDeviceToHost));
    return WTMD_OK;
}

// Holds the stream for a fixed time (bounded by its argument, at most 2 ms)
// so that the host can enqueue a whole profiled step behind it: the step's
// kernels then run back to back and the events between them measure device
// time, not host launch gaps.
// A short spin of `dither` SM cycles (< 4096) at the end moves the start of
// the profiled step by a varying fraction of the event timer's tick, so that
// per-kernel means over many steps are not biased by that granularity.
__global__ static void delay_kernel(long long ns, int dither)
{
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    } while ((long long)(t - t0) < ns && (long long)(t - t0) < 2000000);
    const long long c0 = clock64();
    while (clock64() - c0 < (dither & 4095)) {
    }
}

extern "C" int wtmd_profile_step(wtmd_t* h, int64_t n_steps, char* names, double* ms, int32_t cap, int32_t* n_out)
{
    if (!h) return WTMD_EINVAL;
    if (n_steps < 1 || cap < 1 || !names || !ms || !n_out) FAIL(h, WTMD_EINVAL, "bad profile arguments");
    int rc = ready(h);
    if (rc) return rc;
    if (!h->pos || !h->vel || !h->force) FAIL(h, WTMD_EINVAL, "bind positions, velocities and forces first");
    if ((rc = launch_hills_partial_prealloc(h, h->W))) return rc;
    if (!h->forces_valid) {
        if ((rc = enqueue_forces(h))) return rc;
        h->forces_valid = true;
    }
    std::vector<double> acc;
    std::vector<std::string> nm;
    h->prof = true;
    for (int64_t s = 0; s < n_steps; ++s) {
        h->ev_n = 0;
        delay_kernel<<<1, 32, 0, h->stream>>>(500000, (int)((uint32_t)(s * 2654435761u) >> 20));
        mark(h, "start");
        rc = enqueue_step(h);
        if (rc) break;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            rc = WTMD_ECUDA;
            break;
        }
        if (s == 0) {
            nm.assign(h->ev_names.begin() + 1, h->ev_names.begin() + h->ev_n);
            acc.assign(nm.size(), 0.0);
        }
        for (int i = 1; i < h->ev_n && i - 1 < (int)acc.size(); ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, h->ev_pool[i - 1], h->ev_pool[i]);
            acc[i - 1] += t;
        }
    }
    h->prof = false;
    if (rc) return rc;
    const int n = std::min<int>((int)nm.size(), cap);
    for (int i = 0; i < n; ++i) {
        std::strncpy(names + 32 * i, nm[i].c_str(), 31);
        names[32 * i + 31] = 0;
        ms[i] = acc[i] / n_steps;
    }
    *n_out = n;
    return WTMD_OK;
}

extern "C" int wtmd_wait_limit(wtmd_t* h, int64_t cycles)
{
    if (!h) return WTMD_EINVAL;
    if (cycles < 0 || cycles > kWaitLimit) FAIL(h, WTMD_EINVAL, "wait limit must be in [0, 2^31] SM cycles");
    if (h->wait_limit != cycles) drop_graphs(h);  // the limit is a launch argument
    h->wait_limit = cycles;
    return WTMD_OK;
}

extern "C" int wtmd_fused_step(wtmd_t* h, int32_t enable, int32_t* active)
{
    if (!h) return WTMD_EINVAL;
    if (enable == 0 || enable == 1) {
        if (h->fused_on != (enable == 1)) drop_graphs(h);
        h->fused_on = enable == 1;
    }
    if (active) *active = (h->fused_on && sys_step_eligible(h, nullptr)) ? 1 : 0;
    return WTMD_OK;
}

extern "C" int wtmd_small_step(wtmd_t* h, int32_t enable, int32_t* active)
{
    if (!h) return WTMD_EINVAL;
    if (enable == 0 || enable == 1) {
        if (h->small_on != (enable == 1)) drop_graphs(h);
        h->small_on = enable == 1;
    } else if (enable != -1) {
        FAIL(h, WTMD_EINVAL, "enable must be 0, 1 or -1 (query)");
    }
    if (active) *active = small_step_eligible(h) ? 1 : 0;
    return WTMD_OK;
}

extern "C" int wtmd_walkers_persistent(wtmd_t* h, int32_t enable)
{
    if (!h) return WTMD_EINVAL;
    drop_graphs(h);
    h->no_graph = false;
    if (!enable) {
        h->persistent = false;
        return WTMD_OK;
    }
    return walkers_enable(h);
}

// Times each tile candidate over `steps` eager steps from the same saved
// state (positions, velocities, forces, hill count, step, grid), keeps the
// fastest and restores the state: tuning does not advance the simulation.
extern "C" int wtmd_autotune(wtmd_t* h, int64_t steps, int32_t* choice)
{
    if (!h) return WTMD_EINVAL;
    if (!h->persistent) FAIL(h, WTMD_EINVAL, "autotuning applies to the persistent walker step");
    if (!h->pos || !h->vel || !h->force) FAIL(h, WTMD_EINVAL, "bind particle arrays first");
    if (steps < 1) FAIL(h, WTMD_EINVAL, "steps must be >= 1");
    int rc;
    if (!h->forces_valid) {
        if ((rc = enqueue_forces(h))) return rc;
        h->forces_valid = true;
    }
    const size_t pb = sizeof(float4) * (size_t)h->N;
    void *sx = nullptr, *sv = nullptr, *sf = nullptr, *sg = nullptr, *sh = nullptr;
    const size_t hb = sizeof(double) * (4 * (size_t)h->W + 1);  // umbrella window sums and count
    long long counters[2];
    double centre[3];
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    WTMD_CUDA_TRY(h, cudaMalloc(&sx, pb));
    WTMD_CUDA_TRY(h, cudaMalloc(&sv, pb));
    WTMD_CUDA_TRY(h, cudaMalloc(&sf, pb));
    if (h->grid) WTMD_CUDA_TRY(h, cudaMalloc(&sg, sizeof(double) * h->ncell));
    if (h->harm_sum) WTMD_CUDA_TRY(h, cudaMalloc(&sh, hb));
    auto save = [&]() {
        if (sh) cudaMemcpy(sh, h->harm_sum, hb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(sx, h->pos, pb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(sv, h->vel, pb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(sf, h->force, pb, cudaMemcpyDeviceToDevice);
        if (sg) cudaMemcpy(sg, h->grid, sizeof(double) * h->ncell, cudaMemcpyDeviceToDevice);
        cudaMemcpy(&counters[0], h->count, sizeof(long long), cudaMemcpyDeviceToHost);
        cudaMemcpy(&counters[1], h->step, sizeof(long long), cudaMemcpyDeviceToHost);
        cudaMemcpy(centre, h->ctr, sizeof(centre), cudaMemcpyDeviceToHost);
    };
    auto restore = [&]() {
        cudaStreamSynchronize(h->stream);
        cudaMemcpy(h->pos, sx, pb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(h->vel, sv, pb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(h->force, sf, pb, cudaMemcpyDeviceToDevice);
        if (sg) cudaMemcpy(h->grid, sg, sizeof(double) * h->ncell, cudaMemcpyDeviceToDevice);
        if (sh) cudaMemcpy(h->harm_sum, sh, hb, cudaMemcpyDeviceToDevice);
        cudaMemcpy(h->count, &counters[0], sizeof(long long), cudaMemcpyHostToDevice);
        cudaMemcpy(h->step, &counters[1], sizeof(long long), cudaMemcpyHostToDevice);
        cudaMemcpy(h->ctr, centre, sizeof(centre), cudaMemcpyHostToDevice);
    };
    save();
    const int Ts[] = {32, 64, 128, 256}, Bs[] = {1, 2, 4}, Hs[] = {1, 2};
    float best = 1e30f;
    int bT = 128, bB = 2, bH = 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    rc = WTMD_OK;
    for (int T : Ts)
        for (int B : Bs)
            for (int Hm : Hs) {
                if ((rc = walkers_retile(h, T, B, Hm))) goto done;
                if ((rc = launch_walkers_step(h, 0))) goto done;  // warm-up
                cudaEventRecord(e0, h->stream);
                for (int64_t s = 0; s < steps && rc == WTMD_OK; ++s) rc = launch_walkers_step(h, 0);
                cudaEventRecord(e1, h->stream);
                cudaEventSynchronize(e1);
                if (rc) goto done;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best && h->wk.T == T && h->wk.bps == B) {
                    best = ms;
                    bT = T;
                    bB = B;
                    bH = Hm;
                }
                restore();
            }
done:
    restore();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc2 = walkers_retile(h, bT, bB, bH);
    // hills deposited during the trials lie beyond the restored count: put the
    // FP32 layout back to padding there
    pad_hills32_kernel<<<(unsigned)((h->cap_pairs + 255) / 256), 256, 0, h->stream>>>(h->hills32, h->cap_pairs);
    store_hills32_range(h, 0, counters[0]);
    cudaStreamSynchronize(h->stream);
    cudaFree(sx);
    cudaFree(sv);
    cudaFree(sf);
    cudaFree(sg);
    cudaFree(sh);
    unsigned st = 0;
    cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost);
    st &= ~ST_CAPACITY;  // trial deposits may have hit capacity
    cudaMemcpy(h->status, &st, sizeof(st), cudaMemcpyHostToDevice);
    drop_graphs(h);
    h->no_graph = false;
    if (choice) {
        choice[0] = bT;
        choice[1] = h->wk.bps;
        choice[2] = bH;
    }
    if (rc) return rc;
    return rc2;
}
