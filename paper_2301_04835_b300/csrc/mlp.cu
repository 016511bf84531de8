// MLP surrogate of the hills sum.
//
// Once the hill list is long, the bias V(xi) = sum_k w_k exp(...) costs one
// exponential per hill per step.  The paper represents biases by neural
// networks in its ANN (Sec. 2.1.7) and FUNN (Sec. 2.1.8) methods; here a small network
// stands in for the older part of the hill list:
//     V(xi) = V_nn(xi) + sum_{k >= K} w_k exp(...),
// where V_nn approximates the sum over hills [0, K) and the exact sum covers
// the hills deposited since (K is a multiple of 256 so that the FP32 hill
// layout's range starts on a chunk boundary).  The network is
//     z1 = W1 x + b1, a1 = silu(z1), z2 = W2 a1 + b2, a2 = silu(z2),
//     y = w3 . a2 + b3,   silu(z) = z sigmoid(z),
// 3 -> 64 -> 64 -> 1 (4481 parameters), with x = (xi - mu) inv_s and
// V_nn = Vs y + Vm.  Weights are used in bfloat16 (an FP32 master copy is
// trained); activations and sums are FP32.
//
// Kernels (all hand-written, one warp per point or sample; lane l owns the
// hidden units l and l + 32 of both layers):
//   mlp_eval_kernel   V_nn and dV_nn/dxi at P points (inference; the step
//                     path adds them to the exact tail sum);
//   mlp_grad_kernel   Sobolev loss sum_b (y - V)^2 + lam |grad_x y - G|^2 and
//                     its weight gradient: forward, input gradient and the
//                     double backward through it per warp; W2's gradient (a
//                     sum of outer products) accumulated block-wide, 16
//                     entries per thread, the rest per lane and reduced per
//                     block in a fixed order;
//   mlp_adam_kernel   fixed-order sum of the block partials and the Adam
//                     update (Kingma & Ba 2015) of the FP32 master, which is
//                     re-rounded to bfloat16 (nearest, ties to even).
// Training data come from the run: jittered copies of the most recent hill
// centres, labelled by the exact hills sum over [0, K).  A tenth of them is
// held out; the surrogate is used only while its held-out RMS error (after
// removing the mean offset) is at most the tolerance, else the exact sum
// over all hills is used.
//
// The layer-2 products have 64-long reductions per output and FP32 inputs:
// the tensor-core MMA needs both operands in one 16-bit type, and bfloat16
// activations would put errors of order 1e-2 kT into V.  The work is a few
// microseconds per step, so the FP32 pipe is used.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hills_dev.cuh"
#include "step_dev.cuh"

namespace wtmd {

constexpr int MH = 64;      // hidden width
constexpr int MP = 4481;    // parameters
constexpr int PSTRIDE = (MP + 1 + 3) / 4 * 4;  // floats per block partial (gradient + loss), 16-byte rows
constexpr int O_W1 = 0, O_B1 = 192, O_W2 = 256, O_B2 = 4352, O_W3 = 4416, O_B3 = 4480;
constexpr int W2P = 68;     // shared row pitch of W2: 16-byte rows, conflict-free quad loads
constexpr int MLP_T = 256;  // threads per block of the training kernel
constexpr int MLP_W = MLP_T / 32;
constexpr int EV_T = 256;   // threads per block of the inference kernel (one network staging per 8 warps)
constexpr int EV_W = EV_T / 32;
// block-reduction slots of the parameters other than W2 (+ the loss)
constexpr int RB_B2 = O_W2, RB_W3 = RB_B2 + MH, RB_B3 = RB_W3 + MH, RB_LOSS = RB_B3 + 1, RED_N = RB_LOSS + 1;

struct MlpW;

struct Surrogate {
    float* master = nullptr;        // [MP] FP32 master weights
    unsigned short* wb = nullptr;   // [MP] bfloat16 bits of the weights
    MlpW* img = nullptr;            // the same weights as the kernels' FP32 image
    float* m = nullptr;             // Adam moments [MP]
    float* v = nullptr;
    double* norm = nullptr;         // device [8]: mu[3], inv_s[3], Vm, Vs
    long long* k0 = nullptr;        // device: first hill of the exact tail (0 while inactive)
    long long* kend = nullptr;      // device: end of the fitted hill range
    int* active = nullptr;          // device flag read by the step path
    float* dom = nullptr;           // device [6]: box of the training inputs (normalised), lo[3] then hi[3]
    long long* ctr = nullptr;       // device [2]: (unused), batch iteration of the training launches
    long long adam_t = 0;           // Adam steps taken (host copy; bias corrections)
    float* partial = nullptr;       // [pblocks][PSTRIDE]
    int pblocks = 0;
    float* loss = nullptr;          // device: loss of the last training step
    float* grad = nullptr;          // device [MP + 1] scratch of wtmd_mlp_grad
    double* sx = nullptr;           // training set [S][3] CV points
    float* sV = nullptr;            // [S]
    float* sG = nullptr;            // [S][3]
    float* hV = nullptr;            // held-out predictions [S/10]
    float* hG = nullptr;            // [S/10][3]
    int64_t S = 0;
    double norm_h[8] = {0, 0, 0, 1, 1, 1, 0, 1};
    bool have_norm = false;
    bool enabled = false;
    double tol = 0.05;
    int64_t every = 10000;
    int64_t next_fit = 0;
    int64_t fit_samples = 65540, fit_iters = 80000, batch = 4096;
    double lr = 6e-3, lam = 0.1;
    double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long host_step = 0, host_count = 0;
    uint64_t seed = 0x5eedULL;
    long long round = 0;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_bits_to_f(unsigned short b) { return __uint_as_float((unsigned)b << 16); }

// FP32 -> bfloat16, round to nearest, ties to even (finite inputs)
__device__ __forceinline__ unsigned short f_to_bf16_bits(float x)
{
    unsigned u = __float_as_uint(x);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (unsigned short)(u >> 16);
}

__device__ __forceinline__ float sigm(float z) { return rcp_approx(1.f + ex2_approx(-1.4426950408889634f * z)); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// The network as the kernels read it: FP32 values of the bfloat16 weights
// in a padded layout.  A copy of this image lives in global memory (kept in
// step with the weights) so that a block stages it with plain 16-byte loads.
struct MlpW {
    float W2[MH][W2P];
    float W1[MH][4];  // column 3 is 0
    float b1[MH], b2[MH], w3[MH];
    float b3;
    float pad[3];
};
static_assert(sizeof(MlpW) % 16 == 0, "image copied in 16-byte pieces");

// Parameter q (flat order W1, b1, W2, b2, w3, b3) -> its slot in the image.
__device__ __forceinline__ float* img_slot(MlpW* s, int q)
{
    if (q < O_B1) return &s->W1[q / 3][q % 3];
    if (q < O_W2) return &s->b1[q - O_B1];
    if (q < O_B2) return &s->W2[(q - O_W2) / MH][(q - O_W2) % MH];
    if (q < O_W3) return &s->b2[q - O_B2];
    if (q < O_B3) return &s->w3[q - O_W3];
    return &s->b3;
}

__device__ void mlp_stage(const MlpW* __restrict__ img, MlpW& s)
{
    const float4* src = reinterpret_cast<const float4*>(img);
    float4* dst = reinterpret_cast<float4*>(&s);
    for (int q = threadIdx.x; q < (int)(sizeof(MlpW) / 16); q += blockDim.x) dst[q] = src[q];
}

struct Fwd {
    float z1[2], d1[2], z2[2], a2[2], d2[2], g2[2], h1[2];
    float y, u[3];
};

// Forward pass and input gradient of one point by one warp.  A1 and G2 are
// the warp's shared vectors of 64.
__device__ __forceinline__ void warp_forward(const MlpW& s, const float x[3], float* A1, float* G2, Fwd& f)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int j = lane + 32 * r;
        const float z = fmaf(s.W1[j][0], x[0], fmaf(s.W1[j][1], x[1], fmaf(s.W1[j][2], x[2], s.b1[j])));
        const float sg = sigm(z);
        f.z1[r] = z;
        f.d1[r] = sg * fmaf(z, 1.f - sg, 1.f);
        A1[j] = z * sg;
    }
    __syncwarp();
    float ys = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = lane + 32 * r;
        const float4* wr = reinterpret_cast<const float4*>(&s.W2[i][0]);
        const float4* av = reinterpret_cast<const float4*>(A1);
        // four partial sums (by column mod 4): four short dependency chains
        float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll 8
        for (int q = 0; q < MH / 4; ++q) {
            const float4 w = wr[q], a = av[q];
            z0 = fmaf(w.x, a.x, z0);
            z1 = fmaf(w.y, a.y, z1);
            z2 = fmaf(w.z, a.z, z2);
            z3 = fmaf(w.w, a.w, z3);
        }
        const float z = s.b2[i] + ((z0 + z1) + (z2 + z3));
        const float sg = sigm(z);
        f.z2[r] = z;
        f.a2[r] = z * sg;
        f.d2[r] = sg * fmaf(z, 1.f - sg, 1.f);
        f.g2[r] = f.d2[r] * s.w3[i];
        G2[i] = f.g2[r];
        ys = fmaf(s.w3[i], f.a2[r], ys);
    }
    __syncwarp();
    f.y = warp_sum(ys) + s.b3;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int j = lane + 32 * r;
        float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
#pragma unroll 8
        for (int i = 0; i < MH; i += 4) {
            h0 = fmaf(s.W2[i][j], G2[i], h0);
            h1 = fmaf(s.W2[i + 1][j], G2[i + 1], h1);
            h2 = fmaf(s.W2[i + 2][j], G2[i + 2], h2);
            h3 = fmaf(s.W2[i + 3][j], G2[i + 3], h3);
        }
        const float hs = (h0 + h1) + (h2 + h3);
        f.h1[r] = hs;
        const float g1 = f.d1[r] * hs;
        u0 = fmaf(s.W1[j][0], g1, u0);
        u1 = fmaf(s.W1[j][1], g1, u1);
        u2 = fmaf(s.W1[j][2], g1, u2);
    }
    f.u[0] = warp_sum(u0);
    f.u[1] = warp_sum(u1);
    f.u[2] = warp_sum(u2);
}

// silu''(z) = s (1 - s) (2 + z (1 - 2 s))
__device__ __forceinline__ float silu_dd(float z)
{
    const float sg = sigm(z);
    return sg * (1.f - sg) * fmaf(z, 1.f - 2.f * sg, 2.f);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// The exact sum over the fitted hills [0, K) for a point the network was not
// trained on (the step path's fallback): the FP32 hill layout, lanes over
// hill pairs, compensated sums, a fixed xor tree over the warp.
struct HeadSum {
    const float* dom;         // the training box (normalised inputs); null: no guard
    const float4* hp;         // FP32 pair records
    const long long* kend;    // K
    const double* ctr;        // centre of the scaled layout
    HillPrmF32 prm;
    double gs[3];             // dV/dxi_i = gs_i * sum e D_i
    int* active;              // cleared on a domain exit
    long long* k0;            // set to 0 on a domain exit: the next steps sum every hill
};

__device__ __forceinline__ void head_sum_warp(const HeadSum& hs, const double* xip, int d, int lane, CF4& acc)
{
    float X[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < d; ++k) X[k] = (float)((xip[k] - hs.ctr[k]) * hs.prm.a[k]);
    const long long npairs = *hs.kend >> 1;  // K is a multiple of 256
    float2 v = make_float2(0.f, 0.f), g0 = v, g1 = v, g2 = v;
    for (long long q = lane; q < npairs; q += 32) {
        const float4 A = hs.hp[2 * q], B = hs.hp[2 * q + 1];
        float2 d0 = __fadd2_rn(make_float2(X[0], X[0]), make_float2(A.x, A.y));
        if (hs.prm.per[0] > 0.f) d0 = wrap2(d0, hs.prm.per[0], hs.prm.iper[0]);
        float2 t = __ffma2_rn(d0, d0, make_float2(B.z, B.w));
        float2 d1 = make_float2(0.f, 0.f), d2 = d1;
        if (d >= 2) {
            d1 = __fadd2_rn(make_float2(X[1], X[1]), make_float2(A.z, A.w));
            if (hs.prm.per[1] > 0.f) d1 = wrap2(d1, hs.prm.per[1], hs.prm.iper[1]);
            t = __ffma2_rn(d1, d1, t);
        }
        if (d >= 3) {
            d2 = __fadd2_rn(make_float2(X[2], X[2]), make_float2(B.x, B.y));
            if (hs.prm.per[2] > 0.f) d2 = wrap2(d2, hs.prm.per[2], hs.prm.iper[2]);
            t = __ffma2_rn(d2, d2, t);
        }
        const float2 e = make_float2(ex2_approx(-t.x), ex2_approx(-t.y));
        v = __fadd2_rn(v, e);
        g0 = __ffma2_rn(e, d0, g0);
        g1 = __ffma2_rn(e, d1, g1);
        g2 = __ffma2_rn(e, d2, g2);
    }
    acc.v[0] = cf_add(cf_add(cf{0.f, 0.f}, v.x), v.y);
    acc.v[1] = cf_add(cf_add(cf{0.f, 0.f}, g0.x), g0.y);
    acc.v[2] = cf_add(cf_add(cf{0.f, 0.f}, g1.x), g1.y);
    acc.v[3] = cf_add(cf_add(cf{0.f, 0.f}, g2.x), g2.y);
    cf4_lane_sum<32>(acc);
}

__global__ void __launch_bounds__(EV_T) mlp_eval_kernel(const MlpW* __restrict__ img,
                                                         const double* __restrict__ norm, const int* __restrict__ active,
                                                         const double* __restrict__ xi, int xs, int d, int P,
                                                         float* __restrict__ V, float* __restrict__ dV, int dvs,
                                                         int add, HeadSum hs)
{
    if (active && *active == 0) return;
    __shared__ __align__(16) MlpW s;
    __shared__ __align__(16) float A1[EV_W][MH];
    __shared__ __align__(16) float G2[EV_W][MH];
    mlp_stage(img, s);
    __syncthreads();
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    for (int p = blockIdx.x * EV_W + w; p < P; p += gridDim.x * EV_W) {
        float x[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k < d) x[k] = (float)((xi[(size_t)p * xs + k] - norm[k]) * norm[3 + k]);
        bool out = false;
        if (hs.dom)
            for (int k = 0; k < d; ++k) out = out || !(x[k] >= hs.dom[k] && x[k] <= hs.dom[3 + k]);
        if (out) {  // outside the inputs the network was trained on: the exact sum
            CF4 acc{};
            head_sum_warp(hs, xi + (size_t)p * xs, d, lane, acc);
            if (lane == 0) {
                V[p] += (float)cf_val(acc.v[0]);
                for (int k = 0; k < d; ++k) dV[(size_t)p * dvs + k] += (float)(hs.gs[k] * cf_val(acc.v[1 + k]));
                *hs.active = 0;
                *hs.k0 = 0;
            }
            __syncwarp();
            continue;
        }
        Fwd f;
        warp_forward(s, x, A1[w], G2[w], f);
        if (lane == 0) {
            const float Vn = (float)(norm[7] * (double)f.y + norm[6]);
            if (V) V[p] = add ? V[p] + Vn : Vn;
            if (dV) {
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (k < d) {
                        const float g = (float)(norm[7] * norm[3 + k]) * f.u[k];
                        dV[(size_t)p * dvs + k] = add ? dV[(size_t)p * dvs + k] + g : g;
                    }
            }
        }
        __syncwarp();
    }
}

struct TrainArgs {
    const MlpW* img;
    const double* norm;
    const double* x;        // samples [n][3] (CV units; unused dimensions 0)
    const float* V;         // [n]
    const float* G;         // [n][3]
    long long n;
    int B;                  // batch size
    const long long* iter;  // batch counter (null: batch = samples [0, B))
    long long perm;         // sample order: index (q * perm) mod n, perm coprime with n
    int d;
    float lam;
    float* partial;         // [gridDim.x][PSTRIDE]
};

static_assert(MH * MH % MLP_T == 0 && (MH * MH / MLP_T) % 4 == 0, "outer-product ownership");

__global__ void __launch_bounds__(MLP_T) mlp_grad_kernel(TrainArgs a)
{
    __shared__ __align__(16) MlpW s;
    __shared__ __align__(16) float A1[MLP_W][MH];
    __shared__ __align__(16) float G2[MLP_W][MH];
    __shared__ __align__(16) float HB[MLP_W][MH];
    __shared__ __align__(16) float Z2[MLP_W][MH];
    __shared__ int has[MLP_W];
    mlp_stage(a.img, s);
    __syncthreads();
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * MLP_W + w, nw = gridDim.x * MLP_W;
    const long long it = a.iter ? *a.iter : 0;
    float gsc[3];
    for (int k = 0; k < 3; ++k) gsc[k] = (float)(1.0 / (a.norm[7] * a.norm[3 + k]));
    const double Vm = a.norm[6], iVs = 1.0 / a.norm[7];
    const float invB = 1.f / (float)a.B;

    // W2's gradient sum_b (zb2 a1^T + g2 hb1^T) is accumulated by the whole
    // block: thread t owns OCOL consecutive entries of row t / (64 / OCOL)
    // and adds the outer products of the samples of all warps after each
    // round
    constexpr int OCOL = MH * MH / MLP_T;
    const int oi = threadIdx.x / (MH / OCOL), oj = (threadIdx.x % (MH / OCOL)) * OCOL;
    float acc2[OCOL];
#pragma unroll
    for (int k = 0; k < OCOL; ++k) acc2[k] = 0.f;
    float acc1[2][3], ab1[2], ab2[2], aw3[2];
    float ab3 = 0.f, aloss = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        acc1[r][0] = acc1[r][1] = acc1[r][2] = 0.f;
        ab1[r] = ab2[r] = aw3[r] = 0.f;
    }

    const int rounds = (a.B + nw - 1) / nw;
    for (int rd = 0; rd < rounds; ++rd) {
        const int sm = gw + rd * nw;
        if (lane == 0) has[w] = sm < a.B;
        if (sm < a.B) {
            const long long q = (it * a.B + sm) % a.n;
            const long long idx = (q * a.perm) % a.n;
            float x[3] = {0.f, 0.f, 0.f}, Gt[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k < a.d) {
                    x[k] = (float)((a.x[idx * 3 + k] - a.norm[k]) * a.norm[3 + k]);
                    Gt[k] = a.G[idx * 3 + k] * gsc[k];
                }
            const float Vt = (float)(((double)a.V[idx] - Vm) * iVs);
            Fwd f;
            warp_forward(s, x, A1[w], G2[w], f);
            const float r = f.y - Vt;
            float e[3], du[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                e[k] = f.u[k] - Gt[k];
                du[k] = 2.f * a.lam * e[k] * invB;
            }
            const float dy = 2.f * r * invB;
            if (lane == 0) aloss += r * r + a.lam * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            // upstream of g1 = silu'(z1) * h1 through u = W1^T g1
            float gb1[2];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int j = lane + 32 * rr;
                gb1[rr] = fmaf(s.W1[j][0], du[0], fmaf(s.W1[j][1], du[1], s.W1[j][2] * du[2]));
                HB[w][j] = gb1[rr] * f.d1[rr];  // upstream of h1
            }
            __syncwarp();
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int i = lane + 32 * rr;
                const float4* wr = reinterpret_cast<const float4*>(&s.W2[i][0]);
                const float4* hb = reinterpret_cast<const float4*>(HB[w]);
                float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;  // upstream of g2 = W2 hb1
#pragma unroll 8
                for (int qq = 0; qq < MH / 4; ++qq) {
                    const float4 ww = wr[qq], hh = hb[qq];
                    q0 = fmaf(ww.x, hh.x, q0);
                    q1 = fmaf(ww.y, hh.y, q1);
                    q2 = fmaf(ww.z, hh.z, q2);
                    q3 = fmaf(ww.w, hh.w, q3);
                }
                const float gb2 = (q0 + q1) + (q2 + q3);
                const float w3 = s.w3[i];
                const float zb2 = fmaf(dy * w3, f.d2[rr], gb2 * w3 * silu_dd(f.z2[rr]));
                aw3[rr] = fmaf(dy, f.a2[rr], fmaf(gb2, f.d2[rr], aw3[rr]));
                ab2[rr] += zb2;
                Z2[w][i] = zb2;
            }
            __syncwarp();
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int j = lane + 32 * rr;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;  // upstream of a1 = W2^T zb2
#pragma unroll 8
                for (int i = 0; i < MH; i += 4) {
                    c0 = fmaf(s.W2[i][j], Z2[w][i], c0);
                    c1 = fmaf(s.W2[i + 1][j], Z2[w][i + 1], c1);
                    c2 = fmaf(s.W2[i + 2][j], Z2[w][i + 2], c2);
                    c3 = fmaf(s.W2[i + 3][j], Z2[w][i + 3], c3);
                }
                const float ab = (c0 + c1) + (c2 + c3);
                const float zb1 = fmaf(ab, f.d1[rr], gb1[rr] * f.h1[rr] * silu_dd(f.z1[rr]));
                const float g1 = f.d1[rr] * f.h1[rr];
#pragma unroll
                for (int k = 0; k < 3; ++k) acc1[rr][k] = fmaf(zb1, x[k], fmaf(g1, du[k], acc1[rr][k]));
                ab1[rr] += zb1;
            }
            if (lane == 0) ab3 += dy;
        }
        __syncthreads();  // every warp's a1, g2, hb1, zb2 of this round are in shared memory
        for (int ww = 0; ww < MLP_W; ++ww) {
            if (!has[ww]) continue;
            const float zi = Z2[ww][oi], gi = G2[ww][oi];
            const float4* av = reinterpret_cast<const float4*>(&A1[ww][oj]);
            const float4* hv = reinterpret_cast<const float4*>(&HB[ww][oj]);
#pragma unroll
            for (int qq = 0; qq < OCOL / 4; ++qq) {
                const float4 aa = av[qq], hh = hv[qq];
                acc2[4 * qq + 0] = fmaf(zi, aa.x, fmaf(gi, hh.x, acc2[4 * qq + 0]));
                acc2[4 * qq + 1] = fmaf(zi, aa.y, fmaf(gi, hh.y, acc2[4 * qq + 1]));
                acc2[4 * qq + 2] = fmaf(zi, aa.z, fmaf(gi, hh.z, acc2[4 * qq + 2]));
                acc2[4 * qq + 3] = fmaf(zi, aa.w, fmaf(gi, hh.w, acc2[4 * qq + 3]));
            }
        }
        __syncthreads();  // before the next round overwrites the vectors
    }

    // the other parameters: block sum in warp order
    __shared__ float red[RED_N];
    for (int q = threadIdx.x; q < RED_N; q += MLP_T) red[q] = 0.f;
    __syncthreads();
    for (int ww = 0; ww < MLP_W; ++ww) {
        if (w == ww) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int i = lane + 32 * rr;
                red[RB_B2 + i] += ab2[rr];
                red[RB_W3 + i] += aw3[rr];
                for (int k = 0; k < 3; ++k) red[i * 3 + k] += acc1[rr][k];  // W1 row i
                red[O_B1 + i] += ab1[rr];
            }
            if (lane == 0) {
                red[RB_B3] += ab3;
                red[RB_LOSS] += aloss;
            }
        }
        __syncthreads();
    }
    float* out = a.partial + (size_t)blockIdx.x * PSTRIDE;
    float4* o2 = reinterpret_cast<float4*>(out + O_W2 + oi * MH + oj);
#pragma unroll
    for (int qq = 0; qq < OCOL / 4; ++qq)
        o2[qq] = make_float4(acc2[4 * qq], acc2[4 * qq + 1], acc2[4 * qq + 2], acc2[4 * qq + 3]);
    for (int q = threadIdx.x; q < MP + 1; q += MLP_T) {
        if (q < O_W2) out[q] = red[q];
        else if (q >= O_B2 && q < O_W3) out[q] = red[RB_B2 + (q - O_B2)];
        else if (q >= O_W3 && q < O_B3) out[q] = red[RB_W3 + (q - O_W3)];
        else if (q == O_B3) out[q] = red[RB_B3];
        else if (q == MP) out[q] = red[RB_LOSS];
    }
}

// Block sums of the training partials: a block of AD_T threads covers AD_Q
// consecutive entries (the 4481 parameters, then the loss); warp w adds the
// partials b = w, w + 8, ... of its lane's entry (eight loads in flight),
// then the eight warp sums are added in warp order: a fixed order.
constexpr int AD_T = 256, AD_Q = 32;

__device__ __forceinline__ float block_partial_sum(const float* __restrict__ partial, int nblk, int q)
{
    __shared__ float ps[AD_T / 32][AD_Q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float g = 0.f;
    if (q <= MP)
        for (int b0 = warp; b0 < nblk; b0 += 64) {
            float t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int b = b0 + 8 * k;
                t[k] = b < nblk ? partial[(size_t)b * PSTRIDE + q] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) g += t[k];
        }
    ps[warp][lane] = g;
    __syncthreads();
    float tot = ps[0][lane];
    for (int w = 1; w < AD_T / 32; ++w) tot += ps[w][lane];
    return tot;  // valid in every warp
}

// Gradient and mean loss only.
__global__ void __launch_bounds__(AD_T) mlp_reduce_kernel(const float* __restrict__ partial, int nblk, float invB,
                                                          float* __restrict__ out)
{
    const int q = blockIdx.x * AD_Q + (threadIdx.x & 31);
    const float g = block_partial_sum(partial, nblk, q);
    if (threadIdx.x < 32 && q <= MP) out[q] = q == MP ? g * invB : g;
}

struct AdamPrm {
    float lr, b1, b2, eps, invB;
    float bc1, bc2;  // bias corrections 1 - b1^t, 1 - b2^t of this step
};

__global__ void __launch_bounds__(AD_T) mlp_adam_kernel(const float* __restrict__ partial, int nblk,
                                                        float* __restrict__ master, float* __restrict__ m,
                                                        float* __restrict__ v, unsigned short* __restrict__ wb,
                                                        MlpW* __restrict__ img, AdamPrm p, long long* __restrict__ ctr,
                                                        float* __restrict__ loss_out)
{
    const int q = blockIdx.x * AD_Q + (threadIdx.x & 31);
    const float g = block_partial_sum(partial, nblk, q);
    if (threadIdx.x < 32) {
        if (q < MP) {
            const float mm = fmaf(p.b1, m[q], (1.f - p.b1) * g);
            const float vv = fmaf(p.b2, v[q], (1.f - p.b2) * g * g);
            const float th = master[q] - p.lr * (mm / p.bc1) / (sqrtf(vv / p.bc2) + p.eps);
            master[q] = th;
            m[q] = mm;
            v[q] = vv;
            const unsigned short b = f_to_bf16_bits(th);
            wb[q] = b;
            *img_slot(img, q) = bf16_bits_to_f(b);
        } else if (q == MP && loss_out) {
            *loss_out = g * p.invB;
        }
    }
    // the next training launch reads the batch counter after this kernel
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[1] += 1;
}

__global__ void mlp_round_kernel(const float* __restrict__ master, unsigned short* __restrict__ wb,
                                 MlpW* __restrict__ img)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < MP) {
        const unsigned short b = f_to_bf16_bits(master[q]);
        wb[q] = b;
        *img_slot(img, q) = bf16_bits_to_f(b);
    }
}

// Training points: jittered copies of the most recent M hill centres of
// [0, K); every tenth sample goes to the held-out part at the end.
__global__ void mlp_samples_kernel(const dbl4* __restrict__ h64, long long K, long long M, long long S, double j0,
                                   double j1, double j2, int d, uint64_t seed, long long round, double* __restrict__ out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const long long k = K - M + s % M;
    const Normal3<double> n = noise3<double>(seed, round, (uint32_t)s);
    const dbl4 c = h64[k];
    const long long Str = S - S / 10;
    const long long dst = (s % 10 == 9) ? Str + s / 10 : s - s / 10;
    const double cc[3] = {c.x, c.y, c.z}, jj[3] = {j0, j1, j2};
    for (int i = 0; i < 3; ++i) out[dst * 3 + i] = i < d ? cc[i] + jj[i] * n.g[i] : 0.0;
}

__global__ void set_ll_kernel(long long* p, long long v) { *p = v; }
__global__ void set_int_kernel(int* p, int v) { *p = v; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grad_blocks()
{
    static int n = 0;
    if (!n) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = 2 * (sms > 0 ? sms : 148);
    }
    return n;
}

static uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void surrogate_free(Surrogate* s)
{
    if (!s) return;
    void* p[] = {s->master, s->wb, s->img, s->m, s->v, s->norm, s->k0, s->kend, s->active, s->dom, s->ctr,
                 s->partial, s->loss, s->grad, s->sx, s->sV, s->sG, s->hV, s->hG};
    for (void* q : p) cudaFree(q);
    delete s;
}

// Allocate the surrogate state with a seeded Glorot-uniform initialisation.
static int sur_get(wtmd_t* h, Surrogate** out)
{
    if (h->sur) {
        *out = h->sur;
        return WTMD_OK;
    }
    if (h->prec != WTMD_F32) {
        h->err = "the surrogate runs on FP32 handles";
        return WTMD_EINVAL;
    }
    Surrogate* s = new Surrogate();
    h->sur = s;
    WTMD_CUDA_TRY(h, cudaMalloc(&s->master, sizeof(float) * MP));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->wb, sizeof(unsigned short) * MP));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->img, sizeof(MlpW)));
    WTMD_CUDA_TRY(h, cudaMemset(s->img, 0, sizeof(MlpW)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->m, sizeof(float) * MP));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->v, sizeof(float) * MP));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->norm, sizeof(double) * 8));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->k0, sizeof(long long)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->kend, sizeof(long long)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->active, sizeof(int)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->dom, sizeof(float) * 6));
    {
        const float inf_box[6] = {-INFINITY, -INFINITY, -INFINITY, INFINITY, INFINITY, INFINITY};
        WTMD_CUDA_TRY(h, cudaMemcpy(s->dom, inf_box, sizeof(inf_box), cudaMemcpyHostToDevice));
    }
    WTMD_CUDA_TRY(h, cudaMalloc(&s->ctr, sizeof(long long) * 2));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->loss, sizeof(float)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s->grad, sizeof(float) * (MP + 1)));
    s->pblocks = grad_blocks();
    WTMD_CUDA_TRY(h, cudaMalloc(&s->partial, sizeof(float) * PSTRIDE * (size_t)s->pblocks));
    std::vector<float> w(MP, 0.f);
    uint64_t st = s->seed;
    auto uni = [&](float lim) { return (float)(((splitmix(st) >> 11) * 0x1.0p-53 * 2.0 - 1.0) * lim); };
    const float l1 = std::sqrt(6.f / (3 + MH)), l2 = std::sqrt(6.f / (MH + MH)), l3 = std::sqrt(6.f / (MH + 1));
    for (int q = O_W1; q < O_B1; ++q) w[q] = uni(l1);
    for (int q = O_W2; q < O_B2; ++q) w[q] = uni(l2);
    for (int q = O_W3; q < O_B3; ++q) w[q] = uni(l3);
    WTMD_CUDA_TRY(h, cudaMemcpy(s->master, w.data(), sizeof(float) * MP, cudaMemcpyHostToDevice));
    WTMD_CUDA_TRY(h, cudaMemset(s->m, 0, sizeof(float) * MP));
    WTMD_CUDA_TRY(h, cudaMemset(s->v, 0, sizeof(float) * MP));
    WTMD_CUDA_TRY(h, cudaMemset(s->ctr, 0, sizeof(long long) * 2));
    WTMD_CUDA_TRY(h, cudaMemset(s->k0, 0, sizeof(long long)));
    WTMD_CUDA_TRY(h, cudaMemset(s->active, 0, sizeof(int)));
    WTMD_CUDA_TRY(h, cudaMemcpy(s->norm, s->norm_h, sizeof(double) * 8, cudaMemcpyHostToDevice));
    mlp_round_kernel<<<(MP + 255) / 256, 256>>>(s->master, s->wb, s->img);
    WTMD_CUDA_TRY(h, cudaDeviceSynchronize());
    *out = s;
    return WTMD_OK;
}

const long long* surrogate_k0(const wtmd_t* h) { return h->sur && h->sur->enabled ? h->sur->k0 : nullptr; }

// With refits every `every` hills the exact tail never exceeds every + W
// hills (+ one deposit of slack); while the network is inactive k0 = 0 and
// the whole list is summed, which the plan must also cover, so the bound
// applies only once a fit made the network active.
long long surrogate_tail_bound(const wtmd_t* h)
{
    if (!h->sur || !h->sur->enabled || h->sur->every <= 0 || h->sur->stats[5] == 0.0) return 0;
    return h->sur->every + 2ll * h->W + 256;
}

// Step path: V += V_nn, dV += dV_nn at the walkers' CVs when the surrogate
// is active (the kernel returns at once otherwise).
int launch_mlp_add(wtmd_t* h)
{
    if (!h->sur || !h->sur->enabled) return WTMD_OK;
    Surrogate& s = *h->sur;
    const int nb = std::max(1, std::min((h->W + EV_W - 1) / EV_W, grad_blocks()));
    HeadSum hs{};
    hs.dom = s.dom;
    hs.hp = h->hills32;
    hs.kend = s.kend;
    hs.ctr = h->ctr;
    for (int i = 0; i < 3; ++i) {
        hs.prm.a[i] = h->a[i];
        const double pp = i < h->d ? h->cv[i].period * h->a[i] : 0.0;
        hs.prm.per[i] = (float)pp;
        hs.prm.iper[i] = pp > 0.0 ? (float)(1.0 / pp) : 0.f;
        hs.gs[i] = -2.0 * 0.69314718055994530942 * h->a[i];
    }
    hs.active = s.active;
    hs.k0 = s.k0;
    mlp_eval_kernel<<<nb, EV_T, 0, h->stream>>>(s.img, s.norm, s.active, h->xi, 4, h->d, h->W, (float*)h->V,
                                                 (float*)h->dV, 4, 1, hs);
    mark(h, "mlp_surrogate");
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

static int launch_train(wtmd_t* h, const double* x, const float* V, const float* G, long long n, int B,
                        const long long* iter, long long perm, double lam, bool adam, double lr, float* grad_out)
{
    Surrogate& s = *h->sur;
    TrainArgs a{s.img, s.norm, x, V, G, n, B, iter, perm, h->d, (float)lam, s.partial};
    const int nb = std::max(1, std::min(s.pblocks, (B + MLP_W - 1) / MLP_W));
    mlp_grad_kernel<<<nb, MLP_T, 0, h->stream>>>(a);
    mark(h, "mlp_grad");
    if (adam) {
        const long long t = ++s.adam_t;
        AdamPrm p{(float)lr, 0.9f, 0.999f, 1e-8f, 1.f / (float)B, (float)(1.0 - std::pow(0.9, (double)t)),
                  (float)(1.0 - std::pow(0.999, (double)t))};
        mlp_adam_kernel<<<(MP + 1 + AD_Q - 1) / AD_Q, AD_T, 0, h->stream>>>(s.partial, nb, s.master, s.m, s.v, s.wb,
                                                                            s.img, p, s.ctr, s.loss);
        mark(h, "mlp_adam");
    } else {
        mlp_reduce_kernel<<<(MP + 1 + AD_Q - 1) / AD_Q, AD_T, 0, h->stream>>>(s.partial, nb, 1.f / (float)B, grad_out);
    }
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

static long long coprime_step(long long n)
{
    long long a = (long long)(0.6180339887498949 * (double)n) | 1;
    auto gcd = [](long long x, long long y) {
        while (y) {
            const long long t = x % y;
            x = y;
            y = t;
        }
        return x;
    };
    while (a > 1 && gcd(a, n) != 1) a += 2;
    return a < 1 ? 1 : a;
}

static int sur_ensure_samples(wtmd_t* h, int64_t S)
{
    Surrogate& s = *h->sur;
    if (S <= s.S) return WTMD_OK;
    cudaFree(s.sx);
    cudaFree(s.sV);
    cudaFree(s.sG);
    cudaFree(s.hV);
    cudaFree(s.hG);
    s.sx = nullptr;
    s.sV = s.sG = s.hV = s.hG = nullptr;
    s.S = 0;
    WTMD_CUDA_TRY(h, cudaMalloc(&s.sx, sizeof(double) * 3 * S));
    WTMD_CUDA_TRY(h, cudaMalloc(&s.sV, sizeof(float) * S));
    WTMD_CUDA_TRY(h, cudaMalloc(&s.sG, sizeof(float) * 3 * S));
    WTMD_CUDA_TRY(h, cudaMalloc(&s.hV, sizeof(float) * (S / 10 + 1)));
    WTMD_CUDA_TRY(h, cudaMalloc(&s.hG, sizeof(float) * 3 * (S / 10 + 1)));
    s.S = S;
    return WTMD_OK;
}

// Fit the network to the hills [0, K), K = count rounded down to a multiple
// of 256, and switch the step path to network + exact tail if the held-out
// error is within the tolerance (else to the exact sum).  Synchronizes.
static int sur_fit(wtmd_t* h)
{
    Surrogate& s = *h->sur;
    int rc;
    long long count = 0;
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(&count, h->count, sizeof(count), cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const long long K = count / 256 * 256;
    s.stats[0] = (double)K;
    if (K < 512) {  // too few hills to be worth a network
        s.stats[5] = 0.0;
        set_int_kernel<<<1, 1, 0, h->stream>>>(s.active, 0);
        set_ll_kernel<<<1, 1, 0, h->stream>>>(s.k0, 0);
        s.next_fit = K + 512;
        return WTMD_OK;
    }
    const int64_t S = std::max<int64_t>(10 * ((s.fit_samples + 9) / 10), 20);
    if ((rc = sur_ensure_samples(h, S))) return rc;
    const long long M = std::min<long long>(K, S);
    set_ll_kernel<<<1, 1, 0, h->stream>>>(s.kend, K);
    mlp_samples_kernel<<<(unsigned)((S + 255) / 256), 256, 0, h->stream>>>(
        (const dbl4*)h->hills64, K, M, S, h->cfg.sigma[0], h->cfg.sigma[1], h->cfg.sigma[2], h->d, s.seed, s.round++,
        s.sx);
    WTMD_CUDA_TRY(h, cudaMemsetAsync(s.sG, 0, sizeof(float) * 3 * S, h->stream));
    if ((rc = launch_hills_range(h, s.sx, true, 3, S, s.sV, s.sG, 3, nullptr, s.kend, 0, false))) return rc;
    const int64_t Str = S - S / 10, Sho = S / 10;
    if (!s.have_norm) {
        // input and output scales from the first training set; kept fixed
        // afterwards so that later fits continue from the current weights
        std::vector<double> hx(3 * S);
        std::vector<float> hv(S);
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(hx.data(), s.sx, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, h->stream));
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(hv.data(), s.sV, sizeof(float) * S, cudaMemcpyDeviceToHost, h->stream));
        WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        double nm[8] = {0, 0, 0, 1, 1, 1, 0, 1};
        for (int k = 0; k < h->d; ++k) {
            double m1 = 0.0, m2 = 0.0;
            for (int64_t i = 0; i < S; ++i) m1 += hx[3 * i + k];
            m1 /= (double)S;
            for (int64_t i = 0; i < S; ++i) m2 += (hx[3 * i + k] - m1) * (hx[3 * i + k] - m1);
            const double sd = std::sqrt(m2 / (double)S);
            nm[k] = m1;
            nm[3 + k] = sd > 0.0 ? 1.0 / sd : 1.0;
        }
        double v1 = 0.0, v2 = 0.0;
        for (int64_t i = 0; i < S; ++i) v1 += hv[i];
        v1 /= (double)S;
        for (int64_t i = 0; i < S; ++i) v2 += (hv[i] - v1) * (hv[i] - v1);
        nm[6] = v1;
        nm[7] = v2 > 0.0 ? std::sqrt(v2 / (double)S) : 1.0;
        std::memcpy(s.norm_h, nm, sizeof(nm));
        WTMD_CUDA_TRY(h, cudaMemcpy(s.norm, nm, sizeof(nm), cudaMemcpyHostToDevice));
        s.have_norm = true;
    }
    {
        // the box of the training inputs in the network's units: the step
        // path uses the network only inside it
        std::vector<double> hx(3 * S);
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(hx.data(), s.sx, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, h->stream));
        WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        float box[6] = {-INFINITY, -INFINITY, -INFINITY, INFINITY, INFINITY, INFINITY};
        for (int k = 0; k < h->d; ++k) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t i = 0; i < S; ++i) {
                const double u = (hx[3 * i + k] - s.norm_h[k]) * s.norm_h[3 + k];
                lo = std::min(lo, u);
                hi = std::max(hi, u);
            }
            box[k] = (float)lo;
            box[3 + k] = (float)hi;
        }
        WTMD_CUDA_TRY(h, cudaMemcpyAsync(s.dom, box, sizeof(box), cudaMemcpyHostToDevice, h->stream));
    }
    // Adam over batches of the training part, in a fixed pseudo-random order
    const int B = (int)std::min<int64_t>(s.batch, Str);
    const long long perm = coprime_step(Str);
    WTMD_CUDA_TRY(h, cudaMemsetAsync(s.ctr + 1, 0, sizeof(long long), h->stream));
    for (int64_t it = 0; it < s.fit_iters; ++it) {
        // cosine decay from lr to lr/100 over the fit
        const double c = 0.5 * (1.0 + std::cos(3.141592653589793 * (double)it / (double)s.fit_iters));
        const double lr = s.lr * (0.01 + 0.99 * c);
        if ((rc = launch_train(h, s.sx, s.sV, s.sG, Str, B, s.ctr + 1, perm, s.lam, true, lr, nullptr))) return rc;
    }
    // held-out error
    const int nbe = (int)std::min<int64_t>((Sho + EV_W - 1) / EV_W, grad_blocks());
    mlp_eval_kernel<<<std::max(nbe, 1), EV_T, 0, h->stream>>>(s.img, s.norm, nullptr, s.sx + 3 * Str, 3, h->d,
                                                                (int)Sho, s.hV, s.hG, 3, 0, HeadSum{});
    WTMD_CUDA_TRY(h, cudaGetLastError());
    std::vector<float> pv(Sho), tv(Sho), pg(3 * Sho), tg(3 * Sho);
    float L = 0.f;
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(pv.data(), s.hV, sizeof(float) * Sho, cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(tv.data(), s.sV + Str, sizeof(float) * Sho, cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(pg.data(), s.hG, sizeof(float) * 3 * Sho, cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(tg.data(), s.sG + 3 * Str, sizeof(float) * 3 * Sho, cudaMemcpyDeviceToHost,
                                     h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(&L, s.loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    double off = 0.0;
    for (int64_t i = 0; i < Sho; ++i) off += (double)pv[i] - (double)tv[i];
    off /= (double)std::max<int64_t>(Sho, 1);
    double se = 0.0, mx = 0.0, ge = 0.0, gn = 0.0;
    for (int64_t i = 0; i < Sho; ++i) {
        const double e = (double)pv[i] - (double)tv[i] - off;
        se += e * e;
        mx = std::max(mx, std::fabs(e));
        for (int k = 0; k < h->d; ++k) {
            const double g = (double)pg[3 * i + k] - (double)tg[3 * i + k];
            ge += g * g;
            gn += (double)tg[3 * i + k] * (double)tg[3 * i + k];
        }
    }
    const double kT = h->cfg.kT;
    const double rms = std::sqrt(se / (double)std::max<int64_t>(Sho, 1)) / kT;
    const bool ok = std::isfinite(rms) && rms <= s.tol;
    s.stats[1] = rms;
    s.stats[2] = mx / kT;
    s.stats[3] = gn > 0.0 ? std::sqrt(ge / gn) : 0.0;
    s.stats[4] = L;
    if ((s.stats[5] != 0.0) != ok) drop_step_graphs(h);  // the tail plan depends on it
    s.stats[5] = ok ? 1.0 : 0.0;
    s.stats[6] += 1.0;
    s.stats[7] += (double)s.fit_iters;
    set_int_kernel<<<1, 1, 0, h->stream>>>(s.active, ok ? 1 : 0);
    set_ll_kernel<<<1, 1, 0, h->stream>>>(s.k0, ok ? K : 0);
    s.next_fit = K + std::max<int64_t>(s.every, 256);
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return WTMD_OK;
}

// Host mirrors of the step and hill counters, used to schedule refits
// without reading the device every step.
static int sur_sync_counters(wtmd_t* h)
{
    Surrogate& s = *h->sur;
    long long c[2];
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(&c[0], h->step, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaMemcpyAsync(&c[1], h->count, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    s.host_step = c[0];
    s.host_count = c[1];
    return WTMD_OK;
}

// Steps (>= 1) until the hill count reaches `target`, given the deposit
// schedule (after step t when (t + 1) % stride == 0, W hills each time).
static int64_t steps_until(const wtmd_t* h, long long target)
{
    const Surrogate& s = *h->sur;
    const long long st = h->cfg.stride;
    if (st <= 0 || target <= s.host_count) return 1;
    const long long q = (target - s.host_count + h->W - 1) / h->W;  // deposits needed
    const long long m0 = s.host_step / st + 1;                     // first deposit event index ahead
    return (int64_t)(st * (m0 + q - 1) - s.host_step);
}

static void advance_counters(wtmd_t* h, int64_t n)
{
    Surrogate& s = *h->sur;
    const long long st = h->cfg.stride;
    if (st > 0) {
        const long long ev = (s.host_step + n) / st - s.host_step / st;
        s.host_count = std::min<long long>(s.host_count + ev * h->W, h->cap);
    }
    s.host_step += n;
}

// Called by step_n: how many of the n steps to run before the next refit
// (refitting first when one is due).
int surrogate_segment(wtmd_t* h, int64_t n, int64_t* seg)
{
    *seg = n;
    if (!h->sur || !h->sur->enabled || h->sur->every <= 0) return WTMD_OK;
    Surrogate& s = *h->sur;
    if (s.host_count >= s.next_fit) {
        int rc = sur_fit(h);
        if (rc) return rc;
        if ((rc = sur_sync_counters(h))) return rc;
    }
    *seg = std::max<int64_t>(1, std::min<int64_t>(n, steps_until(h, s.next_fit)));
    return WTMD_OK;
}

void surrogate_advanced(wtmd_t* h, int64_t n)
{
    if (h->sur && h->sur->enabled) advance_counters(h, n);
}

// The hill list was replaced: the fitted range no longer applies.
int surrogate_invalidate(wtmd_t* h)
{
    if (!h->sur) return WTMD_OK;
    Surrogate& s = *h->sur;
    set_int_kernel<<<1, 1, 0, h->stream>>>(s.active, 0);
    set_ll_kernel<<<1, 1, 0, h->stream>>>(s.k0, 0);
    s.stats[5] = 0.0;
    if (!s.enabled) return WTMD_OK;
    int rc = sur_sync_counters(h);
    if (rc) return rc;
    s.next_fit = s.every > 0 ? s.host_count : (1ll << 62);
    return WTMD_OK;
}

}  // namespace wtmd

using namespace wtmd;

#define SFAIL(h, code, msg) \
    do {                    \
        (h)->err = (msg);   \
        return (code);      \
    } while (0)

extern "C" int wtmd_surrogate(wtmd_t* h, int32_t enable, double tol_kT, int64_t retrain_every)
{
    if (!h) return WTMD_EINVAL;
    if (!enable) {
        if (h->sur && h->sur->enabled) {
            h->sur->enabled = false;
            set_int_kernel<<<1, 1, 0, h->stream>>>(h->sur->active, 0);
            set_ll_kernel<<<1, 1, 0, h->stream>>>(h->sur->k0, 0);
            drop_step_graphs(h);
        }
        return WTMD_OK;
    }
    if (!(tol_kT > 0.0) || retrain_every < 0) SFAIL(h, WTMD_EINVAL, "tolerance must be > 0, retrain_every >= 0");
    if (h->persistent) SFAIL(h, WTMD_EINVAL, "the surrogate is not available with the persistent walker step");
    if (h->bias_grid || h->bias_harm) SFAIL(h, WTMD_EINVAL, "the surrogate replaces the hills sum; another bias source is on");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    s->tol = tol_kT;
    s->every = retrain_every;
    if (!s->enabled) {
        s->enabled = true;
        drop_step_graphs(h);
    }
    if ((rc = sur_sync_counters(h))) return rc;
    s->next_fit = s->host_count;  // fit at the next step_n (or now, by wtmd_surrogate_fit)
    return WTMD_OK;
}

extern "C" int wtmd_surrogate_config(wtmd_t* h, int64_t n_samples, int64_t iters, int64_t batch, double lr,
                                     double lambda)
{
    if (!h) return WTMD_EINVAL;
    if (n_samples < 20 || iters < 0 || batch < 1 || !(lr > 0.0) || !(lambda >= 0.0))
        SFAIL(h, WTMD_EINVAL, "bad surrogate training parameters");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    s->fit_samples = n_samples;
    s->fit_iters = iters;
    s->batch = batch;
    s->lr = lr;
    s->lam = lambda;
    return WTMD_OK;
}

extern "C" int wtmd_surrogate_fit(wtmd_t* h, double* stats)
{
    if (!h) return WTMD_EINVAL;
    if (h->ncv != h->d) SFAIL(h, WTMD_EINVAL, "define all n_cv CVs first");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    if ((rc = sur_fit(h))) return rc;
    if (s->enabled && (rc = sur_sync_counters(h))) return rc;
    if (stats) std::memcpy(stats, s->stats, sizeof(s->stats));
    return WTMD_OK;
}

extern "C" int wtmd_surrogate_status(wtmd_t* h, double* stats)
{
    if (!h || !stats) return WTMD_EINVAL;
    if (!h->sur) {
        for (int i = 0; i < 8; ++i) stats[i] = 0.0;
        return WTMD_OK;
    }
    Surrogate& s = *h->sur;
    if (s.active) {  // a walker leaving the fitted inputs switches the network off on the device
        int act = 0;
        WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        WTMD_CUDA_TRY(h, cudaMemcpy(&act, s.active, sizeof(int), cudaMemcpyDeviceToHost));
        if (s.stats[5] != 0.0 && act == 0) s.stats[5] = 0.0;
    }
    std::memcpy(stats, s.stats, sizeof(s.stats));
    return WTMD_OK;
}

extern "C" int wtmd_surrogate_set(wtmd_t* h, int64_t k0, int32_t active)
{
    if (!h) return WTMD_EINVAL;
    if (k0 < 0 || k0 % 256 || k0 > h->cap) SFAIL(h, WTMD_EINVAL, "k0 must be a multiple of 256 within capacity");
    if (h->persistent) SFAIL(h, WTMD_EINVAL, "the surrogate is not available with the persistent walker step");
    if (h->bias_grid || h->bias_harm) SFAIL(h, WTMD_EINVAL, "the surrogate replaces the hills sum; another bias source is on");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    if (!s->enabled) {
        s->enabled = true;
        drop_step_graphs(h);
    }
    s->every = 0;  // no refits: the caller owns the network
    set_int_kernel<<<1, 1, 0, h->stream>>>(s->active, active ? 1 : 0);
    set_ll_kernel<<<1, 1, 0, h->stream>>>(s->k0, active ? k0 : 0);
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

extern "C" int wtmd_mlp_params(wtmd_t* h, const float* in, float* out, const double* norm_in, double* norm_out)
{
    if (!h) return WTMD_EINVAL;
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    WTMD_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (in) {
        WTMD_CUDA_TRY(h, cudaMemcpy(s->master, in, sizeof(float) * MP, cudaMemcpyHostToDevice));
        WTMD_CUDA_TRY(h, cudaMemset(s->m, 0, sizeof(float) * MP));
        WTMD_CUDA_TRY(h, cudaMemset(s->v, 0, sizeof(float) * MP));
        WTMD_CUDA_TRY(h, cudaMemset(s->ctr, 0, sizeof(long long) * 2));
        s->adam_t = 0;
        mlp_round_kernel<<<(MP + 255) / 256, 256>>>(s->master, s->wb, s->img);
        WTMD_CUDA_TRY(h, cudaDeviceSynchronize());
    }
    if (norm_in) {
        if (!(norm_in[7] != 0.0) || !std::isfinite(norm_in[7])) SFAIL(h, WTMD_EINVAL, "Vs must be finite and nonzero");
        std::memcpy(s->norm_h, norm_in, sizeof(s->norm_h));
        s->have_norm = true;
        WTMD_CUDA_TRY(h, cudaMemcpy(s->norm, norm_in, sizeof(double) * 8, cudaMemcpyHostToDevice));
    }
    if (out) WTMD_CUDA_TRY(h, cudaMemcpy(out, s->master, sizeof(float) * MP, cudaMemcpyDeviceToHost));
    if (norm_out) std::memcpy(norm_out, s->norm_h, sizeof(s->norm_h));
    return WTMD_OK;
}

extern "C" int wtmd_mlp_eval(wtmd_t* h, const double* xi, int64_t P, float* V, float* dV)
{
    if (!h) return WTMD_EINVAL;
    if (P < 0 || P > (1 << 30) || (P > 0 && !xi)) SFAIL(h, WTMD_EINVAL, "bad points");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    if (P == 0) return WTMD_OK;
    // each block stages the network once: a few blocks per SM, points by grid stride
    const int nb = (int)std::min<int64_t>((P + EV_W - 1) / EV_W, grad_blocks());
    mlp_eval_kernel<<<nb, EV_T, 0, h->stream>>>(s->img, s->norm, nullptr, xi, h->d, h->d, (int)P, V, dV, h->d, 0,
                                                 HeadSum{});
    WTMD_CUDA_TRY(h, cudaGetLastError());
    return WTMD_OK;
}

extern "C" int wtmd_mlp_grad(wtmd_t* h, const double* xi, const float* V, const float* dV, int64_t B, double lambda,
                             float* grad_out)
{
    if (!h) return WTMD_EINVAL;
    if (B < 1 || B > (1 << 30) || !xi || !V || !dV || !grad_out || !(lambda >= 0.0))
        SFAIL(h, WTMD_EINVAL, "bad batch");
    if (h->d != 3 && h->d != 2 && h->d != 1) SFAIL(h, WTMD_EINVAL, "bad CV count");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    return launch_train(h, xi, V, dV, B, (int)B, nullptr, 1, lambda, false, 0.0, grad_out);
}

extern "C" int wtmd_mlp_train(wtmd_t* h, const double* xi, const float* V, const float* dV, int64_t n, int64_t B,
                              int64_t iters, double lr, double lambda, float* loss_out)
{
    if (!h) return WTMD_EINVAL;
    if (n < 1 || B < 1 || B > n || iters < 0 || !xi || !V || !dV || !(lr > 0.0) || !(lambda >= 0.0))
        SFAIL(h, WTMD_EINVAL, "bad training arguments");
    Surrogate* s = nullptr;
    int rc = sur_get(h, &s);
    if (rc) return rc;
    WTMD_CUDA_TRY(h, cudaMemsetAsync(s->ctr + 1, 0, sizeof(long long), h->stream));
    for (int64_t it = 0; it < iters; ++it)
        if ((rc = launch_train(h, xi, V, dV, n, (int)B, s->ctr + 1, 1, lambda, true, lr, nullptr))) return rc;
    if (loss_out) WTMD_CUDA_TRY(h, cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    return WTMD_OK;
}
