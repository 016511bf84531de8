// Analytic test landscapes of the engine (forces of one particle), shared by
// the per-kernel engine (engine.cu) and the single-CTA small-system step
// (small_step.cu).  Each translation unit that includes this header holds
// its own copy of the constant tables.
#pragma once

#include "wtmd_internal.cuh"

namespace wtmd {

// Mueller-Brown (Mueller & Brown 1979): sum of four anisotropic Gaussians,
// U = sum_k A_k exp(a_k dx^2 + b_k dx dy + c_k dy^2), dx = x - x0_k,
// dy = y - y0_k; F = -grad U in the (x, y) plane.
static __constant__ double kMB[6][4] = {
    {-200.0, -100.0, -170.0, 15.0},  // A
    {-1.0, -1.0, -6.5, 0.7},         // a
    {0.0, 0.0, 11.0, 0.6},           // b
    {-10.0, -10.0, -6.5, 0.7},       // c
    {1.0, 0.0, -0.5, -1.0},          // x0
    {0.0, 0.5, 1.5, 1.0},            // y0
};

// Three Gaussian wells in a harmonic confinement (3-D test landscape):
// U = -sum_m A_m exp(-|r - c_m|^2 / (2 s_m^2)) + (k/2) |r|^2, F = -grad U.
static __constant__ double kW3[3][5] = {
    // A, s, c_x, c_y, c_z
    {8.0, 0.45, -1.0, 0.0, 0.0},
    {6.0, 0.40, 1.0, 0.2, -0.3},
    {7.0, 0.50, 0.1, 1.3, 0.6},
};
constexpr double kW3Conf = 1.5;

template <typename R> __device__ __forceinline__ R4<R> mb_force(const R4<R>& p)
{
    R gx = 0, gy = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R dx = p.x - (R)kMB[4][k], dy = p.y - (R)kMB[5][k];
        const R a = (R)kMB[1][k], b = (R)kMB[2][k], c = (R)kMB[3][k];
        const R e = (R)kMB[0][k] * exp(a * dx * dx + b * dx * dy + c * dy * dy);
        gx += e * (R(2) * a * dx + b * dy);
        gy += e * (b * dx + R(2) * c * dy);
    }
    return mk4<R>(-gx, -gy, R(0), R(0));
}

template <typename R> __device__ __forceinline__ R4<R> wells3_force(const R4<R>& p)
{
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
    return mk4<R>(fx, fy, fz, R(0));
}

}  // namespace wtmd
