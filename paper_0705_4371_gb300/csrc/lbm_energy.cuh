// lbm_energy.cuh -- entropic quasiequilibrium with the energy constraint
// (D2Q9): the maximiser of the perfect entropy S = -sum f ln(f/W) ((PerfEnt))
// subject to m(f) = M = (rho, rho u1, rho u2, 2E) ((argmax)).  Its Lagrange
// form (Sec. 3.3) is ln(f*_i / W_i) = mu0 + a . m'_i with m' = (v_x, v_y,
// |v|^2); the density multiplier mu0 is fixed by the normalisation, so
//   f*_i = rho W_i e^{a . m'_i} / Z(a),   Z(a) = sum_i W_i e^{a . m'_i},
// and a solves E[m'] = t = (u_x, u_y, 2E / rho) under p_i = f*_i / rho.
// Newton: a <- a - C^{-1} (E[m'] - t), C the covariance of m' under p
// (symmetric positive definite: the dual is strictly convex, so the root is
// unique and the start point only changes the iteration count).
// Iterations run in FP32 until |E[m'] - t| <= 2e-6; then FP64 steps take
// the residual to <= 1e-12 (max-norm of m(f*) - M over rho).  The FP64
// exponentials are evaluated once, at the FP32 solution; later updates
// multiply them by e^{-delta} from its Taylor series, exact to rounding
// for the tiny FP64 steps.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kNewton32Max = 16;
constexpr int kNewton64Max = 6;
constexpr float kNewton32Tol = 2e-6f;
constexpr double kNewtonTol = 1e-12;

struct NewtonCount {
    unsigned it32, it64, sites, fails;
};

// Unnormalised weights q_i = W_i bx^{v_x} by^{v_y} bc^{|v|^2} from
// b = e^{a} and its reciprocals.
template <typename U>
__device__ __forceinline__ void energy_q(U bx, U by, U bc, U ibx, U iby, U* q) {
    const U bc2 = bc * bc;
    const U w0 = U(4.0 / 9.0), w1 = U(1.0 / 9.0), w5 = U(1.0 / 36.0);
    q[0] = w0;
    q[1] = w1 * bx * bc;
    q[2] = w1 * by * bc;
    q[3] = w1 * ibx * bc;
    q[4] = w1 * iby * bc;
    q[5] = w5 * (bx * by) * bc2;
    q[6] = w5 * (ibx * by) * bc2;
    q[7] = w5 * (ibx * iby) * bc2;
    q[8] = w5 * (bx * iby) * bc2;
}

// From q: Z, the residual g = E[m'] - t and the covariance C (upper
// triangle c00 c01 c02 c11 c12 c22).  Returns max |g|.
template <typename U>
__device__ __forceinline__ U energy_terms(const U* q, const U* tgt, U& Z, U* g, U* C) {
    const U qa = q[1] + q[2] + q[3] + q[4];          // |v|^2 = 1
    const U qd = q[5] + q[6] + q[7] + q[8];          // |v|^2 = 2
    Z = q[0] + qa + qd;
    const U iz = U(1) / Z;
    const U sx = (q[1] - q[3]) + (q[5] - q[6] - q[7] + q[8]);
    const U sy = (q[2] - q[4]) + (q[5] + q[6] - q[7] - q[8]);
    const U sc = qa + U(2) * qd;
    const U sxx = q[1] + q[3] + qd;
    const U syy = q[2] + q[4] + qd;
    const U sxy = q[5] - q[6] + q[7] - q[8];
    const U sxc = (q[1] - q[3]) + U(2) * (q[5] - q[6] - q[7] + q[8]);
    const U syc = (q[2] - q[4]) + U(2) * (q[5] + q[6] - q[7] - q[8]);
    const U scc = qa + U(4) * qd;
    const U ex = sx * iz, ey = sy * iz, ec = sc * iz;
    g[0] = ex - tgt[0];
    g[1] = ey - tgt[1];
    g[2] = ec - tgt[2];
    C[0] = sxx * iz - ex * ex;
    C[1] = sxy * iz - ex * ey;
    C[2] = sxc * iz - ex * ec;
    C[3] = syy * iz - ey * ey;
    C[4] = syc * iz - ey * ec;
    C[5] = scc * iz - ec * ec;
    return fmax(fmax(fabs(g[0]), fabs(g[1])), fabs(g[2]));
}

// Solve C d = g (3 x 3, symmetric positive definite) by Cholesky
// factorisation.  Returns false if C is not positive definite.
template <typename U>
__device__ __forceinline__ bool spd3_solve(const U* C, const U* g, U* d) {
    const U l00 = sqrt(C[0]);
    if (!(l00 > U(0))) return false;
    const U l10 = C[1] / l00, l20 = C[2] / l00;
    const U s11 = C[3] - l10 * l10;
    if (!(s11 > U(0))) return false;
    const U l11 = sqrt(s11);
    const U l21 = (C[4] - l20 * l10) / l11;
    const U s22 = C[5] - l20 * l20 - l21 * l21;
    if (!(s22 > U(0))) return false;
    const U l22 = sqrt(s22);
    const U y0 = g[0] / l00;
    const U y1 = (g[1] - l10 * y0) / l11;
    const U y2 = (g[2] - l20 * y0 - l21 * y1) / l22;
    d[2] = y2 / l22;
    d[1] = (y1 - l21 * d[2]) / l11;
    d[0] = (y0 - l10 * d[1] - l20 * d[2]) / l00;
    return true;
}

// e^{-d} for |d| < 2^-10 from its Taylor series to d^4 (relative error
// below 1e-16 there).
__device__ __forceinline__ double exp_small_neg(double d) {
    return fma(fma(fma(fma(d, 1.0 / 24.0, -1.0 / 6.0), d, 0.5), d, -1.0), d, 1.0);
}

// Energy-constrained quasiequilibrium f*_i (FP64) of one site.  a: start
// point in, solution out.  FP64 steps continue until the residual is at or
// below stop_tol (1e-12, or closer to the rounding floor for FP64 storage).
// Returns false if the residual did not reach 1e-12 (the site then keeps
// the last iterate).
__device__ __forceinline__ bool energy_solve(double rho, double ux, double uy, double e2,
                                             float* a, double* fstar, NewtonCount& nc,
                                             double stop_tol) {
    const double th = e2 / rho;
    // FP32 phase
    const float tf[3] = {(float)ux, (float)uy, (float)th};
    int it = 0;
    for (; it < kNewton32Max; it++) {
        float q[9], Z, g[3], C[6], d[3];
        const float bx = expf(a[0]), by = expf(a[1]), bc = expf(a[2]);
        energy_q<float>(bx, by, bc, 1.0f / bx, 1.0f / by, q);
        const float r = energy_terms<float>(q, tf, Z, g, C);
        if (r <= kNewton32Tol) break;
        if (!spd3_solve<float>(C, g, d)) break;
        // damp very long steps (far start points)
        const float dm = fmaxf(fmaxf(fabsf(d[0]), fabsf(d[1])), fabsf(d[2]));
        const float sc = dm > 0.5f ? 0.5f / dm : 1.0f;
        a[0] -= sc * d[0];
        a[1] -= sc * d[1];
        a[2] -= sc * d[2];
    }
    nc.it32 += (unsigned)it;
    // FP64 phase
    const double tg[3] = {ux, uy, th};
    double ad[3] = {(double)a[0], (double)a[1], (double)a[2]};
    double b[3] = {exp(ad[0]), exp(ad[1]), exp(ad[2])};
    double ib[2] = {1.0 / b[0], 1.0 / b[1]};
    double q[9], Z = 1.0;
    bool ok = false;
    int it64 = 0;
    for (; it64 <= kNewton64Max; it64++) {
        double g[3], C[6], d[3];
        energy_q<double>(b[0], b[1], b[2], ib[0], ib[1], q);
        const double r = energy_terms<double>(q, tg, Z, g, C);
        ok = r <= kNewtonTol;
        if (r <= stop_tol) break;
        if (it64 == kNewton64Max || !spd3_solve<double>(C, g, d)) break;
        const double dm = fmax(fmax(fabs(d[0]), fabs(d[1])), fabs(d[2]));
        for (int j = 0; j < 3; j++) ad[j] -= d[j];
        if (dm < 0x1p-10) {
            for (int j = 0; j < 3; j++) b[j] *= exp_small_neg(d[j]);
            ib[0] *= exp_small_neg(-d[0]);
            ib[1] *= exp_small_neg(-d[1]);
        } else {
            for (int j = 0; j < 3; j++) b[j] = exp(ad[j]);
            ib[0] = 1.0 / b[0];
            ib[1] = 1.0 / b[1];
        }
    }
    nc.it64 += (unsigned)it64;
    nc.sites += 1u;
    if (!ok) nc.fails += 1u;
    a[0] = (float)ad[0];
    a[1] = (float)ad[1];
    a[2] = (float)ad[2];
    const double s = rho / Z;
#pragma unroll
    for (int i = 0; i < 9; i++) fstar[i] = s * q[i];
    return ok;
}

}  // namespace lbm
