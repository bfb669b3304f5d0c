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
// The FP32 phase iterates until the residual |E[m'] - t| is at or below
// 2e-6 and no longer falls fourfold per step (FP32's noise floor, about
// 1e-7), or is below 3e-7.  The FP64 phase then takes Newton steps with the
// residual evaluated in FP64 and the covariance and the 3 x 3 solve in FP32
// (an approximate Jacobian keeps the convergence: its relative error of
// about 1e-7 adds 1e-7 x the residual per step), until the residual (max-norm
// of m(f*) - M over rho) is at or below 1e-12.  GB300's FP64 pipe is slow,
// so the FP64 phase avoids FP64 exponentials, divisions and square roots:
// it starts from the FP32 exponentials b = e^{a} (any positive b gives a
// member of the family above), takes reciprocals from FP32 seeds refined by
// Newton-Raphson, and updates b by the Taylor series of e^{-delta} for the
// tiny FP64 steps.
// FP32 and FP16 storage round f* to FP32 in the end, and their finishing
// steps (energy_solve_ff) run in float-float arithmetic instead of FP64:
// the same steps and the same 1e-12 stop, with about 48 significant bits
// from FP32 operations only.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kNewton32Max = 16;
constexpr int kNewton64Max = 6;
constexpr float kNewton32Tol = 2e-6f;
constexpr float kNewton32Floor = 3e-7f;
constexpr double kNewtonTol = 1e-12;

struct NewtonCount {
    unsigned it32, it64, sites, fails;
};

// 1 / x in FP64 from the FP32 reciprocal refined by two Newton-Raphson
// steps (each squares the relative error: 2^-23 -> 2^-46 -> below one FP64
// ulp).  x must lie in the normal FP32 range.
__device__ __forceinline__ double recip64(double x) {
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
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
    const U iz = recip<U>(Z);
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

// FP64 residual g = E[m'] - t from q; returns max |g| and Z, 1/Z.
__device__ __forceinline__ double energy_residual64(const double* q, const double* tgt, double& Z,
                                                    double& iz, double* g) {
    const double qa = q[1] + q[2] + q[3] + q[4];
    const double qd = q[5] + q[6] + q[7] + q[8];
    Z = q[0] + qa + qd;
    iz = recip64(Z);
    const double sx = (q[1] - q[3]) + (q[5] - q[6] - q[7] + q[8]);
    const double sy = (q[2] - q[4]) + (q[5] + q[6] - q[7] - q[8]);
    const double sc = qa + 2.0 * qd;
    g[0] = sx * iz - tgt[0];
    g[1] = sy * iz - tgt[1];
    g[2] = sc * iz - tgt[2];
    return fmax(fmax(fabs(g[0]), fabs(g[1])), fabs(g[2]));
}

// Solve C d = g (3 x 3, symmetric positive definite) by Cholesky
// factorisation in FP32 with reciprocal square roots (a Newton step needs
// no more).  Returns false if C is not positive definite.
__device__ __forceinline__ bool spd3_solve(const float* C, const float* g, float* d) {
    if (!(C[0] > 0.0f)) return false;
    const float i00 = rsqrtf(C[0]);
    const float l10 = C[1] * i00, l20 = C[2] * i00;
    const float s11 = C[3] - l10 * l10;
    if (!(s11 > 0.0f)) return false;
    const float i11 = rsqrtf(s11);
    const float l21 = (C[4] - l20 * l10) * i11;
    const float s22 = C[5] - l20 * l20 - l21 * l21;
    if (!(s22 > 0.0f)) return false;
    const float i22 = rsqrtf(s22);
    const float y0 = g[0] * i00;
    const float y1 = (g[1] - l10 * y0) * i11;
    const float y2 = (g[2] - l20 * y0 - l21 * y1) * i22;
    d[2] = y2 * i22;
    d[1] = (y1 - l21 * d[2]) * i11;
    d[0] = (y0 - l10 * d[1] - l20 * d[2]) * i00;
    return true;
}

// e^{-d} for |d| < 2^-10 from its Taylor series to d^4 (relative error
// below 1e-16 there).
__device__ __forceinline__ double exp_small_neg(double d) {
    return fma(fma(fma(fma(d, 1.0 / 24.0, -1.0 / 6.0), d, 0.5), d, -1.0), d, 1.0);
}

// Energy-constrained quasiequilibrium f*_i (FP64) of one site from rho,
// u and th = 2E / rho.  a: start point (FP32 multipliers) in, the FP32
// phase's solution out.  FP64 steps continue until the residual is at or
// below stop_tol (1e-12, or closer to the rounding floor for FP64 storage).
// Returns false if the residual did not reach 1e-12 (the site then keeps
// the last iterate).  a64 (optional): the solution's multipliers in FP64.
// The FP32 phase: Newton on a (FP32) towards the targets tf = (u_x, u_y,
// 2E / rho); returns the exponentials b = e^{a} of the last iterate.
__device__ __forceinline__ void energy_phase32(const float* tf, float* a, float& bx, float& by, float& bc,
                                               NewtonCount& nc) {
    float rprev = INFINITY;
    bx = 1.0f;
    by = 1.0f;
    bc = 1.0f;
    int it = 0;
    for (;; it++) {
        float q[9], Z, g[3], C[6], d[3];
        bx = expf(a[0]);
        by = expf(a[1]);
        bc = expf(a[2]);
        energy_q<float>(bx, by, bc, __frcp_rn(bx), __frcp_rn(by), q);
        const float r = energy_terms<float>(q, tf, Z, g, C);
        if (r <= kNewton32Tol && (r <= kNewton32Floor || r > 0.25f * rprev)) break;
        if (it == kNewton32Max || !spd3_solve(C, g, d)) break;
        // damp very long steps (far start points)
        const float dm = fmaxf(fmaxf(fabsf(d[0]), fabsf(d[1])), fabsf(d[2]));
        const float sc = dm > 0.5f ? 0.5f / dm : 1.0f;
        a[0] -= sc * d[0];
        a[1] -= sc * d[1];
        a[2] -= sc * d[2];
        rprev = r;
    }
    nc.it32 += (unsigned)it;
}

__device__ __forceinline__ bool energy_solve(double rho, double ux, double uy, double th, float* a,
                                             double* fstar, NewtonCount& nc, double stop_tol,
                                             double* a64 = nullptr) {
    const float tf[3] = {(float)ux, (float)uy, (float)th};
    float bx, by, bc;
    energy_phase32(tf, a, bx, by, bc, nc);
    // FP64 phase, from the exponentials of the FP32 phase's last iterate
    const double tg[3] = {ux, uy, th};
    double b[3] = {(double)bx, (double)by, (double)bc};
    double ib[2] = {recip64(b[0]), recip64(b[1])};
    double q[9], Z = 1.0, iz = 1.0;
    bool ok = false;
    int it64 = 0;
    for (;; it64++) {
        double g[3];
        energy_q<double>(b[0], b[1], b[2], ib[0], ib[1], q);
        const double r = energy_residual64(q, tg, Z, iz, g);
        ok = r <= kNewtonTol;
        if (r <= stop_tol || it64 == kNewton64Max) break;
        float qf[9], Cf[6], gf[3], df[3], Zf, unused[3];
        const float zero[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 9; i++) qf[i] = (float)q[i];
        energy_terms<float>(qf, zero, Zf, unused, Cf);
        gf[0] = (float)g[0];
        gf[1] = (float)g[1];
        gf[2] = (float)g[2];
        if (!spd3_solve(Cf, gf, df)) break;
        const float dm = fmaxf(fmaxf(fabsf(df[0]), fabsf(df[1])), fabsf(df[2]));
        if (dm < 0x1p-10f) {
            for (int j = 0; j < 3; j++) b[j] *= exp_small_neg((double)df[j]);
            ib[0] *= exp_small_neg(-(double)df[0]);
            ib[1] *= exp_small_neg(-(double)df[1]);
        } else {
            // a long step (the FP32 phase stopped early): damped, exact exponentials
            const double sc = dm > 0.5f ? 0.5 / (double)dm : 1.0;
            for (int j = 0; j < 3; j++) b[j] *= exp(-sc * (double)df[j]);
            ib[0] = recip64(b[0]);
            ib[1] = recip64(b[1]);
        }
    }
    nc.it64 += (unsigned)it64;
    nc.sites += 1u;
    if (!ok) nc.fails += 1u;
    if (a64) {
        a64[0] = log(b[0]);
        a64[1] = log(b[1]);
        a64[2] = log(b[2]);
    }
    const double s = rho * iz;
#pragma unroll
    for (int i = 0; i < 9; i++) fstar[i] = s * q[i];
    return ok;
}

// ---------------------------------------------------------------------------
// Float-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2 (about 48 significant bits).  Built on the
// error-free transformations two-sum (Knuth) and two-product (by one fused
// multiply-add); the addition is the "sloppy" form of Dekker's algorithm
// (its error is relative to |a| + |b|, which is what the residual sums
// below need).  The library is compiled without multiply-add contraction,
// so every rounding written here happens as written.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_scale(ff a, float p2) { return {a.hi * p2, a.lo * p2}; }   // p2 a power of two
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff_fast_two_sum(p, e);
}
// 1 / a: the correctly rounded FP32 reciprocal r plus one Newton-Raphson
// correction r (1 - a r), whose leading part fma(-a.hi, r, 1) is exact.
__device__ __forceinline__ ff ff_recip(ff a) {
    const float r = __frcp_rn(a.hi);
    float e = fmaf(-a.hi, r, 1.0f);
    e = fmaf(-a.lo, r, e);
    return ff_fast_two_sum(r, r * e);
}
// e^{-d} for |d| < 2^-10: 1 - d exactly as a float-float, plus the Taylor
// terms d^2/2 - d^3/6 + d^4/24 (below 2^-21) in FP32.
__device__ __forceinline__ ff ff_exp_small_neg(float d) {
    const ff s = ff_two_sum(1.0f, -d);
    const float tail = d * d * fmaf(-d, fmaf(-d, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
    return ff_fast_two_sum(s.hi, s.lo + tail);
}

// 36 q_i (weights 16, 4, 1: exact in FP32) from b = e^{a} and 1/bx, 1/by.
__device__ __forceinline__ void energy_q_ff(ff bx, ff by, ff bc, ff ibx, ff iby, ff* q) {
    const ff bc2 = ff_mul(bc, bc);
    q[0] = {16.0f, 0.0f};
    q[1] = ff_scale(ff_mul(bx, bc), 4.0f);
    q[2] = ff_scale(ff_mul(by, bc), 4.0f);
    q[3] = ff_scale(ff_mul(ibx, bc), 4.0f);
    q[4] = ff_scale(ff_mul(iby, bc), 4.0f);
    q[5] = ff_mul(ff_mul(bx, by), bc2);
    q[6] = ff_mul(ff_mul(ibx, by), bc2);
    q[7] = ff_mul(ff_mul(ibx, iby), bc2);
    q[8] = ff_mul(ff_mul(bx, iby), bc2);
}

// Residual g = E[m'] - t from q (any common scale); returns max |g| and 1/Z.
__device__ __forceinline__ float energy_residual_ff(const ff* q, const ff* tgt, ff& iz, ff* g) {
    const ff qa = ff_add(ff_add(q[1], q[2]), ff_add(q[3], q[4]));
    const ff qd = ff_add(ff_add(q[5], q[6]), ff_add(q[7], q[8]));
    iz = ff_recip(ff_add(q[0], ff_add(qa, qd)));
    const ff sx = ff_add(ff_sub(q[1], q[3]), ff_sub(ff_add(q[5], q[8]), ff_add(q[6], q[7])));
    const ff sy = ff_add(ff_sub(q[2], q[4]), ff_sub(ff_add(q[5], q[6]), ff_add(q[7], q[8])));
    const ff sc = ff_add(qa, ff_scale(qd, 2.0f));
    g[0] = ff_sub(ff_mul(sx, iz), tgt[0]);
    g[1] = ff_sub(ff_mul(sy, iz), tgt[1]);
    g[2] = ff_sub(ff_mul(sc, iz), tgt[2]);
    return fmaxf(fmaxf(fabsf(g[0].hi), fabsf(g[1].hi)), fabsf(g[2].hi));
}

// Energy-constrained quasiequilibrium for FP32 / FP16 storage from the FP32
// moments (rho, j, 2E): the FP32 phase, then Newton steps with the residual
// in float-float (covariance and 3 x 3 solve in FP32, as in energy_solve)
// until the residual is at or below 1e-12.  Writes the deviations
// gs_i = f*_i - W_i rho0, rounded once to FP32.  Returns false if the
// residual did not reach 1e-12 (the site keeps the last iterate).
__device__ __forceinline__ bool energy_solve_ff(float rho, float jx, float jy, float e2, float rho0, float* a,
                                                float* gs, NewtonCount& nc) {
    const ff ir = ff_recip({rho, 0.0f});
    const ff tg[3] = {ff_mul_f(ir, jx), ff_mul_f(ir, jy), ff_mul_f(ir, e2)};
    const float tf[3] = {tg[0].hi, tg[1].hi, tg[2].hi};
    float bx, by, bc;
    energy_phase32(tf, a, bx, by, bc, nc);
    ff b[3] = {{bx, 0.0f}, {by, 0.0f}, {bc, 0.0f}};
    ff ib[2] = {ff_recip(b[0]), ff_recip(b[1])};
    ff q[9], iz = {1.0f, 0.0f};
    bool ok = false;
    int it = 0;
    for (;; it++) {
        ff g[3];
        energy_q_ff(b[0], b[1], b[2], ib[0], ib[1], q);
        const float r = energy_residual_ff(q, tg, iz, g);
        ok = r <= (float)kNewtonTol;
        if (ok || it == kNewton64Max) break;
        float qf[9], Cf[6], gf[3], df[3], Zf, unused[3];
        const float zero[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 9; i++) qf[i] = q[i].hi;
        energy_terms<float>(qf, zero, Zf, unused, Cf);
        gf[0] = g[0].hi;
        gf[1] = g[1].hi;
        gf[2] = g[2].hi;
        if (!spd3_solve(Cf, gf, df)) break;
        const float dm = fmaxf(fmaxf(fabsf(df[0]), fabsf(df[1])), fabsf(df[2]));
        if (dm < 0x1p-10f) {
            for (int j = 0; j < 3; j++) b[j] = ff_mul(b[j], ff_exp_small_neg(df[j]));
        } else {
            // a long step (the FP32 phase stopped early): damped; any positive
            // b is a member of the family, so the new b need not be exact
            const float sc = dm > 0.5f ? 0.5f / dm : 1.0f;
            for (int j = 0; j < 3; j++) b[j] = {b[j].hi * expf(-sc * df[j]), 0.0f};
        }
        ib[0] = ff_recip(b[0]);
        ib[1] = ff_recip(b[1]);
    }
    nc.it64 += (unsigned)it;
    nc.sites += 1u;
    if (!ok) nc.fails += 1u;
    // f*_i = rho q_i / Z; W_i as float-float constants for the deviation
    const ff s = ff_mul_f(iz, rho);
    constexpr double w[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    constexpr float whi[3] = {(float)w[0], (float)w[1], (float)w[2]};
    constexpr float wlo[3] = {(float)(w[0] - (double)whi[0]), (float)(w[1] - (double)whi[1]),
                              (float)(w[2] - (double)whi[2])};
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const int k = i == 0 ? 0 : (i < 5 ? 1 : 2);
        const ff d = ff_sub(ff_mul(s, q[i]), ff_mul_f({whi[k], wlo[k]}, rho0));
        gs[i] = d.hi + d.lo;
    }
    return ok;
}

}  // namespace lbm
