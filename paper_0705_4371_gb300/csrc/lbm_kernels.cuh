// lbm_kernels.cuh -- kernels of one time step (template definitions; each
// storage type is instantiated in its own translation unit).
//
//   k_collide_d2q9   the whole time step in one persistent launch: every
//                    warp walks row tiles of 32 x VEC sites (pull-stream +
//                    moments + f* + dS + LBGK), appends the sites with
//                    dS > delta to a global candidate list (warp ballot, one
//                    atomic per tile that has any), and the block that
//                    finishes last runs the global radix select of the k
//                    largest dS and the Ehrenfests' step f <- f* at those
//                    sites (Sec. 3.2; (ESLB)).  No block waits for another.
//   k_collide_site   the same step, one site per thread (D1Q3)
//   k_select         the selection as a stand-alone kernel (test hook)
#pragma once

#include <algorithm>

#include <cuda.h>

#include "lbm_device.cuh"
#include "lbm_energy.cuh"
#include "lbm_mlp.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kSelectThreads = 1024;
constexpr int kSiteBlock = 256;      // one-site-per-thread kernels
constexpr int kStage = 1024;         // candidates staged in shared memory by the last block

template <typename L, typename T, int EQ>
__device__ __forceinline__ void equilibrium(const Params& P, T drho, T rho, T ux, T uy, T* gs) {
    if constexpr (EQ == EQ_POLY) feq_poly<L, T>(drho, rho, ux, uy, gs);
    else feq_entropic<L, T>(rho, ux, uy, Par<T>::rho0(P), gs);
}

// Energy-constrained entropic f* (D2Q9 only) as deviations from the
// moments (drho, j, 2E); Newton from the start point a0 (the network's
// warm start in the learned form) or, when a0 is null, from the polynomial
// start point (3 u_x, 3 u_y, 0) (the multipliers of the first-order
// expansion about rest).
template <typename T, int EQ>
__device__ __forceinline__ void equilibrium_energy(const Params& P, T rho, T jx, T jy, T e2, T* gs,
                                                   NewtonCount& nc, const float* a0 = nullptr) {
    if constexpr (sizeof(T) == 4) {
        // FP32 / FP16 storage: the float-float finish (no FP64 work)
        float a[3];
        if (a0) {
            a[0] = a0[0];
            a[1] = a0[1];
            a[2] = a0[2];
        } else {
            const float ir = __frcp_rn(rho);
            a[0] = 3.0f * (jx * ir);
            a[1] = 3.0f * (jy * ir);
            a[2] = 0.0f;
        }
        energy_solve_ff(rho, jx, jy, e2, Par<T>::rho0(P), a, gs, nc);
    } else {
        // FP64 storage: FP64 finish to 4e-15 (the FP64 parity bound)
        const double r = (double)rho, ir = recip64(r);
        const double ux = (double)jx * ir, uy = (double)jy * ir;
        float a[3] = {3.0f * (float)ux, 3.0f * (float)uy, 0.0f};
        if (a0) {
            a[0] = a0[0];
            a[1] = a0[1];
            a[2] = a0[2];
        }
        double fs[9];
        energy_solve(r, ux, uy, (double)e2 * ir, a, fs, nc, 4e-15);
        const double rho0 = P.rho0;
#pragma unroll
        for (int i = 0; i < 9; i++) gs[i] = (T)(fs[i] - D2Q9::w(i) * rho0);
    }
}

template <typename L, typename T>
__device__ __forceinline__ void moments(const T* g, T rho0, T& drho, T& rho, T& jx, T& jy) {
    if constexpr (L::Q == 9) {
        // pairwise sums (D2Q9 numbering: 1..4 E N W S, 5..8 NE NW SW SE)
        drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
        jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
        jy = ((g[2] - g[4]) + (g[5] - g[8])) + (g[6] - g[7]);
    } else {
        // D1Q3: 0 rest, 1 left, 2 right
        drho = (g[0] + g[1]) + g[2];
        jx = g[2] - g[1];
        jy = T(0);
    }
    rho = rho0 + drho;
}

// u = j / rho: FP64 divides (as the oracle does); FP32 multiplies by the
// refined reciprocal (recip).
template <typename T>
__device__ __forceinline__ void velocity(T jx, T jy, T rho, T& ux, T& uy) {
    if constexpr (sizeof(T) == 8) {
        ux = jx / rho;
        uy = jy / rho;
    } else {
        const T r = recip<T>(rho);
        ux = jx * r;
        uy = jy * r;
    }
}

// 2E = sum |v|^2 f = sum |v|^2 g + rho0 sum W |v|^2 of a site's deviations.
template <typename L, typename T>
__device__ __forceinline__ T energy_moment(const T* g, T rho0) {
    T e2 = T(L::sum_w_c2) * rho0;
#pragma unroll
    for (int i = 0; i < L::Q; i++)
        if (L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) == 1) e2 += g[i];
        else if (L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) == 2) e2 += T(2) * g[i];
    return e2;
}

// Quasiequilibrium of a gathered site (shared by the collision, the
// Ehrenfests' step and the exports so that all round identically).  a0:
// Newton start point of the energy forms (null: the polynomial start).
template <typename L, typename T, int EQ>
__device__ __forceinline__ void site_equilibrium(const Params& P, const T* g, T* gs, T& rho, T& ux,
                                                 T& uy, NewtonCount& nc, const float* a0 = nullptr) {
    T drho, jx, jy;
    moments<L, T>(g, Par<T>::rho0(P), drho, rho, jx, jy);
    velocity<T>(jx, jy, rho, ux, uy);
    if constexpr (EQ >= EQ_ENERGY) {
        const T e2 = energy_moment<L, T>(g, Par<T>::rho0(P));
        equilibrium_energy<T, EQ>(P, rho, jx, jy, e2, gs, nc, a0);
    } else {
        (void)nc;
        (void)a0;
        equilibrium<L, T, EQ>(P, drho, rho, ux, uy, gs);
    }
}
template <typename L, typename T, int EQ>
__device__ __forceinline__ void site_equilibrium(const Params& P, const T* g, T* gs, T& rho, T& ux,
                                                 T& uy) {
    NewtonCount nc = {0, 0, 0, 0};
    site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy, nc);
}

// Per-thread Newton counts flushed to the run's statistics (energy forms).
__device__ __forceinline__ void flush_newton(const Params& P, NewtonCount& nc) {
    unsigned v[4] = {nc.it32, nc.it64, nc.sites, nc.fails};
#pragma unroll
    for (int j = 0; j < 4; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    if ((threadIdx.x & 31) == 0 && v[2] > 0) {
        for (int j = 0; j < 4; j++) atomicAdd(P.newton_stats + j, (unsigned long long)v[j]);
        if (v[3] > 0) atomicOr(P.err, ERR_NEWTON);
    }
}

// FP64 recomputation of dS from the stored populations (precision form).
template <typename L, typename T, int EQ>
__device__ __noinline__ double delta_s_fp64(PopArr<L::Q, T> g, double rho0) {
    double gd[L::Q], gs[L::Q], drho, rho, jx, jy, ux, uy;
#pragma unroll
    for (int i = 0; i < L::Q; i++) gd[i] = (double)g.v[i];
    moments<L, double>(gd, rho0, drho, rho, jx, jy);
    velocity<double>(jx, jy, rho, ux, uy);
    if constexpr (EQ >= EQ_ENERGY) {
        double e2 = L::sum_w_c2 * rho0;
#pragma unroll
        for (int i = 0; i < L::Q; i++) e2 += (double)(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)) * gd[i];
        float a[3] = {3.0f * (float)ux, 3.0f * (float)uy, 0.0f};
        double fs[9];
        NewtonCount nc = {0, 0, 0, 0};
        energy_solve(rho, ux, uy, e2 / rho, a, fs, nc, 4e-15);
#pragma unroll
        for (int i = 0; i < L::Q; i++) gs[i] = fs[i] - L::w(i) * rho0;
    } else if constexpr (EQ == EQ_POLY) {
        feq_poly<L, double>(drho, rho, ux, uy, gs);
    } else {
        feq_entropic<L, double>(rho, ux, uy, rho0, gs);
    }
    return delta_s_exact<L, double>(gd, gs, rho0);
}

// Per-site update after the gather: moments, f*, the dS bound, LBGK.
// g: pre-collision deviations in, post-collision deviations out.
// Returns true when the bound does not clear the site (dS may exceed delta):
// its exact dS is then evaluated later from the unchanged source field.
// ELBM (elbmLB): alpha with S(f + alpha (f* - f)) = S(f) for one site, from
// the full populations f and f*, in the arithmetic U of the storage (FP64
// to 1e-15 relative for FP64 storage; FP32 to its rounding for FP32 and
// FP16 storage, whose populations carry FP32 rounding already).  With
// D = f* - f and x_i = D_i / f_i the condition is
// G(a) = sum f_i phi(a x_i) - a R = 0, R = sum D_i log1p(x_i) (sum D = 0 and
// ln f* linear in the conserved moments remove the two entropies'
// cancellation); G is convex, G(0) = 0, G(1) <= 0, so the root in
// [1, alpha_max] (alpha_max = 1 / max(-x_i): f + a D >= 0) is unique.
// Newton with G'(a) = sum D_i log1p(a x_i) - R, falling back to bisection
// whenever a step leaves the bracket.  The start point is the root of the
// series of G to second order in x, a = 2 + S3 / (3 S2) with
// Sn = sum f_i x_i^n; near equilibrium (max |x| < 0.1, so alpha_max > 10)
// the bracket check at alpha_max is skipped.  Stop: FP64 when a step or the
// bracket falls below 1e-15 relative; FP32 once a step is below 3e-4
// relative (Newton converges quadratically with G''/G' ~ 1/2 here, so the
// result of that step is within about 1e-7 of the root, FP32's rounding;
// iterating further in FP32 only chases the rounding noise of G, and the
// slowest lane holds its whole warp).  a = 2 when f = f*; alpha_max when
// the entropy still exceeds S(f) there; -1 when some f_i or f*_i is not
// positive.
// Near equilibrium (max |x| < 0.1, almost every site) both precisions take
// a branch-free path instead: with Sn = sum f_i x_i^n, the series of G / a is
//   P(a) = sum_{n>=2} (-1)^n Sn (a^{n-1}/n - 1)/(n - 1),
// whose terms beyond n = 10 are below 1e-9 S2 for |a x| <= 0.21 (the root
// lies within 2 +- max|x| / 3 there), far below FP32's rounding of P (about
// 1e-7 S2), and beyond n = 24 below 1e-18 S2, under FP64's; Newton steps on
// P from the series root 2 + S3 / (3 S2) (three in FP32, four in FP64: P is
// almost linear, P' ~ S2 / 2, and the start is off by O(max|x|^2)) reach the
// root.  No logarithm and no data-dependent loop, so the lanes of a warp stay
// together.
template <int Q, int NT, typename U>
__device__ __forceinline__ U elbm_alpha_series(const U* D, const U* x) {
    // c_n = (-1)^n Sn / (n - 1), n = 2..NT, with Sn = sum D_i x_i^{n-1}
    U c[NT + 1];
#pragma unroll
    for (int n = 0; n <= NT; n++) c[n] = U(0);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        U t = D[i] * x[i];
#pragma unroll
        for (int n = 2; n <= NT; n++) {
            c[n] += t;
            t *= x[i];
        }
    }
    if (!(c[2] > U(0))) return U(2);
    const U a0 = U(2) + c[3] / (U(3) * c[2]);   // 2 + S3 / (3 S2)
    // P(a) = a B(a) - sum c_n with B(a) = sum b_n a^{n-2}, b_n = c_n / n;
    // P'(a) = sum d_n a^{n-2}, d_n = c_n (n - 1) / n
    U b[NT + 1], d[NT + 1], sumc = U(0);
#pragma unroll
    for (int n = 2; n <= NT; n++) {
        const U cn = ((n & 1) ? -c[n] : c[n]) * U(1.0 / (n - 1));
        sumc += cn;
        b[n] = cn * U(1.0 / n);
        d[n] = cn * U((n - 1.0) / n);
    }
    U a = a0;
#pragma unroll
    for (int it = 0; it < (sizeof(U) == 8 ? 4 : 3); it++) {
        U B = b[NT], dP = d[NT];
#pragma unroll
        for (int n = NT - 1; n >= 2; n--) {
            B = dfma<U>(B, a, b[n]);
            dP = dfma<U>(dP, a, d[n]);
        }
        a -= (a * B - sumc) / dP;
    }
    return a;
}

template <typename L, typename U>
__device__ __noinline__ U elbm_alpha(const U* f, const U* fs) {
    constexpr bool fp64 = sizeof(U) == 8;
    constexpr U step_tol = fp64 ? U(1e-15) : U(3e-4);
    constexpr U bracket_tol = fp64 ? U(1e-15) : U(4.0 * 1.1920929e-7);
    constexpr int max_it = fp64 ? 100 : 40;
    U D[L::Q], x[L::Q], R = U(0), xneg = U(0), s2 = U(0), s3 = U(0), xm = U(0);
    bool moved = false, positive = true;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        positive &= f[i] > U(0) && fs[i] > U(0);
        D[i] = fs[i] - f[i];
        moved |= D[i] != U(0);
        x[i] = D[i] / f[i];
        xneg = fmax(xneg, -x[i]);
        xm = fmax(xm, fabs(x[i]));
    }
    if (!positive) return U(-1);
    if (!moved || !(xneg > U(0))) return U(2);
    // near equilibrium the series path: terms to n = 10 reach FP32's rounding,
    // to n = 24 FP64's (the omitted terms are below 1e-18 S2 for |a x| <= 0.21)
    if (xm < U(0.1)) return elbm_alpha_series<L::Q, fp64 ? 24 : 10, U>(D, x);
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        R += D[i] * log1p(x[i]);
        s2 += D[i] * x[i];
        s3 += D[i] * x[i] * x[i];
    }
    if (!(R > U(0))) return U(2);
    const U amax = U(1) / xneg;
    auto G = [&](U a) {
        U s = U(0);
#pragma unroll
        for (int i = 0; i < L::Q; i++) s += f[i] * phi_fn<U>(a * x[i]);
        return s - a * R;
    };
    U lo = U(1), hi = amax;
    if (!(xm < U(0.1)) && G(hi) <= U(0)) return hi;
    U a = U(2) + s3 / (U(3) * s2);
    if (!(a > lo && a < hi)) a = U(0.5) * (lo + hi);
    for (int it = 0; it < max_it; it++) {
        const U g = G(a);
        if (g <= U(0)) lo = a;
        else hi = a;
        U dg = -R;
#pragma unroll
        for (int i = 0; i < L::Q; i++) dg += D[i] * log1p(a * x[i]);
        U na = a - g / dg;
        const bool newton = na > lo && na < hi;
        if (!newton) na = U(0.5) * (lo + hi);
        const bool done = (newton && fabs(na - a) <= step_tol * a) || hi - lo <= bracket_tol * hi;
        a = na;
        if (done) break;
    }
    return a;
}

// The ELBM step factor -alpha beta of a site from its deviations (kept out
// of line: the LBGK path does not carry its arrays).
template <typename L, typename T>
__device__ __noinline__ T elbm_factor(PopArr<L::Q, T> g, PopArr<L::Q, T> gs, T rho0, T beta) {
    T fd[L::Q], fsd[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        fd[i] = g.v[i] + T(L::w(i)) * rho0;
        fsd[i] = gs.v[i] + T(L::w(i)) * rho0;
    }
    T a = elbm_alpha<L, T>(fd, fsd);
    if (a < T(0)) a = T(2);   // outside the positive cone: dS = +inf, LBGK
    return -a * beta;
}

// Exact dS of a site from its pre-collision deviations g and its
// quasiequilibrium gs (rho0, dl: the run's rho0 and delta in T).  The
// precision form (recheck) decides the sites whose FP32 dS lies within band
// of delta (a bound on the FP32 evaluation error of dS, set by the host) in
// FP64; the value kept for ranking then stays on the same side of delta.
// Returns dS in T (NaN for a non-finite state).  Out of line: the sites the
// bound does not clear are few, and the update path keeps its registers.
template <typename L, typename T, int EQ>
__device__ __noinline__ T resolved_ds(PopArr<L::Q, T> g, PopArr<L::Q, T> gs, T rho0, T dl, double delta,
                                      double rho0d, double band, int recheck) {
    T ds = delta_s_exact<L, T>(g.v, gs.v, rho0);
    if (recheck && isfinite(ds) && fabs((double)ds - delta) <= band) {
        const double d64 = delta_s_fp64<L, T, EQ>(g, rho0d);
        if (d64 > delta) ds = (T)d64 > dl ? (T)d64 : nextafter(dl, T(INFINITY));
        else ds = T(-1);
    }
    return ds;
}

// The same from the site's pre-collision deviations g and quasiequilibrium
// gs already at hand.
template <typename L, typename T, int EQ>
__device__ __forceinline__ T site_ds(const Params& P, const T* g, const T* gs) {
    PopArr<L::Q, T> ga, gsa;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        ga.v[i] = g[i];
        gsa.v[i] = gs[i];
    }
    return resolved_ds<L, T, EQ>(ga, gsa, Par<T>::rho0(P), Par<T>::delta(P), P.delta, P.rho0, P.recheck_band,
                                 P.recheck);
}

// A ghost column of a slab (a copy of a neighbour's sites: never a candidate).
__device__ __forceinline__ bool ghost_column(const Params& P, int x) {
    return P.slab && (x < P.own_x0 || x >= P.own_x1);
}

// PROBE = false: the caller guarantees the site is not the probe site.
// PROJ: remove the rounding defects of the conserved moments of f - f*
// (conserve_neq; FP32 storage).  g leaves as the deviations to store, before
// the storage's rounding (store_round).  RESOLVE: a site the bound does not
// clear has its dS evaluated here, from the pre-collision g and f* at hand
// (site_ds), and stored to *ds_out (-1 for every other site, and for a
// slab's ghost columns).
template <typename L, typename T, int EQ, bool PROJ, bool PROBE = true, bool RESOLVE = false>
__device__ __forceinline__ bool update_site(const Params& P, T* g, int x, int y, long long t,
                                            bool& nonfinite, NewtonCount& nc,
                                            const float* a0 = nullptr, T* ds_out = nullptr) {
    T gs[L::Q], rho, ux, uy;
    site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy, nc, a0);
    nonfinite |= !isfinite(rho + ux + uy);
    if (PROBE && x == P.probe_x && y == P.probe_y && P.probe_ring)
        P.probe_ring[t % P.ring_cap] = (double)ux;
    T d[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) d[i] = g[i] - gs[i];
    if constexpr (PROJ) conserve_neq<L, EQ>(d);
    // (no short-circuit: the site's update stays one branch-free block)
    const bool pending =
        (P.k > 0) & !ds_cleared<L, T, EQ>(d, gs, rho, ux, uy, Par<T>::rho0(P), Par<T>::delta(P));
    if constexpr (RESOLVE) {
        T ds = T(-1);
        if (pending && !ghost_column(P, x)) ds = site_ds<L, T, EQ>(P, g, gs);
        *ds_out = ds;
    }
    T nb2 = T(-2) * Par<T>::beta(P);
    if constexpr (EQ == EQ_ENTROPIC) {
        if (P.elbm) {
            // f' = f + alpha beta (f* - f) (elbmLB)
            PopArr<L::Q, T> ga, gsa;
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                ga.v[i] = g[i];
                gsa.v[i] = gs[i];
            }
            nb2 = elbm_factor<L, T>(ga, gsa, Par<T>::rho0(P), Par<T>::beta(P));
        }
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++) g[i] = dfma<T>(nb2, d[i], g[i]);
    return pending;
}

// Learned form: the network's Newton start point for the warp's 32 sites
// (lane l: its gathered site g, or valid = false).  Every lane must call it.
template <typename T>
__device__ __forceinline__ void mlp_site_start(const Params& P, const MlpSmem& ms, bool valid,
                                               const T* g, float* a) {
    float rho = 1.0f, ux = 0.0f, uy = 0.0f, e2 = 0.0f;
    if (valid) {
        T drho, r, jx, jy;
        moments<D2Q9, T>(g, Par<T>::rho0(P), drho, r, jx, jy);
        rho = (float)r;
        const float ir = 1.0f / rho;
        ux = (float)jx * ir;
        uy = (float)jy * ir;
        e2 = (float)energy_moment<D2Q9, T>(g, Par<T>::rho0(P));
        valid = rho > 0.0f && isfinite(rho + ux + uy + e2);
    }
    mlp_warm_start(ms, valid, rho, ux, uy, e2, a);
}

// Shared copy of the network in the learned form's kernels (empty otherwise).
template <int EQ> struct MlpSlot {
    __device__ void fill(const Params&) {}
};
template <> struct MlpSlot<EQ_ENERGY_MLP> {
    MlpSmem s;
    __device__ void fill(const Params& P) { mlp_fill(s, P.mlp); }
};

// Exact dS of site (x, y) with the pre-collision state re-gathered from the
// source field (not written during a step); -1 on a slab's ghost column.
template <typename L, typename S, int EQ>
__device__ __noinline__ typename Store<S>::T resolve_ds(const Params& P, int x, int y) {
    using T = typename Store<S>::T;
    if (ghost_column(P, x)) return T(-1);
    T g[L::Q], gs[L::Q], rho, ux, uy;
    gather_site<L, S>(P, x, y, g);
    site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
    return site_ds<L, T, EQ>(P, g, gs);
}

// Warp-level append of candidates (sites with dS > delta) to the global
// list: one ballot, one atomic per warp when any lane has a candidate.
// Every lane of the warp must call it.
template <typename T>
__device__ __forceinline__ void warp_push(const Params& P, bool cand, T ds, unsigned site) {
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(P.cand_count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cand) {
        const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
        P.cand_key[slot] = ds_key((double)ds);
        P.cand_idx[slot] = site;
    }
}

// ---------------------------------------------------------------------------
// Block stage of the selection (k sites of the whole grid are selected, so a
// block never contributes more than its own k best): a block holds its
// candidates in shared memory, cuts them to its k largest (dS, -index) with
// the block radix select whenever the buffer fills, and flushes what it kept
// to the global list when it ends.  The global select then ranks at most
// k x blocks keys.  With k too large for a cut to free room, the block
// flushes its buffer to the global list instead (which holds one slot per
// site and cannot overflow).  CAP entries: room for the entries kept by a
// cut plus one round of appends (a round of pending sites resolved by the
// block, or the sites of one staged tile).
// ---------------------------------------------------------------------------
constexpr int kBlockCand = 320;   // room for a round of 256 candidates above a cut

template <int CAP>
struct BlockCandT {
    static constexpr int kCap = CAP;
    unsigned long long key[CAP];
    unsigned idx[CAP];
    unsigned n;          // candidates appended (entries beyond CAP went to the global list)
    unsigned base;
};
using BlockCand = BlockCandT<kBlockCand>;

// Warp-level append to the block's buffer (every lane calls).  Returns the
// number of candidates the warp appended (the same on every lane).
template <typename T, int CAP>
__device__ __forceinline__ unsigned block_push(const Params& P, BlockCandT<CAP>& bc, bool cand, T ds,
                                               unsigned site) {
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (m == 0) return 0u;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&bc.n, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cand) {
        const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
        const unsigned long long key = ds_key((double)ds);
        if (slot < (unsigned)CAP) {
            bc.key[slot] = key;
            bc.idx[slot] = site;
        } else {
            // no room (the callers cut or flush before it can happen)
            const unsigned g = atomicAdd(P.cand_count, 1u);
            P.cand_key[g] = key;
            P.cand_idx[g] = site;
        }
    }
    return (unsigned)__popc(m);
}

// Keep the k best of the buffer (all threads call; blockDim >= 128).
template <int CAP>
__device__ __noinline__ void block_cut(BlockCandT<CAP>& bc, TopkScratch& sc, int k) {
    constexpr int kPer = (CAP + 127) / 128;
    const int tid = threadIdx.x, nt = blockDim.x;
    __syncthreads();
    const int n = (int)min(bc.n, (unsigned)CAP);
    if (n <= k) return;   // uniform: n was read after the barrier
    const Thresh th = block_topk(sc, n, k, [&](int e) { return bc.key[e]; }, [&](int e) { return bc.idx[e]; });
    unsigned long long kk[kPer];
    unsigned ii[kPer];
    bool keep[kPer];
#pragma unroll
    for (int r = 0; r < kPer; r++) {
        const int e = tid + r * nt;
        keep[r] = e < n && th.selected(bc.key[e], bc.idx[e]);
        kk[r] = keep[r] ? bc.key[e] : 0ull;
        ii[r] = keep[r] ? bc.idx[e] : 0u;
    }
    __syncthreads();
    if (tid == 0) bc.n = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; r++) {
        if (keep[r]) {
            const unsigned slot = atomicAdd(&bc.n, 1u);
            bc.key[slot] = kk[r];
            bc.idx[slot] = ii[r];
        }
    }
    __syncthreads();
}

// Move the buffer to the global candidate list (all threads call).
template <int CAP>
__device__ __noinline__ void block_flush(const Params& P, BlockCandT<CAP>& bc) {
    __syncthreads();
    const int n = (int)min(bc.n, (unsigned)CAP);
    if (n == 0) return;   // uniform
    if (threadIdx.x == 0) bc.base = atomicAdd(P.cand_count, (unsigned)n);
    __syncthreads();
    const unsigned base = bc.base;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        P.cand_key[base + e] = bc.key[e];
        P.cand_idx[base + e] = bc.idx[e];
    }
    __syncthreads();
    if (threadIdx.x == 0) bc.n = 0;
    __syncthreads();
}

// Make room for another blockDim candidates (all threads call).
template <int CAP>
__device__ __forceinline__ void block_room(const Params& P, BlockCandT<CAP>& bc, TopkScratch& sc) {
    __syncthreads();
    const int room = CAP - (int)blockDim.x;
    if ((int)bc.n > room) {   // uniform
        if (P.k <= room) block_cut(bc, sc, P.k);
        else block_flush(P, bc);
    }
}

// What the block contributes to the global select: its k best (all threads).
template <int CAP>
__device__ __forceinline__ void block_finish(const Params& P, BlockCandT<CAP>& bc, TopkScratch& sc) {
    if (P.k > 0) block_cut(bc, sc, P.k);
    block_flush(P, bc);
}

// ---------------------------------------------------------------------------
// Global selection and Ehrenfests' step, run by one block: the last block of
// a stream-collide launch, or the stand-alone select kernel.
//   mode 0: select among the candidates (or replay a given list), overwrite
//           the LBGK output of the selected sites with f* (Sec. 3.2; (ESLB)),
//           log the count and advance the step counter;
//   mode 1: select only (the select-only test hook; and a slab's own k best,
//           with their keys, when the global selection is made across
//           slabs).
// Candidates are staged in shared memory when they fit; larger sets are
// ranked in place in global memory.
// ---------------------------------------------------------------------------
struct SelectShared {
    TopkScratch sc;
    int nsel;
    unsigned cnt;
};

template <typename L, typename S, int EQ>
__device__ __noinline__ void select_and_fix(const Params& P, SelectShared& ss,
                                            unsigned long long* stage_key, unsigned* stage_idx,
                                            int stage_cap, int mode) {
    using T = typename Store<S>::T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long t = __ldcg(P.step);   // used at the end: its latency overlaps the selection
    long long r = 0;
    bool replay = false;
    if (P.replay_cnt) {
        r = t - P.replay_t0;
        replay = r >= 0 && r < P.replay_n;
    }
    int mine = -1;   // the site this thread selected itself, when it did (j = tid)
    if (replay) {
        const int c = P.replay_cnt[r];
        const long long off = P.replay_off[r];
        for (int j = tid; j < c; j += nt) P.sel_idx[j] = P.replay_idx[off + j];
        if (tid == 0) ss.nsel = c;
    } else if (P.k <= 0) {
        if (tid == 0) ss.nsel = 0;
    } else {
        const int n = (int)__ldcg(P.cand_count);
        if (n <= P.k) {
            for (int j = tid; j < n; j += nt) {
                const int id = (int)__ldcg(P.cand_idx + j);
                P.sel_idx[j] = id;
                if (j == tid) mine = id;
                if (P.sel_key) P.sel_key[j] = __ldcg(P.cand_key + j);
            }
            if (tid == 0) ss.nsel = n;
        } else {
            const bool staged = n <= stage_cap;
            if (staged) {
                for (int j = tid; j < n; j += nt) {
                    stage_key[j] = __ldcg(P.cand_key + j);
                    stage_idx[j] = __ldcg(P.cand_idx + j);
                }
                __syncthreads();
            }
            auto keyat = [&](int e) { return staged ? stage_key[e] : __ldcg(P.cand_key + e); };
            auto idat = [&](int e) { return staged ? stage_idx[e] : __ldcg(P.cand_idx + e); };
            const Thresh th = block_topk(ss.sc, n, P.k, keyat, idat);
            if (tid == 0) ss.cnt = 0;
            __syncthreads();
            for (int j = tid; j < n; j += nt) {
                const unsigned id = idat(j);
                const unsigned long long key = keyat(j);
                if (th.selected(key, id)) {
                    const unsigned s = atomicAdd(&ss.cnt, 1u);
                    if (s < (unsigned)P.k) {   // exactly k; bounds the write
                        P.sel_idx[s] = (int)id;
                        if (P.sel_key) P.sel_key[s] = key;
                    }
                }
            }
            if (tid == 0) ss.nsel = P.k;
        }
    }
    __syncthreads();
    const int m = ss.nsel;
    if (mode == 0) {
        const long long nsites = (long long)P.nx * P.ny;
        for (int j = tid; j < m; j += nt) {
            const int site = j == tid && mine >= 0 ? mine : P.sel_idx[j];
            if (site < 0 || site >= nsites) { atomicOr(P.err, ERR_REPLAY); continue; }
            const int x = site % P.nx, y = site / P.nx;
            if (is_solid(P, x, y)) { atomicOr(P.err, ERR_REPLAY); continue; }
            const long long o = (long long)y * P.nxp + x;
            // f* of the site from its post-collision populations: the
            // collision conserves every moment f* depends on, so this is f*
            // of the pre-collision state, read at the site itself (nine
            // independent loads, no boundary rules: the block that runs this
            // is alone on the device by then, and its code path stays short)
            T g[L::Q], gs[L::Q], rho, ux, uy;
#pragma unroll
            for (int i = 0; i < L::Q; i++) g[i] = Store<S>::load(P.dst, i * P.plane + o);
            site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
            if constexpr (Store<S>::kProject) {
                // f' = f* = f - (f - f*), with the conserved moments of
                // f - f* freed of rounding as in the collision
                T d[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; i++) d[i] = g[i] - gs[i];
                conserve_neq<L, EQ>(d);
#pragma unroll
                for (int i = 0; i < L::Q; i++) gs[i] = g[i] - d[i];
            }
#pragma unroll
            for (int i = 0; i < L::Q; i++)
                Store<S>::store(P.dst, i * P.plane + o, store_round<L, S>(i, gs[i]));
        }
    }
    __syncthreads();
    if (tid == 0) {
        *P.sel_count = m;
        *P.cand_count = 0;
        if (mode == 0) {
            P.count_ring[t % P.ring_cap] = m;
            *P.step = t + 1;
        }
    }
}

// End of a stream-collide block: resolve the block's pending sites (exact
// dS, candidates appended), publish the block's writes, take a ticket; the
// block that takes the last ticket first resolves the pending sites that did
// not fit in any block's list, then runs the global selection and the
// Ehrenfests' step for the whole grid.  No block ever waits for another.
constexpr int kPend = 2048;   // pending sites kept per block in shared memory

struct FinishShared {
    SelectShared ss;
    unsigned long long key[kStage];
    unsigned idx[kStage];
    unsigned pend[kPend];
    BlockCand bc;
    unsigned npend;
    int is_last;
};

// Warp-level append of pending sites to the block list of capacity cap
// (overflow: global).  Returns the number the warp appended (the same on
// every lane).
__device__ __forceinline__ unsigned warp_pend(const Params& P, unsigned* list, unsigned* nlist, int cap, bool pend,
                                              unsigned site) {
    const unsigned m = __ballot_sync(0xffffffffu, pend);
    if (m == 0) return 0u;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(nlist, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pend) {
        const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < (unsigned)cap) list[slot] = site;
        else P.pend_idx[atomicAdd(P.pend_count, 1u)] = site;
    }
    return (unsigned)__popc(m);
}
__device__ __forceinline__ unsigned warp_pend(const Params& P, FinishShared& fs, bool pend, unsigned site) {
    return warp_pend(P, fs.pend, &fs.npend, kPend, pend, site);
}

// Exact dS of n pending sites, appending the candidates to the block's
// buffer bc (its k best reach the global list) or, with bc null, straight
// to the global list; all threads call with the same n.
template <typename L, typename S, int EQ, typename SiteAt, typename BC = BlockCand>
__device__ void resolve_list(const Params& P, int n, SiteAt site_at, BC* bc, TopkScratch* sc) {
    using T = typename Store<S>::T;
    const T delta = Par<T>::delta(P);
    for (int b = 0; b < n; b += blockDim.x) {
        if (bc) block_room(P, *bc, *sc);
        const int j = b + (int)threadIdx.x;
        unsigned site = 0;
        T ds = T(-1);
        if (j < n) {
            site = site_at(j);
            ds = resolve_ds<L, S, EQ>(P, (int)(site % (unsigned)P.nx), (int)(site / (unsigned)P.nx));
        }
        if (bc) block_push<T>(P, *bc, ds > delta, ds, site);
        else warp_push<T>(P, ds > delta, ds, site);
    }
}

template <typename L, typename S, int EQ, typename BC>
__device__ __forceinline__ void finish_parts(const Params& P, const unsigned* pend, unsigned npend, int pend_cap,
                                             int& is_last, SelectShared& ss, BC& bc,
                                             unsigned long long* stage_key, unsigned* stage_idx,
                                             int stage_cap) {
    const int np = (int)min(npend, (unsigned)pend_cap);
    if (np > 0) resolve_list<L, S, EQ>(P, np, [&](int j) { return pend[j]; }, &bc, &ss.sc);
    block_finish(P, bc, ss.sc);
    // the barrier makes the block's writes visible to thread 0, whose
    // device-scope fence then orders all of them before the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nb = gridDim.x * gridDim.y;
        const unsigned tk = atomicAdd(P.ticket, 1u);
        __threadfence();
        is_last = (tk == nb - 1);
    }
    __syncthreads();
    if (is_last) {
        // (a kernel without pending lists, pend null, never appends to the global one)
        const int ng = pend ? (int)__ldcg(P.pend_count) : 0;
        if (ng > 0) {
            resolve_list<L, S, EQ>(P, ng, [&](int j) { return __ldcg(P.pend_idx + j); }, &bc, &ss.sc);
            block_finish(P, bc, ss.sc);
            __syncthreads();
            if (threadIdx.x == 0) *P.pend_count = 0;
        }
        __threadfence_block();
        select_and_fix<L, S, EQ>(P, ss, stage_key, stage_idx, stage_cap, P.slab ? 1 : 0);
        if (threadIdx.x == 0) {
            *P.ticket = 0;
            if (P.tile_counter) *P.tile_counter = 0;
        }
    }
}

template <typename L, typename S, int EQ>
__device__ __forceinline__ void finish_block(const Params& P, FinishShared& fs) {
    __syncthreads();
    finish_parts<L, S, EQ>(P, fs.pend, fs.npend, kPend, fs.is_last, fs.ss, fs.bc, fs.key, fs.idx, kStage);
}

// Boundary site (or any site of the first step after a state upload): gather
// with the boundary rules, update, store.  Returns bit 0: non-finite,
// bit 1: pending.
template <typename S, int EQ>
__device__ __noinline__ int boundary_site(const Params& P, int x, int y, long long t) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    const long long o = (long long)y * P.nxp + x;
    T g[L::Q];
    bool nonfinite = false, pending = false;
    NewtonCount nc = {0, 0, 0, 0};
    if (is_solid(P, x, y)) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) g[i] = T(0);
    } else {
        gather_site<L, S>(P, x, y, g);
        pending = update_site<L, T, EQ, Store<S>::kProject>(P, g, x, y, t, nonfinite, nc);
#pragma unroll
        for (int i = 0; i < L::Q; i++) g[i] = store_round<L, S>(i, g[i]);
    }
    if constexpr (EQ >= EQ_ENERGY) {
        if (nc.sites) {
            atomicAdd(P.newton_stats + 0, (unsigned long long)nc.it32);
            atomicAdd(P.newton_stats + 1, (unsigned long long)nc.it64);
            atomicAdd(P.newton_stats + 2, (unsigned long long)nc.sites);
            if (nc.fails) {
                atomicAdd(P.newton_stats + 3, (unsigned long long)nc.fails);
                atomicOr(P.err, ERR_NEWTON);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, g[i]);
    return (nonfinite ? 1 : 0) | (pending ? 2 : 0);
}

// ---------------------------------------------------------------------------
// Vector loads and stores of VEC consecutive populations (aligned).
// ---------------------------------------------------------------------------
template <typename S, int VEC> struct VecIO;
template <typename S> struct VecIO<S, 1> {
    __device__ static void load(const void* p, long long i, typename Store<S>::T* v) {
        v[0] = Store<S>::load(p, i);
    }
    __device__ static void store(void* p, long long i, const typename Store<S>::T* v) {
        Store<S>::store(p, i, v[0]);
    }
};
template <> struct VecIO<float, 4> {
    __device__ static void load(const void* p, long long i, float* v) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + i));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ static void store(void* p, long long i, const float* v) {
        *reinterpret_cast<float4*>(static_cast<float*>(p) + i) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct VecIO<float, 2> {
    __device__ static void load(const void* p, long long i, float* v) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(p) + i));
        v[0] = a.x; v[1] = a.y;
    }
    __device__ static void store(void* p, long long i, const float* v) {
        *reinterpret_cast<float2*>(static_cast<float*>(p) + i) = make_float2(v[0], v[1]);
    }
};
template <> struct VecIO<double, 4> {
    __device__ static void load(const void* p, long long i, double* v) {
        const double2* q = reinterpret_cast<const double2*>(static_cast<const double*>(p) + i);
        const double2 a = __ldg(q), b = __ldg(q + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void store(void* p, long long i, const double* v) {
        double2* q = reinterpret_cast<double2*>(static_cast<double*>(p) + i);
        q[0] = make_double2(v[0], v[1]);
        q[1] = make_double2(v[2], v[3]);
    }
};
template <> struct VecIO<double, 2> {
    __device__ static void load(const void* p, long long i, double* v) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(static_cast<const double*>(p) + i));
        v[0] = a.x; v[1] = a.y;
    }
    __device__ static void store(void* p, long long i, const double* v) {
        *reinterpret_cast<double2*>(static_cast<double*>(p) + i) = make_double2(v[0], v[1]);
    }
};
template <> struct VecIO<__half, 4> {
    __device__ static void load(const void* p, long long i, float* v) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(static_cast<const __half*>(p) + i));
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
        v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
    }
    __device__ static void store(void* p, long long i, const float* v) {
        __half2 lo = __floats2half2_rn(v[0], v[1]);
        __half2 hi = __floats2half2_rn(v[2], v[3]);
        uint2 a;
        a.x = *reinterpret_cast<unsigned*>(&lo);
        a.y = *reinterpret_cast<unsigned*>(&hi);
        *reinterpret_cast<uint2*>(static_cast<__half*>(p) + i) = a;
    }
};
template <> struct VecIO<__half, 2> {
    __device__ static void load(const void* p, long long i, float* v) {
        const unsigned a = __ldg(reinterpret_cast<const unsigned*>(static_cast<const __half*>(p) + i));
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&a));
        v[0] = f.x; v[1] = f.y;
    }
    __device__ static void store(void* p, long long i, const float* v) {
        __half2 h = __floats2half2_rn(v[0], v[1]);
        *reinterpret_cast<unsigned*>(static_cast<__half*>(p) + i) = *reinterpret_cast<unsigned*>(&h);
    }
};

template <> struct VecIO<plain32, 4> {
    __device__ static void load(const void* p, long long i, float* v) { VecIO<float, 4>::load(p, i, v); }
    __device__ static void store(void* p, long long i, const float* v) { VecIO<float, 4>::store(p, i, v); }
};
template <> struct VecIO<plain32, 2> {
    __device__ static void load(const void* p, long long i, float* v) { VecIO<float, 2>::load(p, i, v); }
    __device__ static void store(void* p, long long i, const float* v) { VecIO<float, 2>::store(p, i, v); }
};

// Two adjacent populations (columns c, c + 1 with c even: 8-byte aligned
// for FP32, 4-byte for FP16, 16-byte for FP64) of a staged plane row or of
// a population plane, loaded or stored with one access.
template <typename S> struct PairIO;
template <> struct PairIO<float> {
    __device__ static void load(const float* p, float& a, float& b) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static void store(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
};
template <> struct PairIO<plain32> {
    __device__ static void load(const plain32* p, float& a, float& b) {
        PairIO<float>::load(reinterpret_cast<const float*>(p), a, b);
    }
    __device__ static void store(plain32* p, float a, float b) {
        PairIO<float>::store(reinterpret_cast<float*>(p), a, b);
    }
};
template <> struct PairIO<__half> {
    __device__ static void load(const __half* p, float& a, float& b) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
        a = v.x;
        b = v.y;
    }
    __device__ static void store(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct PairIO<double> {
    __device__ static void load(const double* p, double& a, double& b) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static void store(double* p, double a, double b) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
};

// Interior-path accessors with 32-bit element indices (every population
// array holds fewer than 2^31 elements; checked at creation).
template <typename S, int VEC>
__device__ __forceinline__ void load_vec(const S* __restrict__ p, int i, typename Store<S>::T* v) {
    VecIO<S, VEC>::load(p + i, 0, v);
}
template <typename S, int VEC>
__device__ __forceinline__ void store_vec(S* __restrict__ p, int i, const typename Store<S>::T* v) {
    VecIO<S, VEC>::store(p + i, 0, v);
}

// A row tile [x0, x0 + TX) of row y is interior when the tile and its
// one-site halo are fluid and inside the grid: its gather is a pure shift.
template <int TX>
__device__ __forceinline__ bool tile_interior(const Params& P, int x0, int y) {
    if (x0 < 1 || x0 + TX > P.nx - 1 || y < 1 || y > P.ny - 2) return false;
    if (P.ow > 0) {
        const bool apart = (x0 + TX + 1 <= P.ox0) || (x0 - 1 >= P.ox0 + P.ow) ||
                           (y + 2 <= P.oy0) || (y - 1 >= P.oy0 + P.oh);
        if (!apart) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// K1 for D2Q9, persistent: the grid holds as many blocks as fit on the
// GPU at once; each block processes a contiguous range of row tiles of
// 32 x VEC consecutive sites, its warps taking the range's tiles in turn.
// Interior tiles: aligned VEC-wide loads per population plane, the
// x-shifted planes completed by one warp shuffle and one halo load.
// Boundary tiles (and the first step after a state upload): per-site gather
// with the boundary rules.
// ---------------------------------------------------------------------------
template <typename S, int EQ, int VEC, int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_collide_d2q9(const __grid_constant__ Params P) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    constexpr int TX = 32 * VEC;
    __shared__ FinishShared fs;
    __shared__ MlpSlot<EQ> mslot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        fs.npend = 0;
        fs.bc.n = 0;
    }
    mslot.fill(P);
    __syncthreads();
    const long long t = *P.step;
    const S* __restrict__ src = static_cast<const S*>(P.src);
    S* __restrict__ dst = static_cast<S*>(P.dst);
    const int nxp = P.nxp, plane = (int)P.plane;
    // Each block owns a contiguous range of row tiles (row-major); its warps
    // take the range's tiles in turn.  Boundary tiles, which cost more, are
    // then spread evenly over blocks.
    const int tiles_x = (P.nx + TX - 1) / TX;
    const int tiles = tiles_x * P.ny;
    const int per_block = (tiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per_block;
    const int t1 = min(t0 + per_block, tiles);
    bool nonfinite = false;
    NewtonCount nc = {0, 0, 0, 0};
    unsigned wpend = 0u;   // pending sites this warp appended since the last drain
    // one row tile of 32 * VEC sites: row y, tile column xt
    auto do_tile = [&](int y, int xt) {
        const int x0 = xt * TX;
        const int xs = x0 + lane * VEC;
        if (!P.prestream && tile_interior<TX>(P, x0, y)) {
            const int row = y * nxp + xs;
            T g[VEC][L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                const int at = i * plane + row - L::cy(i) * nxp;
                T v[VEC];
                load_vec<S, VEC>(src, at, v);
                if (L::cx(i) == 0) {
#pragma unroll
                    for (int s = 0; s < VEC; s++) g[s][i] = v[s];
                } else if (L::cx(i) == 1) {
                    // source x - 1: the previous lane's last element
                    T prev = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
                    if (lane == 0) prev = Store<S>::load(src + at - 1, 0);
                    g[0][i] = prev;
#pragma unroll
                    for (int s = 1; s < VEC; s++) g[s][i] = v[s - 1];
                } else {
                    // source x + 1: the next lane's first element
                    T next = __shfl_down_sync(0xffffffffu, v[0], 1);
                    if (lane == 31) next = Store<S>::load(src + at + VEC, 0);
#pragma unroll
                    for (int s = 0; s < VEC - 1; s++) g[s][i] = v[s + 1];
                    g[VEC - 1][i] = next;
                }
            }
            bool pend[VEC];
#pragma unroll
            for (int s = 0; s < VEC; s++) {
                if constexpr (EQ == EQ_ENERGY_MLP) {
                    // interior tile: every lane holds a fluid site
                    float a0[3];
                    mlp_site_start<T>(P, mslot.s, true, g[s], a0);
                    pend[s] = update_site<L, T, EQ, Store<S>::kProject>(P, g[s], xs + s, y, t, nonfinite,
                                                                         nc, a0);
                } else {
                    pend[s] = update_site<L, T, EQ, Store<S>::kProject>(P, g[s], xs + s, y, t, nonfinite,
                                                                         nc);
                }
            }
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                T v[VEC];
#pragma unroll
                for (int s = 0; s < VEC; s++) v[s] = store_round<L, S>(i, g[s][i]);
                store_vec<S, VEC>(dst, i * plane + row, v);
            }
#pragma unroll
            for (int s = 0; s < VEC; s++) wpend += warp_pend(P, fs, pend[s], (unsigned)(y * P.nx + xs + s));
        } else {
#pragma unroll 1
            for (int s = 0; s < VEC; s++) {
                const int x = xs + s;
                int r = 0;
                if (x < P.nx) r = boundary_site<S, EQ>(P, x, y, t);
                nonfinite |= (r & 1) != 0;
                wpend += warp_pend(P, fs, (r & 2) != 0, (unsigned)(y * P.nx + x));
            }
        }
    };
    if constexpr (EQ < EQ_ENERGY) {
        int w = t0 + warp;
        int y = w / tiles_x, xt = w - y * tiles_x;
        for (; w < t1; w += WARPS) {
            do_tile(y, xt);
            xt += WARPS;
            while (xt >= tiles_x) { xt -= tiles_x; y++; }
        }
    } else {
        // The energy forms go in rounds of one tile per warp and resolve the
        // block's pending sites before its list could overflow in the next
        // round: a start far from equilibrium then cannot overflow many sites
        // to the global list, which the last block alone resolves.  The
        // block drains once some warp appended more than its share (1 /
        // WARPS) of the room left for a round; one vote over the warps' own
        // counts decides, so every warp takes the same branch.
        static_assert(kPend > TX * WARPS, "a round must fit in the pending list");
        constexpr unsigned kShare = (unsigned)((kPend - TX * WARPS) / WARPS);
        const int rounds = t1 > t0 ? (t1 - t0 + WARPS - 1) / WARPS : 0;
        for (int r = 0; r < rounds; r++) {
            const int w = t0 + r * WARPS + warp;
            if (w < t1) {
                const int y = w / tiles_x;
                do_tile(y, w - y * tiles_x);
            }
            if (__syncthreads_or(wpend > kShare)) {
                resolve_list<L, S, EQ>(P, (int)min(fs.npend, (unsigned)kPend),
                                       [&](int j) { return fs.pend[j]; }, &fs.bc, &fs.ss.sc);
                __syncthreads();
                if (threadIdx.x == 0) fs.npend = 0;
                __syncthreads();
                wpend = 0u;
            }
        }
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if constexpr (EQ >= EQ_ENERGY) flush_newton(P, nc);
    finish_block<L, S, EQ>(P, fs);
}

// ---------------------------------------------------------------------------
// K1 for D2Q9 with tiles staged in shared memory by the tensor memory
// accelerator.  A block tile is R rows x 128 sites.  Population i at row y
// comes from row y - v_iy of the source field, so for each of the 9 planes
// one 3-D bulk tensor copy brings exactly the R rows y0 - v_iy ..
// y0 - v_iy + R - 1 the tile pulls from that plane, over columns x0 - H ..
// x0 + 128 + H (H elements = 16 bytes on each side, which keeps every copy
// 16-byte aligned).  Copies complete on an mbarrier; STAGES tiles are in
// flight per block, so the bytes in flight do not depend on registers.
// Warp w computes row w of the tile, lane l the site pairs x0 + 2 l + 64 s,
// + 1: shared-memory reads and global stores are both consecutive across the
// warp.  In tiles that touch the y sides or the obstacle the sites use the
// rule-by-rule gather, from shared memory where the source lies in its
// plane's window and from the source field otherwise; the x = 0 and
// x = nx - 1 columns are edge items of their own.  Every wait on an
// mbarrier is bounded: on expiry the block flags ERR_TIMEOUT, stops issuing
// copies, waits (bounded) for the copies it issued, and ends.
// ---------------------------------------------------------------------------
constexpr int kTmaTX = 128;
constexpr long long kWaitLimit = 1ll << 22;   // try_wait polls before a wait is declared failed

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the limit expired
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (long long it = 0; it < kWaitLimit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

template <typename S, int R, int TX = kTmaTX>
struct TmaLayout {
    static constexpr int H = 16 / (int)sizeof(S);          // halo columns (16 bytes)
    static constexpr int W = TX + 2 * H;                   // staged row length
    static constexpr int ROWS = R;                         // plane i: rows y0 - v_iy .. y0 - v_iy + R - 1
    static constexpr int BOX_BYTES = ROWS * W * (int)sizeof(S);
    static constexpr int PLANE_BYTES = (BOX_BYTES + 127) / 128 * 128;   // 128-byte aligned boxes
    static constexpr int PLANE = PLANE_BYTES / (int)sizeof(S);
    static constexpr int STAGE_BYTES = 9 * PLANE_BYTES;
    static constexpr int TX_BYTES = 9 * BOX_BYTES;         // bytes one tile's copies deliver
};

// Candidate buffer of a staged block: room for one tile's sites above what
// a cut keeps (the block cuts between tiles).
template <int R, int TX>
constexpr int tma_cand_cap() {
    return TX * R + kBlockCand;
}

// Shared state of a staged block besides its tiles.  p: the launch's
// parameters, for the out-of-line paths (a reference to the kernel's
// __grid_constant__ parameter passed to a function that is not inlined
// reads it through generic loads of the parameter space; the shared copy
// answers at shared-memory latency).
template <int CAP>
struct TmaShared {
    Params p;
    SelectShared ss;
    BlockCandT<CAP> bc;
    int is_last;
    int abort;
    int tile[8];   // tile held by each stage (-1: none left)
};

template <typename S, int R, int STAGES, int EQ, int TX = kTmaTX>
constexpr size_t tma_smem_bytes() {
    return 128 + (size_t)STAGES * TmaLayout<S, R, TX>::STAGE_BYTES + 8 * STAGES +
           sizeof(TmaShared<tma_cand_cap<R, TX>()>) + 16 +
           (EQ == EQ_ENERGY_MLP ? sizeof(MlpSlot<EQ>) + 16 : 0);
}

// Where a staged tile's candidates go (put: every lane of the warp calls,
// with its site's dS, -1 for a site the dS bound cleared; the sites the
// bound does not clear have their exact dS evaluated on the tile, from the
// staged planes or in the update).  CandSink: the block's buffer; count is
// what the warp appended since the block's last cut (the same on every
// lane).  GlobalCandSink: the run's global list (a kernel whose tiles belong
// to different runs).
template <int CAP>
struct CandSink {
    BlockCandT<CAP>* bc;
    unsigned count;
    template <typename T>
    __device__ __forceinline__ void put(const Params& P, T ds, unsigned site) {
        count += block_push<T>(P, *bc, ds > Par<T>::delta(P), ds, site);
    }
};
struct GlobalCandSink {
    template <typename T>
    __device__ __forceinline__ void put(const Params& P, T ds, unsigned site) {
        warp_push<T>(P, ds > Par<T>::delta(P), ds, site);
    }
};

// Pre-collision deviations of site (x, y) of a staged tile: the same rules
// as gather_site (free flight, Sec. 4.2 boundaries).  Plane j's window holds
// source rows y0 - v_jy .. y0 - v_jy + R - 1 (box[j][row][col] with
// row = sy - y0 + v_jy, col = sx - x0 + H); a rule that reads a plane
// outside its window (a bounce-back or a mirror at the tile's edge rows, the
// outlet column) reads the source field instead.  Not used with periodic
// sides.
template <typename S, int R, int TX = kTmaTX>
__device__ __forceinline__ void gather_site_smem(const Params& P, const S* box, int x0, int y0, int x,
                                                 int y, typename Store<S>::T* g) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    using LY = TmaLayout<S, R, TX>;
    auto at = [&](int j, int sx, int sy) {
        const int r = sy - y0 + L::cy(j), c = sx - x0 + LY::H;
        if ((unsigned)r < (unsigned)R && (unsigned)c < (unsigned)LY::W)
            return Store<S>::load(box + j * LY::PLANE + r * LY::W + c, 0);
        return Store<S>::load(P.src, j * P.plane + (long long)sy * P.nxp + sx);
    };
    if (P.prestream) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) g[i] = at(i, x, y);
        return;
    }
    bool have_in = false, have_out = false;
    unsigned wall_mask = 0u;
    T gin[L::Q], gout[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const int cx = L::cx(i), cy = L::cy(i);
        int sx = x - cx;
        const int sy = y - cy;
        if (sx < 0 || sx >= P.nx) {
            const int kind = sx < 0 ? P.bc[0] : P.bc[1];
            if (kind == BC_OUTLET_COPY) {
                sx = x;   // the column beyond the side is a copy of the side column
            } else if (kind == BC_INLET) {
                if (!have_in) {
                    inlet_equilibrium<L, T>(P, gin);
                    have_in = true;
                }
                g[i] = gin[i];
            } else if (kind == BC_OUTLET) {
                if (!have_out) {
                    T v[L::Q];
#pragma unroll
                    for (int j = 0; j < L::Q; j++) v[j] = at(j, P.nx - 2, y);
                    outlet_equilibrium<L, T>(P, v, gout);
#pragma unroll
                    for (int j = 0; j < L::Q; j++) gout[j] = store_round<L, S>(j, gout[j]);
                    have_out = true;
                }
                g[i] = gout[i];
            } else {
                g[i] = at(L::opp(i), x, y);
            }
            if (kind != BC_OUTLET_COPY) continue;
        }
        if (sy < 0 || sy >= P.ny) {
            const int kind = sy < 0 ? P.bc[2] : P.bc[3];
            g[i] = kind == BC_FREESLIP ? at(L::mir_y(i), sx, y) : at(L::opp(i), x, y);
            continue;
        }
        if (is_solid(P, sx, sy)) {
            g[i] = at(L::opp(i), x, y);
            if (P.wall == WALL_DIFFUSE) wall_mask |= 1u << i;
        } else {
            g[i] = at(i, sx, sy);
        }
    }
    if (wall_mask) diffuse_wall<L, T>(wall_mask, g);
}

// The sites of a staged tile that touches a boundary, the obstacle or the
// probe site, one by one with the boundary rules (kept out of line so that
// the interior path is allocated registers on its own).
template <typename S, int EQ, int R, int TX, bool SPLIT, typename Sink>
__device__ __noinline__ void tma_tile_general(const Params& P, const S* box, int x0, int y0, long long t,
                                              Sink& sink, MlpSlot<EQ>& mslot,
                                              bool& nonfinite, NewtonCount& nc, bool clean) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    using LY = TmaLayout<S, R, TX>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S* __restrict__ dst = static_cast<S*>(P.dst);
    const int nxp = P.nxp, plane = (int)P.plane;
    const bool periodic = P.bc[0] == BC_PERIODIC || P.bc[2] == BC_PERIODIC;
    const int y = y0 + warp;
    const S* sb = box + warp * LY::W + LY::H;
#pragma unroll 1
    for (int s = 0; s < TX / 32; s++) {
        const int x = x0 + lane + 32 * s;
        T ds = T(-1);
        // the learned form enters with every lane (its warm start is a
        // warp-wide evaluation); lanes outside the grid then carry no site
        // SPLIT: the columns x = 0 and x = nx - 1 are updated apart (edge_item)
        const bool mine = x < P.nx && y < P.ny && !(SPLIT && (x == 0 || x == P.nx - 1));
        if (EQ == EQ_ENERGY_MLP || mine) {
            const bool inside = mine;
            const int c = x - x0;
            const int o = y * nxp + x;
            bool shift = clean;
            if (!shift) {
                const bool near_obstacle = P.ow > 0 && x >= P.ox0 - 1 && x <= P.ox0 + P.ow &&
                                           y >= P.oy0 - 1 && y <= P.oy0 + P.oh;
                shift = !P.prestream && x >= 1 && x <= P.nx - 2 && y >= 1 && y <= P.ny - 2 &&
                        !near_obstacle;
            }
            T g[L::Q];
            bool fluid = inside;
            if (!inside) {
#pragma unroll
                for (int i = 0; i < L::Q; i++) g[i] = T(0);
            } else if (shift) {
#pragma unroll
                for (int i = 0; i < L::Q; i++) g[i] = Store<S>::load(sb + i * LY::PLANE + c - L::cx(i), 0);
            } else if (is_solid(P, x, y)) {
                fluid = false;
#pragma unroll
                for (int i = 0; i < L::Q; i++) g[i] = T(0);
            } else if (periodic) {
                gather_site<L, S>(P, x, y, g);
            } else {
                gather_site_smem<S, R, TX>(P, box, x0, y0, x, y, g);
            }
            if constexpr (EQ == EQ_ENERGY_MLP) {
                float a0[3];
                __syncwarp();
                mlp_site_start<T>(P, mslot.s, fluid, g, a0);
                if (fluid)
                    update_site<L, T, EQ, Store<S>::kProject, true, true>(P, g, x, y, t, nonfinite, nc, a0, &ds);
            } else {
                if (fluid)
                    update_site<L, T, EQ, Store<S>::kProject, true, true>(P, g, x, y, t, nonfinite, nc, nullptr,
                                                                          &ds);
            }
            if (inside) {
#pragma unroll
                for (int i = 0; i < L::Q; i++)
                    Store<S>::store(dst + i * plane + o, 0, fluid ? store_round<L, S>(i, g[i]) : g[i]);
            }
        }
        sink.put(P, ds, (unsigned)(y * P.nx + x));
    }
}


// The columns x = 0 and x = nx - 1 of the grid (the sites whose sources
// leave the grid in x), apart from the staged tiles: edge item e covers
// sites e * 32 R .. (e + 1) * 32 R - 1 of the list x = 0 (rows 0 .. ny - 1)
// then x = nx - 1, one site per lane, gathered from the source field with
// the boundary rules (gather_site).  Every lane of the block calls.
template <typename S, int EQ, int R, typename Sink>
__device__ __noinline__ void edge_item(const Params& P, int item, long long t, Sink& sink, MlpSlot<EQ>& mslot,
                                       bool& nonfinite, NewtonCount& nc) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncols = P.nx > 1 ? 2 : 1;
    const int e = (item * R + warp) * 32 + lane;
    const bool inside = e < ncols * P.ny;
    const int x = inside && e >= P.ny ? P.nx - 1 : 0;
    const int y = inside ? (e >= P.ny ? e - P.ny : e) : 0;
    const bool fluid = inside && !is_solid(P, x, y);
    T g[L::Q];
    if (fluid) {
        gather_site<L, S>(P, x, y, g);
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; i++) g[i] = T(0);
    }
    T ds = T(-1);
    if constexpr (EQ == EQ_ENERGY_MLP) {
        float a0[3];
        mlp_site_start<T>(P, mslot.s, fluid, g, a0);
        if (fluid) update_site<L, T, EQ, Store<S>::kProject, true, true>(P, g, x, y, t, nonfinite, nc, a0, &ds);
    } else {
        if (fluid)
            update_site<L, T, EQ, Store<S>::kProject, true, true>(P, g, x, y, t, nonfinite, nc, nullptr, &ds);
    }
    if (inside) {
        S* dst = static_cast<S*>(P.dst);
        const long long o = (long long)y * P.nxp + x;
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            Store<S>::store(dst, i * P.plane + o, fluid ? store_round<L, S>(i, g[i]) : g[i]);
    }
    sink.put(P, ds, (unsigned)(y * P.nx + x));
}

// Exact dS of the pending sites of a clean staged row (warp w: row y; lane
// l: bit 2 s + h of pmask for column x0 + 2 l + 64 s + h), from the staged
// planes (the same values the update read) and f* recomputed as the update
// computed it; the sites go to the sink (which keeps the candidates).  Every
// lane of the warp calls.
template <typename S, int EQ, int R, int TX, typename Sink>
__device__ __noinline__ void resolve_staged_row(const Params& P, const S* box, int x0, int y, unsigned pmask,
                                                Sink& sink) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    using LY = TmaLayout<S, R, TX>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S* sb = box + warp * LY::W + LY::H;
#pragma unroll 1
    for (int b = 0; b < TX / 32; b++) {
        const int c = 2 * lane + 64 * (b >> 1) + (b & 1);
        T ds = T(-1);
        if ((pmask >> b) & 1u) {
            T g[L::Q], gs[L::Q], rho, ux, uy;
#pragma unroll
            for (int i = 0; i < L::Q; i++) g[i] = Store<S>::load(sb + i * LY::PLANE + c - L::cx(i), 0);
            site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
            if (!ghost_column(P, x0 + c)) ds = site_ds<L, T, EQ>(P, g, gs);
        }
        sink.put(P, ds, (unsigned)(y * P.nx + x0 + c));
    }
}

// One staged tile: rows y0 .. y0 + R - 1 and columns x0 .. x0 + 127 of the
// run P, from box (the tile's staged source planes); warp w computes row
// y0 + w, lane l the sites x0 + l + 32 s.  The updated sites go to sink.
// Pc: the parameters for the out-of-line rule-by-rule path (the same values
// as P, held where that path reads them fast).
// SPLIT: the columns x = 0 and x = nx - 1 are not updated here (edge_item
// updates them); a tile then takes the interior path whenever it spans TX
// columns of the grid and its rows and columns stay away from the y sides
// and the obstacle.
template <typename S, int EQ, int R, int TX = kTmaTX, bool SPLIT = false, typename Sink>
__device__ __forceinline__ void tma_tile(const Params& P, const S* box, int x0, int y0, long long t, Sink& sink,
                                         MlpSlot<EQ>& mslot, bool& nonfinite, NewtonCount& nc,
                                         const Params& Pc) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    using LY = TmaLayout<S, R, TX>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S* __restrict__ dst = static_cast<S*>(P.dst);
    const int nxp = P.nxp, plane = (int)P.plane;
    const int y = y0 + warp;
    const bool xin = SPLIT ? x0 + TX <= P.nx : x0 >= 1 && x0 + TX <= P.nx - 1;
    const bool clean = !P.prestream && xin && y0 >= 1 && y0 + R <= P.ny - 1 &&
                       (P.ow == 0 || x0 + TX + 1 <= P.ox0 || x0 - 1 >= P.ox0 + P.ow ||
                        y0 + R + 1 <= P.oy0 || y0 - 1 >= P.oy0 + P.oh);
    const S* sb = box + warp * LY::W + LY::H;
    // Interior tile without the probe site (almost every tile): every site is
    // fluid and away from every boundary rule, so the sites take the shifted
    // shared-memory reads with no per-site checks (the branch is uniform).
    const bool probe_here = P.probe_ring && P.probe_y >= y0 && P.probe_y < y0 + R &&
                            P.probe_x >= x0 && P.probe_x < x0 + TX;
    if (clean && !probe_here) {
        const int row = y * nxp + x0;
        unsigned pmask = 0u;   // pending sites of the lane (bit 2 s + h: column 2 l + 64 s + h)
        const bool edge_tile = SPLIT && (x0 == 0 || x0 + TX >= P.nx - 1);
        // two adjacent sites per lane, columns c and c + 1 (c = 2 l + 64 s):
        // planes at rest and every store move both with one access, and the
        // two updates are independent work for the scheduler
#pragma unroll 1
        for (int s = 0; s < TX / 64; s++) {
            const int c = 2 * lane + 64 * s;
            T ga[L::Q], gb[L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                const S* q = sb + i * LY::PLANE + c;
                if (L::cx(i) == 0) {
                    PairIO<S>::load(q, ga[i], gb[i]);
                } else {
                    ga[i] = Store<S>::load(q - L::cx(i), 0);
                    gb[i] = Store<S>::load(q + 1 - L::cx(i), 0);
                }
            }
            // SPLIT: a site of column 0 or nx - 1 (lane 0 or 31 of an edge
            // tile) is left to edge_item; it is updated here from the rest
            // state at unit density (whatever the staged halo holds) and is
            // neither stored nor pending
            bool ea = false, eb = false;
            if constexpr (SPLIT) {
                if (edge_tile) {   // uniform: only the tiles at either end of the rows
                    ea = x0 + c == 0 || x0 + c == P.nx - 1;
                    eb = x0 + c + 1 == P.nx - 1;
                    const T r1 = T(1) - Par<T>::rho0(P);
#pragma unroll
                    for (int i = 0; i < L::Q; i++) {
                        ga[i] = ea ? T(L::w(i)) * r1 : ga[i];
                        gb[i] = eb ? T(L::w(i)) * r1 : gb[i];
                    }
                }
            }
            bool pa, pb;
            if constexpr (EQ == EQ_ENERGY_MLP) {
                float a0[3];
                mlp_site_start<T>(P, mslot.s, true, ga, a0);
                pa = update_site<L, T, EQ, Store<S>::kProject, false>(P, ga, x0 + c, y, t, nonfinite, nc, a0);
                mlp_site_start<T>(P, mslot.s, true, gb, a0);
                pb = update_site<L, T, EQ, Store<S>::kProject, false>(P, gb, x0 + c + 1, y, t, nonfinite, nc, a0);
            } else {
                pa = update_site<L, T, EQ, Store<S>::kProject, false>(P, ga, x0 + c, y, t, nonfinite, nc);
                pb = update_site<L, T, EQ, Store<S>::kProject, false>(P, gb, x0 + c + 1, y, t, nonfinite, nc);
            }
            if (!(ea | eb)) {
#pragma unroll
                for (int i = 0; i < L::Q; i++)
                    PairIO<S>::store(dst + i * plane + row + c, store_round<L, S>(i, ga[i]),
                                     store_round<L, S>(i, gb[i]));
            } else {
#pragma unroll
                for (int i = 0; i < L::Q; i++) {
                    if (!ea) Store<S>::store(dst + i * plane + row + c, 0, store_round<L, S>(i, ga[i]));
                    if (!eb) Store<S>::store(dst + i * plane + row + c + 1, 0, store_round<L, S>(i, gb[i]));
                }
            }
            pa = pa && !ea;
            pb = pb && !eb;
            pmask |= ((pa ? 1u : 0u) | (pb ? 2u : 0u)) << (2 * s);
        }
        // the row's pending sites, from the staged planes (valid until the
        // next tile's barrier), out of line: the update keeps its registers
        if (__any_sync(0xffffffffu, pmask != 0u)) resolve_staged_row<S, EQ, R, TX>(Pc, box, x0, y, pmask, sink);
        return;
    }
    tma_tile_general<S, EQ, R, TX, SPLIT>(Pc, box, x0, y0, t, sink, mslot, nonfinite, nc, clean);
}
// Resident blocks per SM the staged kernel is compiled for: two in general
// (128 registers per thread with 8-row tiles, 170 with 6-row tiles); three
// (85 registers per thread) where the tiles take half the shared memory:
// FP16 storage, or FP32 tiles 64 sites wide.
template <typename S, int R, int TX>
constexpr int tma_min_blocks() {
    return (sizeof(S) == 2 && R == 8) || (sizeof(S) == 4 && TX == 64 && R == 8) ? 3 : 2;
}

template <typename S, int EQ, int R, int STAGES, int TX = kTmaTX>
__global__ void __launch_bounds__(32 * R, tma_min_blocks<S, R, TX>())
    k_collide_d2q9_tma(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    using LY = TmaLayout<S, R, TX>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    S* stages = reinterpret_cast<S*>(smem);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + STAGES * LY::STAGE_BYTES);
    constexpr int kCap = tma_cand_cap<R, TX>();
    constexpr int kRoom = kCap - TX * R;   // what the buffer holds at the top of a tile
    using Shared = TmaShared<kCap>;
    Shared& sh = *reinterpret_cast<Shared*>(smem + STAGES * LY::STAGE_BYTES + 8 * STAGES);
    constexpr size_t kMlpOff = (STAGES * LY::STAGE_BYTES + 8 * STAGES + sizeof(Shared) + 15) / 16 * 16;
    MlpSlot<EQ>& mslot = *reinterpret_cast<MlpSlot<EQ>*>(smem + kMlpOff);
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; st++) mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.p = P;
        sh.abort = 0;
        sh.bc.n = 0;
    }
    // Launched as a programmatic dependent of the previous kernel in the
    // stream: the block may start while that kernel finishes, and the code
    // above reads only the launch's parameters and writes only shared
    // memory.  Every thread waits here until the previous kernel has
    // completed and its writes are visible, then lets the next kernel of the
    // stream start its blocks as this one's leave the SMs (they wait here in
    // turn).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    mslot.fill(P);
    __syncthreads();
    const long long t = *P.step;
    const int tiles_x = (P.nx + TX - 1) / TX;
    const int tiles = tiles_x * ((P.ny + R - 1) / R);
    // the x = 0 and x = nx - 1 columns go first, as edge items of 32 R sites
    const int edge_items = ((P.nx > 1 ? 2 : 1) * P.ny + 32 * R - 1) / (32 * R);
    const int claims = edge_items + tiles;

    // Work is handed out by claims: claim c < edge_items is edge item c, the
    // others tile tile_order[c - edge_items] (boundary tiles spread over the
    // first claims) or c - edge_items.  Thread 0 refills a
    // stage with the work it claimed at the previous refill and claims the
    // next (the latencies of the atomic and of the order entry then overlap
    // a tile's computation), and publishes it with the stage's mbarrier:
    // the tile's index, -2 - e for edge item e, -1 when none is left (the
    // phase is then completed by a plain arrive, without a copy, as for an
    // edge item).
    // A block's first STAGES claims are fixed (b, b + G, b + 2 G, ... for
    // block b of G): the pipeline fills without waiting for the atomic; the
    // counter hands out the claims from STAGES G on.
    int next_claim = 0, next_tile = 0, fixed = 0;
    auto claim = [&]() {
        if (fixed < STAGES) next_claim = (int)blockIdx.x + fixed++ * (int)gridDim.x;
        else next_claim = (int)atomicAdd(P.tile_counter, 1u) + STAGES * (int)gridDim.x;
        const int c = next_claim - edge_items;
        next_tile = c < 0 ? -2 - next_claim : c;
        if (P.tile_order && c >= 0 && c < tiles) next_tile = __ldg(P.tile_order + c);
    };
    auto fill = [&](int st) {
        unsigned long long* bar = &full[st];
        if (next_claim >= claims || next_tile < 0) {
            sh.tile[st] = next_claim >= claims ? -1 : next_tile;
            if (next_claim < claims) claim();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
            return;
        }
        const int tile = next_tile;
        claim();
        sh.tile[st] = tile;
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        mbar_expect_tx(bar, (unsigned)LY::TX_BYTES);
        S* base = stages + (size_t)st * (LY::STAGE_BYTES / sizeof(S));
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            tma_load_3d(base + i * LY::PLANE, &tm, tx * TX - LY::H, ty * R - L::cy(i), i, bar);
    };
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tm))
                     : "memory");
        claim();
        for (int st = 0; st < STAGES - 1; st++) fill(st);
    }
    bool nonfinite = false;
    NewtonCount nc = {0, 0, 0, 0};
    // The sites the dS bound does not clear are resolved as they are
    // updated; the candidates go to the block's buffer, which the block cuts
    // to its k best between tiles.  A cut happens once some warp appended
    // more than its share (1 / R) of the room above what a cut keeps: the
    // buffer then never holds more than kRoom entries at the top of a tile,
    // and one tile adds at most TX * R.
    const int kept = P.k > 0 && P.k < kRoom ? P.k : 0;
    const unsigned share = (unsigned)((kRoom - kept) / R);
    CandSink<kCap> sink{&sh.bc, 0u};
    int jj = 0;
    for (;; jj++) {
        const int st = jj % STAGES;
        const unsigned parity = (unsigned)((jj / STAGES) & 1);
        // every thread waits.  One vote decides, for every warp at once, to
        // stop (a wait that gave up anywhere: abort is written before the
        // barrier only) or to cut the candidates (a warp's count is its own),
        // so that the barriers stay matched
        const bool ok = mbar_wait(&full[st], parity);
        if (!ok) sh.abort = 1;
        if (__syncthreads_or(!ok || sink.count > share)) {
            if (sh.abort) {
                if (threadIdx.x == 0) atomicOr(P.err, ERR_TIMEOUT);
                break;
            }
            if (P.k < kRoom) block_cut(sh.bc, sh.ss.sc, P.k);
            else block_flush(sh.p, sh.bc);
            sink.count = 0;
        }
        const int tile = sh.tile[st];
        if (tile == -1) break;
        if (threadIdx.x == 0) {
            // the stage being refilled was last read in iteration jj - 1,
            // whose reads the barrier at the top of this iteration ordered
            // before this point
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fill((jj + STAGES - 1) % STAGES);
        }
        if (tile <= -2) {
            edge_item<S, EQ, R>(sh.p, -2 - tile, t, sink, mslot, nonfinite, nc);
            continue;
        }
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const S* box = stages + (size_t)st * (LY::STAGE_BYTES / sizeof(S));
        tma_tile<S, EQ, R, TX, true>(P, box, tx * TX, ty * R, t, sink, mslot, nonfinite, nc, sh.p);
    }
    __syncthreads();
    if (sh.abort && threadIdx.x == 0) {
        // wait (bounded) for copies still in flight into every stage
        for (int k2 = 0; k2 < STAGES; k2++) {
            const int j2 = jj + k2;
            mbar_wait(&full[j2 % STAGES], (unsigned)((j2 / STAGES) & 1));
        }
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if constexpr (EQ >= EQ_ENERGY) flush_newton(P, nc);
    __syncthreads();
    // the staged tiles are no longer needed: their memory holds the last
    // block's candidate staging
    const int scap = (int)min((size_t)kStage, (size_t)STAGES * LY::STAGE_BYTES / 12);
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(smem);
    unsigned* sidx = reinterpret_cast<unsigned*>(smem + 8 * scap);
    finish_parts<L, S, EQ>(sh.p, nullptr, 0u, 0, sh.is_last, sh.ss, sh.bc, skey, sidx, scap);
}

// ---------------------------------------------------------------------------
// K1, one site per thread (D1Q3).
// ---------------------------------------------------------------------------
template <typename L, typename S, int EQ>
__global__ void __launch_bounds__(kSiteBlock) k_collide_site(const __grid_constant__ Params P) {
    using T = typename Store<S>::T;
    __shared__ FinishShared fs;
    if (threadIdx.x == 0) {
        fs.npend = 0;
        fs.bc.n = 0;
    }
    __syncthreads();
    const long long t = *P.step;
    const long long sid = (long long)blockIdx.x * kSiteBlock + threadIdx.x;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    const bool inside = sid < (long long)P.nx * P.ny;
    const bool valid = inside && !is_solid(P, x, y);
    bool nonfinite = false, pending = false;
    NewtonCount nc = {0, 0, 0, 0};
    T g[L::Q];
    if (valid) {
        gather_site<L, S>(P, x, y, g);
        pending = update_site<L, T, EQ, Store<S>::kProject>(P, g, x, y, t, nonfinite, nc);
    }
    if (inside) {
        const long long o = (long long)y * P.nxp + x;
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            Store<S>::store(P.dst, i * P.plane + o, valid ? store_round<L, S>(i, g[i]) : T(0));
    }
    warp_pend(P, fs, pending, (unsigned)sid);
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    finish_block<L, S, EQ>(P, fs);
}

// Stand-alone selection (select-only test hook).
template <typename L, typename S, int EQ>
__global__ void __launch_bounds__(kSelectThreads) k_select(const __grid_constant__ Params P, int stage_cap,
                                                           int mode) {
    extern __shared__ unsigned long long dyn[];
    __shared__ SelectShared ss;
    select_and_fix<L, S, EQ>(P, ss, dyn, reinterpret_cast<unsigned*>(dyn + stage_cap), stage_cap, mode);
}

#ifdef LBM_DEFINE_EMIT_FROM_DS
// Candidates from a given dS array (select-only test hook): each block of
// 256 threads takes kEmitPerBlock consecutive values through the same block
// stage as K1 (its k best reach the global list).
constexpr int kEmitPerBlock = 2048;
__global__ void __launch_bounds__(256) k_emit_from_ds(const __grid_constant__ Params P, const double* ds,
                                                      int n) {
    __shared__ BlockCand bc;
    __shared__ TopkScratch sc;
    if (threadIdx.x == 0) bc.n = 0;
    if (P.k <= 0) return;
    const long long b0 = (long long)blockIdx.x * kEmitPerBlock;
    for (int r = 0; r < kEmitPerBlock; r += 256) {
        block_room(P, bc, sc);
        const long long i = b0 + r + threadIdx.x;
        const double v = i < n ? ds[i] : -INFINITY;
        block_push<double>(P, bc, i < n && v > P.delta, v, (unsigned)i);
    }
    block_finish(P, bc, sc);
}
#endif

// ---------------------------------------------------------------------------
// State import / export and field kernels (one site per thread).
// ---------------------------------------------------------------------------

// Quasiequilibrium of given (rho, u) at every fluid site; zero elsewhere.
template <typename L, typename S, int EQ>
__global__ void k_init_eq(const __grid_constant__ Params P, const double* rho, const double* ux,
                          const double* uy, const double* e2) {
    using T = typename Store<S>::T;
    const long long sid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= (long long)P.nx * P.ny) return;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    const long long o = (long long)y * P.nxp + x;
    T gs[L::Q];
    if (is_solid(P, x, y)) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) gs[i] = T(0);
    } else {
        const double v = uy ? uy[sid] : 0.0;
        bool done = false;
        if constexpr (EQ >= EQ_ENERGY) {
            if (e2) {
                const T r = T(rho[sid]), u = T(ux[sid]);
                NewtonCount nc = {0, 0, 0, 0};
                equilibrium_energy<T, EQ>(P, r, r * u, r * T(v), T(e2[sid]), gs, nc);
#pragma unroll
                for (int i = 0; i < L::Q; i++) gs[i] = store_round<L, S>(i, gs[i]);
                done = true;
            }
        }
        // polynomial or entropic f* (the energy forms without a given energy:
        // the isothermal entropic formula) in FP64, held as the storage
        // holds it
        if (!done) bc_equilibrium<L, S>(P, rho[sid], ux[sid], v, gs);
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, gs[i]);
}

// FP64 populations [Q][ny][nx] -> deviation storage, planes [i0, i1).
template <typename L, typename S>
__global__ void k_import(const __grid_constant__ Params P, const double* f, int i0, int i1) {
    const long long N = (long long)P.nx * P.ny;
    const long long sid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= N) return;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    const long long o = (long long)y * P.nxp + x;
    const bool solid = is_solid(P, x, y);
    using T = typename Store<S>::T;
    if (P.rho0 == 0.0) {
        // FP64 storage: a copy (no FP64 arithmetic)
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            if (i >= i0 && i < i1) Store<S>::store(P.dst, i * P.plane + o, (T)(solid ? 0.0 : f[i * N + sid]));
        return;
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++)
        if (i >= i0 && i < i1)
            Store<S>::store(P.dst, i * P.plane + o, solid ? T(0) : dev_of_f64<L, S>(P, i, f[i * N + sid]));
}

// Pre-collision state of the current step (gather of src) at sites
// [s0, s1), exported as mode 0: populations f [Q][ny][nx]; 1: rho, ux, uy,
// 2E; 2: exact dS (outputs indexed by the site's index y nx + x).
template <typename L, typename S, int EQ>
__global__ void k_export(const __grid_constant__ Params P, int mode, double* o0, double* o1, double* o2,
                         double* o3, long long s0, long long s1) {
    using T = typename Store<S>::T;
    const long long N = (long long)P.nx * P.ny;
    const long long sid = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= s1) return;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    if (is_solid(P, x, y)) {
        if (mode == 0) for (int i = 0; i < L::Q; i++) o0[i * N + sid] = 0.0;
        if (mode == 1) {
            o0[sid] = 0.0;
            if (o1) o1[sid] = 0.0;
            if (o2) o2[sid] = 0.0;
            if (o3) o3[sid] = 0.0;
        }
        if (mode == 2) o0[sid] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    T g[L::Q];
    gather_site<L, S>(P, x, y, g);
    if (mode == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) o0[i * N + sid] = pop_f64<L, S>(P, i, g[i]);
    } else if (mode == 1) {
        if constexpr (sizeof(T) == 4) {
            // FP32 / FP16 storage: the sums of the stored values in float-float
            // (exact for these nine floats) and u = j / rho by one corrected
            // FP32 quotient, so that only the conversions to FP64 touch the FP64
            // pipe; the rho0 parts (sum W = 1, sum W v = 0, sum W |v|^2) are added
            // in FP64 at the end.
            ff r = {0.0f, 0.0f}, jx = {0.0f, 0.0f}, jy = {0.0f, 0.0f}, e = {0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                const ff gi = {g[i], 0.0f};
                r = ff_add(r, gi);
                if (L::cx(i) == 1) jx = ff_add(jx, gi);
                if (L::cx(i) == -1) jx = ff_sub(jx, gi);
                if (L::cy(i) == 1) jy = ff_add(jy, gi);
                if (L::cy(i) == -1) jy = ff_sub(jy, gi);
                const int c2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i);
                if (c2 > 0) e = ff_add(e, ff_scale(gi, (float)c2));
            }
            // the stored deviations' offsets: sum W rho0 (= rho0), and for
            // plain FP32 the sums of the FP32 weights (exact in FP64)
            double off0 = P.rho0, off2 = L::sum_w_c2 * P.rho0;
            if constexpr (Store<S>::kPlain) {
                off0 = 0.0;
                off2 = 0.0;
#pragma unroll
                for (int i = 0; i < L::Q; i++) {
                    off0 += (double)(float)L::w(i);
                    off2 += (double)(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)) * (double)(float)L::w(i);
                }
            }
            const double rho = (off0 + (double)r.hi) + (double)r.lo;
            const float o0h = (float)off0;
            const ff rf = ff_add({o0h, (float)(off0 - (double)o0h)}, r);
            const ff ir = ff_recip(rf);
            o0[sid] = rho;
            if (o1) {
                const ff u = ff_mul(jx, ir);
                o1[sid] = (double)u.hi + (double)u.lo;
            }
            if (o2) {
                const ff v = ff_mul(jy, ir);
                o2[sid] = (double)v.hi + (double)v.lo;
            }
            if (o3) o3[sid] = (off2 + (double)e.hi) + (double)e.lo;
        } else {
            double rho = 0, jx = 0, jy = 0, e2 = 0;
#pragma unroll
            for (int i = 0; i < L::Q; i++) {
                const double f = (double)g[i] + L::w(i) * P.rho0;
                rho += f;
                jx += L::cx(i) * f;
                jy += L::cy(i) * f;
                e2 += (L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)) * f;
            }
            o0[sid] = rho;
            if (o1) o1[sid] = jx / rho;
            if (o2) o2[sid] = jy / rho;
            if (o3) o3[sid] = e2;
        }
    } else {
        T gs[L::Q], rho, ux, uy;
        site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
        o0[sid] = (double)delta_s_exact<L, T>(g, gs, Par<T>::rho0(P));
    }
}

// Ghost exchange of a slab (runs sharded in x): copies the three
// populations that cross a face -- moving right (v_x = +1: 1, 5, 8) or left
// (v_x = -1: 3, 6, 7) -- of column col of the field, between the field and
// a packed buffer [3][ny] (dir 0: field -> buffer; 1: buffer -> field).
template <typename S>
__global__ void k_ghost(const __grid_constant__ Params P, S* field, int col, int right, S* buf, int dir) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * P.ny) return;
    const int p = j / P.ny, y = j - p * P.ny;
    const int plane = right ? (p == 0 ? 1 : (p == 1 ? 5 : 8)) : (p == 0 ? 3 : (p == 1 ? 6 : 7));
    S* at = field + plane * P.plane + (long long)y * P.nxp + col;
    if (dir == 0) buf[j] = *at;
    else *at = buf[j];
}

// ---------------------------------------------------------------------------
// Launchers for one storage type.  Tile shapes of the D2Q9 kernel (sites per
// thread in x, warps per block, minimum resident blocks per SM):
//   0: 1, 8, 3     1: 1, 8, 4     2: 2, 8, 2     3: 4, 8, 1
// and of the staged kernel (rows x columns per block tile, tiles in flight):
//   4: 8 x 128, 2     5: 6 x 128, 3     6: 8 x 64, 2
// The persistent grid is (resident blocks per SM) x (SM count), from the
// occupancy calculator, capped by the number of tiles (small grids then
// spread over as many SMs as they have tiles: their step is latency-bound).
// ---------------------------------------------------------------------------
template <typename S, int EQ, int VEC, int WARPS, int MINB>
cudaError_t launch_d2q9(const Params& P, cudaStream_t st) {
    const long long tiles = (long long)((P.nx + 32 * VEC - 1) / (32 * VEC)) * P.ny;
    const long long want = (tiles + WARPS - 1) / WARPS;   // at least one tile per warp
    const unsigned blocks = (unsigned)std::max(1ll, std::min(want, (long long)P.grid_blocks));
    k_collide_d2q9<S, EQ, VEC, WARPS, MINB><<<blocks, 32 * WARPS, 0, st>>>(P);
    return cudaGetLastError();
}

// Resident blocks per SM of a D2Q9 tile shape (occupancy calculator).
template <typename S, int EQ, int VEC, int WARPS, int MINB>
cudaError_t occupancy_d2q9(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_collide_d2q9<S, EQ, VEC, WARPS, MINB>,
                                                         32 * WARPS, 0);
}

template <typename S, int EQ, int R, int STAGES, int TX = kTmaTX>
cudaError_t launch_d2q9_tma(const Params& P, const void* tmap, cudaStream_t st) {
    constexpr size_t smem = tma_smem_bytes<S, R, STAGES, EQ, TX>();
    const long long tiles = (long long)((P.nx + TX - 1) / TX) * ((P.ny + R - 1) / R);
    const long long want = tiles;   // at least one tile per block
    const unsigned blocks = (unsigned)std::max(1ll, std::min(want, (long long)P.grid_blocks));
    // programmatic stream serialisation: the launch may begin before the
    // previous kernel in the stream completes (the kernel waits for it with
    // griddepcontrol.wait before touching device memory)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32 * R);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_collide_d2q9_tma<S, EQ, R, STAGES, TX>, P,
                              *static_cast<const CUtensorMap*>(tmap));
}

template <typename S, int EQ, int R, int STAGES, int TX = kTmaTX>
cudaError_t setup_d2q9_tma(int* per_sm) {
    constexpr size_t smem = tma_smem_bytes<S, R, STAGES, EQ, TX>();
    cudaError_t e = cudaFuncSetAttribute(k_collide_d2q9_tma<S, EQ, R, STAGES, TX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_collide_d2q9_tma<S, EQ, R, STAGES, TX>,
                                                         32 * R, smem);
}

template <typename L, typename S, int EQ>
struct LaunchImpl {
    static cudaError_t collide(const Params& P, int shape, const void* tmap, cudaStream_t st) {
        if constexpr (L::Q == 9 && EQ >= EQ_ENERGY) {
            // the energy forms are built for two register-fed shapes (0: two
            // resident blocks, 128 registers per thread; 1-3: four, 64) and
            // two staged shapes (5: 6-row tiles, 168 registers; 4: 8-row
            // tiles, 128); shape 6 is refused for them by the host
            if (shape == 5) return launch_d2q9_tma<S, EQ, 6, 3>(P, tmap, st);
            if (shape == 4) return launch_d2q9_tma<S, EQ, 8, 2>(P, tmap, st);
            if (shape == 0) return launch_d2q9<S, EQ, 1, 8, 2>(P, st);
            return launch_d2q9<S, EQ, 1, 8, 4>(P, st);
        } else if constexpr (L::Q == 9) {
            switch (shape) {
                case 1: return launch_d2q9<S, EQ, 1, 8, 4>(P, st);
                case 2: return launch_d2q9<S, EQ, 2, 8, 2>(P, st);
                case 3: return launch_d2q9<S, EQ, 4, 8, 1>(P, st);
                case 4: return launch_d2q9_tma<S, EQ, 8, 2>(P, tmap, st);
                case 5: return launch_d2q9_tma<S, EQ, 6, 3>(P, tmap, st);
                case 6: return launch_d2q9_tma<S, EQ, 8, 2, 64>(P, tmap, st);
                default: return launch_d2q9<S, EQ, 1, 8, 3>(P, st);
            }
        } else {
            (void)shape;
            (void)tmap;
            const long long N = (long long)P.nx * P.ny;
            const unsigned blocks = (unsigned)((N + kSiteBlock - 1) / kSiteBlock);
            k_collide_site<L, S, EQ><<<blocks, kSiteBlock, 0, st>>>(P);
            return cudaGetLastError();
        }
    }
    static cudaError_t occupancy(int shape, int* per_sm) {
        *per_sm = 1;
        if constexpr (L::Q == 9 && EQ >= EQ_ENERGY) {
            if (shape == 5) return setup_d2q9_tma<S, EQ, 6, 3>(per_sm);
            if (shape == 4) return setup_d2q9_tma<S, EQ, 8, 2>(per_sm);
            if (shape == 0) return occupancy_d2q9<S, EQ, 1, 8, 2>(per_sm);
            return occupancy_d2q9<S, EQ, 1, 8, 4>(per_sm);
        } else if constexpr (L::Q == 9) {
            switch (shape) {
                case 1: return occupancy_d2q9<S, EQ, 1, 8, 4>(per_sm);
                case 2: return occupancy_d2q9<S, EQ, 2, 8, 2>(per_sm);
                case 3: return occupancy_d2q9<S, EQ, 4, 8, 1>(per_sm);
                case 4: return setup_d2q9_tma<S, EQ, 8, 2>(per_sm);
                case 5: return setup_d2q9_tma<S, EQ, 6, 3>(per_sm);
                case 6: return setup_d2q9_tma<S, EQ, 8, 2, 64>(per_sm);
                default: return occupancy_d2q9<S, EQ, 1, 8, 3>(per_sm);
            }
        }
        return cudaSuccess;
    }
    static cudaError_t select(const Params& P, int stage_cap, int mode, cudaStream_t st) {
        const size_t smem = (size_t)stage_cap * (sizeof(unsigned long long) + sizeof(unsigned));
        k_select<L, S, EQ><<<1, kSelectThreads, smem, st>>>(P, stage_cap, mode);
        return cudaGetLastError();
    }
    static cudaError_t init_eq(const Params& P, const double* rho, const double* ux,
                               const double* uy, const double* e2, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        k_init_eq<L, S, EQ><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, rho, ux, uy, e2);
        return cudaGetLastError();
    }
    static cudaError_t import_state(const Params& P, const double* f, int i0, int i1, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        if (i0 < 0 || i1 > L::Q || i0 >= i1 || N <= 0) return cudaErrorInvalidValue;
        k_import<L, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, f, i0, i1);
        return cudaGetLastError();
    }
    static cudaError_t export_state(const Params& P, int mode, double* o0, double* o1, double* o2,
                                    double* o3, long long s0, long long s1, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        if (s0 < 0 || s1 > N || s0 >= s1) return cudaErrorInvalidValue;
        k_export<L, S, EQ><<<(unsigned)((s1 - s0 + 255) / 256), 256, 0, st>>>(P, mode, o0, o1, o2, o3, s0, s1);
        return cudaGetLastError();
    }
    static cudaError_t ghost(const Params& P, void* field, int col, int right, void* buf, int dir,
                             cudaStream_t st) {
        const int n = 3 * P.ny;
        k_ghost<S><<<(n + 255) / 256, 256, 0, st>>>(P, static_cast<S*>(field), col, right, static_cast<S*>(buf),
                                                   dir);
        return cudaGetLastError();
    }
    static cudaError_t set_smem(int stage_cap) {
        const size_t smem = (size_t)stage_cap * (sizeof(unsigned long long) + sizeof(unsigned));
        return cudaFuncSetAttribute(k_select<L, S, EQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    }
    static Launchers get() {
        Launchers l;
        l.collide = &collide;
        l.select = &select;
        l.init_eq = &init_eq;
        l.import_state = &import_state;
        l.export_state = &export_state;
        l.set_smem = &set_smem;
        l.ghost = &ghost;
        l.occupancy = &occupancy;
        return l;
    }
};

// Polynomial and entropic (mass and momentum) equilibria of one storage
// type; the energy forms are instantiated in their own translation units.
template <typename S>
Launchers launchers_basic(int lattice, int eq) {
    if (lattice == 0) {
        if (eq == EQ_POLY) return LaunchImpl<D1Q3, S, EQ_POLY>::get();
        return LaunchImpl<D1Q3, S, EQ_ENTROPIC>::get();
    }
    if (eq == EQ_POLY) return LaunchImpl<D2Q9, S, EQ_POLY>::get();
    return LaunchImpl<D2Q9, S, EQ_ENTROPIC>::get();
}

template <typename S>
Launchers launchers_energy(int eq) {
    if (eq == EQ_ENERGY_MLP) return LaunchImpl<D2Q9, S, EQ_ENERGY_MLP>::get();
    return LaunchImpl<D2Q9, S, EQ_ENERGY>::get();
}

}  // namespace lbm
