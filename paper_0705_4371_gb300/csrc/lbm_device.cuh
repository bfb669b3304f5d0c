// lbm_device.cuh -- device building blocks of the Ehrenfest-regularised
// lattice Boltzmann step (Brownlee, Gorban, Levesley 2007) for sm_103a.
//
// Layout in HBM: populations are SoA planes f[Q][ny][nxp] (x fastest, rows
// padded to nxp = round_up(nx, 32) elements so that every row starts on a
// 128-byte boundary).  Deviation storage keeps g_i = f_i - W_i rho0.
// All arithmetic is done in deviation variables (rho0 = 0 for FP64
// storage, 1 for the FP32 and FP16 forms; plain FP32 storage keeps each
// population as its exact difference from the FP32 weight), so the same
// code serves FP64, FP32 and the FP32/FP16 deviation forms.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices (Sec. 4.1: D1Q3 {0, -1, +1}; Sec. 4.2: D2Q9 0 rest, 1..4 E N W S,
// 5..8 NE NW SW SE, weights 4/9, 1/9, 1/36).  D1Q3 weights 2/3, 1/6, 1/6 are
// those of the rest-state quasiequilibrium of Sec. 4.1.
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // population with the opposite velocity / with v_y reversed
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
    __host__ __device__ static constexpr int mir_y(int i) {
        return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
    }
    static constexpr double sum_w_c2 = 2.0 / 3.0;   // sum_i W_i |v_i|^2
};

struct D1Q3 {
    static constexpr int Q = 3;
    __host__ __device__ static constexpr int cx(int i) { return i == 1 ? -1 : (i == 2 ? 1 : 0); }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : 3 - i; }
    __host__ __device__ static constexpr int mir_y(int i) { return i; }
    static constexpr double sum_w_c2 = 1.0 / 3.0;
};

static_assert(D2Q9::opp(1) == 3 && D2Q9::opp(2) == 4 && D2Q9::opp(3) == 1 && D2Q9::opp(4) == 2,
              "D2Q9 opposite of unit speeds");
static_assert(D2Q9::opp(5) == 7 && D2Q9::opp(6) == 8 && D2Q9::opp(7) == 5 && D2Q9::opp(8) == 6,
              "D2Q9 opposite of diagonals");

// ---------------------------------------------------------------------------
// Run parameters (passed by value to every kernel).
// ---------------------------------------------------------------------------
enum : int { EQ_POLY = 0, EQ_ENTROPIC = 1, EQ_ENERGY = 2, EQ_ENERGY_MLP = 3 };
enum : int { BC_BB = 0, BC_FREESLIP = 1, BC_INLET = 2, BC_OUTLET = 3, BC_PERIODIC = 4, BC_OUTLET_COPY = 5 };
enum : int { WALL_BOUNCE_BACK = 0, WALL_DIFFUSE = 1 };
enum : unsigned { ERR_NONFINITE = 1u, ERR_NEWTON = 2u, ERR_TIMEOUT = 4u, ERR_REPLAY = 8u };

struct Params {
    int nx, ny, nxp;
    long long plane;          // ny * nxp elements
    int eq;
    double beta, delta, rho0;
    float betaf, deltaf, rho0f;   // the same in FP32 (no FP64 work in FP32 kernels)
    int k;
    int bc[4];
    double rho_in, ux_in, uy_in;
    double gin[9];            // inlet populations f*(rho_in, u_in) in FP64, as the storage holds them
    int ox0, oy0, ow, oh;
    const void* src;          // post-collision populations of step t-1 (or pre-collision if prestream)
    void* dst;                // post-collision populations of step t
    int prestream;            // src holds pre-collision populations at their own sites
    // candidates and selection
    unsigned long long* cand_key;
    unsigned* cand_idx;
    unsigned* cand_count;
    int cand_per_block;
    int* sel_idx;
    unsigned long long* sel_key;   // keys of the selected candidates (written when not null)
    int* sel_count;
    // logs
    int* count_ring;
    double* probe_ring;
    int ring_cap;
    int probe_x, probe_y;
    long long* step;
    unsigned* err;
    // replay of given selections
    const int* replay_cnt;
    const long long* replay_off;
    const int* replay_idx;
    long long replay_t0, replay_n;
    // precision form: FP64 recheck of dS within recheck_band of delta
    int recheck;
    double recheck_band;
    // energy form
    const float* mlp;         // device copy of the network (FP32 master; rounded to BF16 at use)
    unsigned long long* newton_stats;   // it32, it64, sites, fails
    // completion ticket of the stream-collide blocks (the last block selects)
    unsigned* ticket;
    // sites whose dS the bound could not clear and that did not fit in their
    // block's shared list (resolved by the last block)
    unsigned* pend_idx;
    unsigned* pend_count;
    int grid_blocks;          // persistent grid size (resident blocks x SMs)
    unsigned* tile_counter;   // next tile to hand out (staged shapes)
    const int* tile_order;    // staged shapes: tile of each claim (null: row-major)
    int elbm;                 // ELBM collision (elbmLB) instead of LBGK (entropic f* only)
    int wall;                 // rule on the obstacle's faces: WALL_BOUNCE_BACK / WALL_DIFFUSE
    // slab of a run sharded in x: only columns [own_x0, own_x1) are the
    // slab's sites (the others are ghost copies of the neighbours' columns);
    // the stream-collide launch ends with the slab's own k best candidates
    // (select only), the global selection being applied afterwards
    int slab, own_x0, own_x1;
    int pad_[2];              // size a multiple of 16 bytes (bulk copies)
};

template <int Q, typename T> struct PopArr { T v[Q]; };

// ---------------------------------------------------------------------------
// Storage traits: load / store a population as a deviation in type T.
// ---------------------------------------------------------------------------
// kProject: the collision removes the rounding defects of the conserved
// moments of f - f* (conserve_neq below) -- FP32 storage, whose arithmetic
// error would otherwise exceed the storage rounding; FP64 arithmetic is
// exact enough, and FP16 storage rounding dominates its FP32 arithmetic.
// kPlain: plain FP32 storage (plain32): each population f is held as an FP32
// value, kept in the buffer as its exact difference g = f - fl32(W_i) from
// the FP32 weight, so that the FP32 arithmetic works on deviations for
// every FP32 form.
struct plain32 {
    float v;
};
template <typename S> struct Store;
template <> struct Store<double> {
    using T = double;
    static constexpr bool kProject = false, kPlain = false;
    __device__ static T load(const void* p, long long i) { return static_cast<const double*>(p)[i]; }
    __device__ static void store(void* p, long long i, T v) { static_cast<double*>(p)[i] = v; }
};
template <> struct Store<float> {
    using T = float;
    static constexpr bool kProject = true, kPlain = false;
    __device__ static T load(const void* p, long long i) { return static_cast<const float*>(p)[i]; }
    __device__ static void store(void* p, long long i, T v) { static_cast<float*>(p)[i] = v; }
};
template <> struct Store<plain32> {
    using T = float;
    static constexpr bool kProject = true, kPlain = true;
    __device__ static T load(const void* p, long long i) { return static_cast<const float*>(p)[i]; }
    __device__ static void store(void* p, long long i, T v) { static_cast<float*>(p)[i] = v; }
};
template <> struct Store<__half> {
    using T = float;
    static constexpr bool kProject = false, kPlain = false;
    __device__ static T load(const void* p, long long i) {
        return __half2float(static_cast<const __half*>(p)[i]);
    }
    __device__ static void store(void* p, long long i, T v) {
        static_cast<__half*>(p)[i] = __float2half_rn(v);
    }
};

// ---------------------------------------------------------------------------
// Geometry helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_solid(const Params& P, int x, int y) {
    return P.ow > 0 && x >= P.ox0 && x < P.ox0 + P.ow && y >= P.oy0 && y < P.oy0 + P.oh;
}

// ---------------------------------------------------------------------------
// Quasiequilibria as deviations gs_i = f*_i - W_i rho0 in type T.
// ---------------------------------------------------------------------------

// Polynomial (Sec. 4.1 for D1Q3; standard second-order D2Q9 form).
// gs_i = W_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)).
// The library is compiled without automatic multiply-add contraction; every
// fused multiply-add is written out, so each kernel that evaluates these
// functions produces the same bits (bit-exact checkpoint / resume).
template <typename T> __host__ __device__ __forceinline__ T dfma(T a, T b, T c);
template <> __host__ __device__ __forceinline__ float dfma<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __host__ __device__ __forceinline__ double dfma<double>(double a, double b, double c) { return fma(a, b, c); }

// v . u for lattice velocity components in {-1, 0, 1}: additions only.
template <typename L, typename T>
__host__ __device__ __forceinline__ T cdotu(int i, T ux, T uy) {
    const T a = L::cx(i) == 1 ? ux : -ux;
    const T b = L::cy(i) == 1 ? uy : -uy;
    if (L::cx(i) == 0) return L::cy(i) == 0 ? T(0) : b;
    if (L::cy(i) == 0) return a;
    return a + b;
}

// Populations i and opp(i) share (v.u)^2 and have opposite v.u, so each
// pair is evaluated once: gs = W (c0 + 9/2 rho (v.u)^2) +- W 3 rho (v.u),
// c0 = drho - 3/2 rho u^2.
template <typename L, typename T>
__host__ __device__ __forceinline__ void feq_poly(T drho, T rho, T ux, T uy, T* gs) {
    const T usq = dfma<T>(ux, ux, uy * uy);
    const T c0 = dfma<T>(T(-1.5) * rho, usq, drho);
    const T r45 = T(4.5) * rho, r3 = T(3) * rho;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        if (i == 0) {
            gs[0] = T(L::w(0)) * c0;
        } else if (i < L::opp(i)) {
            const T cu = cdotu<L, T>(i, ux, uy);
            const T w = T(L::w(i));
            const T a = dfma<T>(r45 * cu, cu, c0);
            const T b = r3 * cu;
            gs[i] = w * (a + b);
            gs[L::opp(i)] = w * (a - b);
        }
    }
}

// Run parameters in the arithmetic type T.
template <typename T> struct Par;
template <> struct Par<float> {
    __device__ static float beta(const Params& P) { return P.betaf; }
    __device__ static float delta(const Params& P) { return P.deltaf; }
    __device__ static float rho0(const Params& P) { return P.rho0f; }
};
template <> struct Par<double> {
    __device__ static double beta(const Params& P) { return P.beta; }
    __device__ static double delta(const Params& P) { return P.delta; }
    __device__ static double rho0(const Params& P) { return P.rho0; }
};

// ---------------------------------------------------------------------------
// Stored values and the deviations the arithmetic works on.  FP64 storage
// holds f (rho0 = 0); FP32 / FP16 deviation storage holds g = f - W_i rho0
// (rho0 = 1); plain FP32 storage holds the FP32 value of f, kept as the
// exact difference g = f - fl32(W_i).  FP32 arithmetic takes rho0 = 1 for
// every FP32 / FP16 form.
// ---------------------------------------------------------------------------

// FP64 value of population i whose stored deviation is g.
template <typename L, typename S>
__device__ __forceinline__ double pop_f64(const Params& P, int i, typename Store<S>::T g) {
    if constexpr (Store<S>::kPlain) return (double)g + (double)(float)L::w(i);
    else return (double)g + L::w(i) * P.rho0;
}

// Deviation of a population whose value f was computed in FP64 (initial and
// imported states), as a stored field holds it: plain FP32 rounds f, the
// deviation forms round f - W_i rho0.
template <typename L, typename S>
__device__ __forceinline__ typename Store<S>::T dev_of_f64(const Params& P, int i, double f) {
    using T = typename Store<S>::T;
    if constexpr (Store<S>::kPlain) return (float)f - (float)L::w(i);
    else return (T)(f - L::w(i) * P.rho0);
}

// A deviation computed in the arithmetic, rounded as the storage rounds it:
// plain FP32 storage rounds f = g + fl32(W_i) to FP32 (the difference with
// fl32(W_i) is then exact when f lies within a factor two of W_i); the other
// forms round at the store itself.
template <typename L, typename S>
__device__ __forceinline__ typename Store<S>::T store_round(int i, typename Store<S>::T g) {
    if constexpr (Store<S>::kPlain) {
        const float w = (float)L::w(i);
        return (g + w) - w;
    } else {
        (void)i;
        return g;
    }
}

// Conserved moments of the nonequilibrium part d = f - f*: zero in exact
// arithmetic, since f* has the conserved moments of f (mass and momentum
// (lbgkLB), and the energy 2E for the energy-constrained quasiequilibrium,
// Sec. 3.3).  The FP32 evaluation of f* leaves errors of a few ulps in each
// f*_i, whose sums the over-relaxed collision f' = f - 2 beta d (beta ~ 1)
// would turn into a drift of the conserved quantities by about twice their
// value per step, the same at every site of a smooth flow.  They are removed
// by subtracting the combination W_i (a + b . v_i + e |v_i|^2) of the
// collision invariants that has the same moments as d (D2Q9: sum W = 1,
// sum W v v = I/3, sum W |v|^2 = 2/3, sum W |v|^4 = 8/9; e = 0 without the
// energy constraint; D1Q3: sum W v^2 = 1/3).  The sums are of the small
// nonequilibrium parts, so the conserved moments of the result are exact to
// their rounding; in exact arithmetic nothing changes.
template <typename L, int EQ>
__device__ __forceinline__ void conserve_neq(float* d) {
    if constexpr (L::Q == 9) {
        const float D0 = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const float Dx = ((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7]);
        const float Dy = ((d[2] - d[4]) + (d[5] - d[8])) + (d[6] - d[7]);
        float a = D0, e = 0.0f;
        if constexpr (EQ >= EQ_ENERGY) {
            const float DE = ((d[1] + d[2]) + (d[3] + d[4])) + 2.0f * ((d[5] + d[6]) + (d[7] + d[8]));
            a = fmaf(-1.5f, DE, 2.0f * D0);     // a = 2 D0 - 3/2 DE
            e = fmaf(2.25f, DE, -1.5f * D0);    // e = 9/4 DE - 3/2 D0
        }
        // W_i (a + 3 v_i . D + e |v_i|^2), weights 4/9, 1/9, 1/36
        const float m1 = (a + e) * (1.0f / 9.0f), px = Dx * (1.0f / 3.0f), py = Dy * (1.0f / 3.0f);
        const float m5 = fmaf(2.0f, e, a) * (1.0f / 36.0f), qx = Dx * (1.0f / 12.0f), qy = Dy * (1.0f / 12.0f);
        d[0] -= a * (4.0f / 9.0f);
        d[1] -= m1 + px;
        d[3] -= m1 - px;
        d[2] -= m1 + py;
        d[4] -= m1 - py;
        const float s1 = m5 + qy, s2 = m5 - qy;
        d[5] -= s1 + qx;
        d[6] -= s1 - qx;
        d[7] -= s2 - qx;
        d[8] -= s2 + qx;
    } else {
        const float D0 = (d[0] + d[1]) + d[2];
        const float Dx = d[2] - d[1];
        const float m = D0 * (1.0f / 6.0f), p = Dx * 0.5f;   // W (D0 + 3 v Dx), W = 1/6
        d[0] -= D0 * (2.0f / 3.0f);
        d[1] -= m - p;
        d[2] -= m + p;
    }
}

template <typename T> __host__ __device__ __forceinline__ T dsqrt(T x);
template <> __host__ __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __host__ __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// Entropic for mass and momentum.  D1Q3: closed form of Sec. 4.1 with the
// left/right labels read so that the momentum is +rho u (rest
// (2 rho/3)(2 - s), left (rho/6)(2s - 3u - 1), right (rho/6)(3u - 1 + 2s),
// s = sqrt(1 + 3u^2)).  D2Q9: product formula of Sec. 4.2.
template <typename L, typename T>
__host__ __device__ __forceinline__ void feq_entropic(T rho, T ux, T uy, T rho0, T* gs) {
    if constexpr (L::Q == 3) {
        const T s = dsqrt<T>(T(1) + T(3) * ux * ux);
        gs[0] = T(2) * rho / T(3) * (T(2) - s) - T(L::w(0)) * rho0;
        gs[1] = rho / T(6) * (T(2) * s - T(3) * ux - T(1)) - T(L::w(1)) * rho0;
        gs[2] = rho / T(6) * (T(3) * ux - T(1) + T(2) * s) - T(L::w(2)) * rho0;
    } else {
        const T sx = dsqrt<T>(T(1) + T(3) * ux * ux), sy = dsqrt<T>(T(1) + T(3) * uy * uy);
        const T ax = T(2) - sx, ay = T(2) - sy;
        const T bx = (T(2) * ux + sx) / (T(1) - ux), by = (T(2) * uy + sy) / (T(1) - uy);
        const T ibx = T(1) / bx, iby = T(1) / by;
        const T base = rho * ax * ay;
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            T p = base * T(L::w(i));
            if (L::cx(i) == 1) p *= bx;
            if (L::cx(i) == -1) p *= ibx;
            if (L::cy(i) == 1) p *= by;
            if (L::cy(i) == -1) p *= iby;
            gs[i] = p - T(L::w(i)) * rho0;
        }
    }
}

// Boundary equilibrium from (rho, u): polynomial or entropic formula (the
// energy forms use the isothermal entropic formula, whose energy
// multiplier is zero).
template <typename L, typename T>
__host__ __device__ __forceinline__ void feq_rho_u(int eq, T rho, T ux, T uy, T rho0, T* gs) {
    if (eq == EQ_POLY) feq_poly<L, T>(rho - rho0, rho, ux, uy, gs);
    else feq_entropic<L, T>(rho, ux, uy, rho0, gs);
}

// ---------------------------------------------------------------------------
// Nonequilibrium entropy (DelS).
// With x_i = (f_i - f*_i) / f*_i and phi(x) = (1+x) ln(1+x) - x >= 0,
//   sum_i f*_i phi(x_i) = sum_i f_i ln(f_i/f*_i) - sum_i (f_i - f*_i),
// which is dS because f and f* share their density.  The phi form has no
// first-order cancellation.  phi is evaluated by its Taylor series
// sum_{n>=2} (-1)^n x^n / (n (n-1)) for small |x| and from log1p otherwise.
// Outside the positive cone (some f_i < 0 or f*_i <= 0) dS = +inf.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T phi_fn(T x);

template <> __device__ __forceinline__ float phi_fn<float>(float x) {
    if (fabsf(x) <= 0.25f) {
        // terms n = 2..13; truncation < 1e-9 relative at |x| = 1/4
        float p = -1.0f / 156.0f;
        p = fmaf(p, x, 1.0f / 132.0f);
        p = fmaf(p, x, -1.0f / 110.0f);
        p = fmaf(p, x, 1.0f / 90.0f);
        p = fmaf(p, x, -1.0f / 72.0f);
        p = fmaf(p, x, 1.0f / 56.0f);
        p = fmaf(p, x, -1.0f / 42.0f);
        p = fmaf(p, x, 1.0f / 30.0f);
        p = fmaf(p, x, -1.0f / 20.0f);
        p = fmaf(p, x, 1.0f / 12.0f);
        p = fmaf(p, x, -1.0f / 6.0f);
        p = fmaf(p, x, 0.5f);
        return x * x * p;
    }
    if (x <= -1.0f) return 1.0f;  // f_i = 0: 0 ln 0 - (0 - f*) = f*
    return fmaf(1.0f + x, log1pf(x), -x);
}

template <> __device__ __forceinline__ double phi_fn<double>(double x) {
    if (fabs(x) <= 0.0625) {
        // terms n = 2..17; truncation < 1e-18 relative at |x| = 1/16
        double p = 0.0;
#pragma unroll
        for (int n = 17; n >= 2; n--) {
            const double c = ((n & 1) ? -1.0 : 1.0) / (double(n) * double(n - 1));
            p = fma(p, x, c);
        }
        return x * x * p;
    }
    if (x <= -1.0) return 1.0;
    return fma(1.0 + x, log1p(x), -x);
}

// 1 / x: FP32 from the hardware approximation refined by one Newton-Raphson
// step r + r (1 - x r) (the relative error e of the seed becomes ~e^2, below
// one ulp); FP64 divides.
template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ float recip<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }

// Exact dS of one site in type T; +inf outside the positive cone.
template <typename L, typename T>
__device__ __forceinline__ T delta_s_exact(const T* g, const T* gs, T rho0) {
    bool bad = false;
    T x[L::Q], fs[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        fs[i] = dfma<T>(T(L::w(i)), rho0, gs[i]);
        const T f = dfma<T>(T(L::w(i)), rho0, g[i]);
        bad |= !(fs[i] > T(0)) || (f < T(0));
        x[i] = (g[i] - gs[i]) / fs[i];
    }
    if (bad) return T(INFINITY);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; i++) s = dfma<T>(fs[i], phi_fn<T>(x[i]), s);
    return s;
}

// Out-of-line copy for the rare sites that the bound below does not clear.
template <typename L, typename T>
__device__ __noinline__ T delta_s_slow(PopArr<L::Q, T> g, PopArr<L::Q, T> gs, T rho0) {
    return delta_s_exact<L, T>(g.v, gs.v, rho0);
}

// Division-free bound that clears a site (dS <= delta) without evaluating
// dS.  With d_i = f_i - f*_i, x_i = d_i / f*_i and m <= min_i f*_i / W_i:
//   Q = sum_i d_i^2 / W_i >= m sum_i d_i^2 / f*_i  and  x_i^2 <= Q / (W_min m^2),
// so Q <= m^2 W_min / 16 gives |x_i| <= 1/4 (hence f_i > 0), where
// phi(x) <= 0.5478 x^2, and then dS = sum f* phi(x) <= 0.55 Q / m.
// The site is cleared when m > 0, 16 Q <= W_min m^2 and 0.55 Q <= delta m.
// Polynomial f*: f*_i / W_i = rho (1 + 3 v.u + 9/2 (v.u)^2 - 3/2 u^2) >=
// rho (1 - 3 (|u_x| + |u_y|) - 3/2 u^2) = m.  Other f*: m = min_i f*_i / W_i.
template <typename L, typename T, int EQ>
__device__ __forceinline__ bool ds_cleared(const T* d, const T* gs, T rho, T ux, T uy, T rho0,
                                           T delta) {
    T q0 = T(0), q1 = T(0), q2 = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        if (L::w(i) == L::w(0)) q0 = dfma<T>(d[i], d[i], q0);
        else if (L::w(i) == L::w(1)) q1 = dfma<T>(d[i], d[i], q1);
        else q2 = dfma<T>(d[i], d[i], q2);
    }
    constexpr double wmin = L::Q == 9 ? 1.0 / 36.0 : 1.0 / 6.0;
    const T Q = dfma<T>(q0, T(1.0 / L::w(0)), dfma<T>(q1, T(1.0 / L::w(1)),
                        L::Q == 9 ? q2 * T(1.0 / L::w(5)) : T(0)));
    T m;
    if constexpr (EQ == 0) {
        const T usq = dfma<T>(ux, ux, uy * uy);
        m = rho * dfma<T>(T(-1.5), usq, dfma<T>(T(-3), fabs(ux) + fabs(uy), T(1)));
    } else {
        m = T(INFINITY);
#pragma unroll
        for (int i = 0; i < L::Q; i++) m = fmin(m, dfma<T>(gs[i], T(1.0 / L::w(i)), rho0));
    }
    return (m > T(0)) && (T(16.0 / wmin) * Q <= m * m) && (T(0.55) * Q <= delta * m);
}

// Monotone map of a double onto uint64 (larger double <=> larger key).
__device__ __forceinline__ unsigned long long ds_key(double d) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// ---------------------------------------------------------------------------
// Free flight with boundary rules (Sec. 3 map Theta_tau; Sec. 4.2).
// Pre-collision deviation populations at fluid site (x, y) from the
// post-collision field src.  Rules where x - v_i leaves the fluid:
//   x side: PERIODIC wraps, INLET = f*(rho_in, u_in), OUTLET = f*(rho, u of
//           column nx-2 in the same row), BB = own opposite population;
//   y side: PERIODIC wraps, FREESLIP = population (v_x, -v_y) of (x - v_x, y),
//           BB = own opposite population;
//   solid source: own opposite population (half-way bounce-back), or with
//           wall = WALL_DIFFUSE the diffuse kinetic wall (diffuse_wall).
// The x rule is applied first (inlet and outlet win at corners).
// ---------------------------------------------------------------------------

// Diffuse kinetic wall at rest (Maxwell's diffuse reflection, the kinetic
// boundary condition cited in Sec. 4.2): the wall re-emits the mass it
// absorbed as its rest quasiequilibrium W_i rho_w.  The links in mask
// (source inside the obstacle) enter holding f'_{-i}(x), the absorbed
// populations, and leave with
//   f_i = W_i (sum_{j in mask} f'_{-j}) / (sum_{j in mask} W_j).
// The same map holds for deviations g = f - W rho0 (the W_i rho0 parts
// cancel), so it applies to every storage form as it stands.
template <typename L, typename T>
__device__ __forceinline__ void diffuse_wall(unsigned mask, T* g) {
    T absorbed = T(0), wsum = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; i++)
        if ((mask >> i) & 1u) {
            absorbed += g[i];
            wsum += T(L::w(i));
        }
    const T rho_w = absorbed / wsum;
#pragma unroll
    for (int i = 0; i < L::Q; i++)
        if ((mask >> i) & 1u) g[i] = T(L::w(i)) * rho_w;
}

// Quasiequilibrium f*(rho, u) evaluated in FP64 and held as the storage
// holds a population (dev_of_f64): the initial state.
template <typename L, typename S>
__device__ __forceinline__ void bc_equilibrium(const Params& P, double rho, double ux, double uy,
                                               typename Store<S>::T* g) {
    double fs[L::Q];
    feq_rho_u<L, double>(P.eq, rho, ux, uy, 0.0, fs);
#pragma unroll
    for (int i = 0; i < L::Q; i++) g[i] = dev_of_f64<L, S>(P, i, fs[i]);
}

// Outlet rule of Sec. 4.2: the quasiequilibrium of the density and velocity
// of column nx - 2 (stored deviations v), in the run's arithmetic (the
// callers round it as the storage holds a population).
template <typename L, typename T>
__device__ __forceinline__ void outlet_equilibrium(const Params& P, const T* v, T* g) {
    const T rho0 = Par<T>::rho0(P);
    T drho = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int j = 0; j < L::Q; j++) {
        drho += v[j];
        jx += T(L::cx(j)) * v[j];
        jy += T(L::cy(j)) * v[j];
    }
    const T rho = rho0 + drho;
    feq_rho_u<L, T>(P.eq, rho, jx / rho, jy / rho, rho0, g);
}

// Inlet rule of Sec. 4.2: the quasiequilibrium of the free stream, computed
// once in FP64 by the host (Params::gin).
template <typename L, typename T>
__device__ __forceinline__ void inlet_equilibrium(const Params& P, T* g) {
#pragma unroll
    for (int i = 0; i < L::Q; i++) g[i] = (T)P.gin[i];
}

template <typename L, typename S>
__device__ void gather_site(const Params& P, int x, int y, typename Store<S>::T* g) {
    using T = typename Store<S>::T;
    const long long s0 = (long long)y * P.nxp + x;
    if (P.prestream) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) g[i] = Store<S>::load(P.src, i * P.plane + s0);
        return;
    }
    bool have_in = false, have_out = false;
    unsigned wall_mask = 0u;
    T gin[L::Q], gout[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const int cx = L::cx(i), cy = L::cy(i);
        int sx = x - cx, sy = y - cy;
        if (sx < 0 || sx >= P.nx) {
            const int kind = sx < 0 ? P.bc[0] : P.bc[1];
            if (kind == BC_PERIODIC) {
                sx = sx < 0 ? sx + P.nx : sx - P.nx;
            } else if (kind == BC_INLET) {
                if (!have_in) {
                    inlet_equilibrium<L, T>(P, gin);
                    have_in = true;
                }
                g[i] = gin[i];
                continue;
            } else if (kind == BC_OUTLET) {
                if (!have_out) {
                    const long long sp = (long long)y * P.nxp + (P.nx - 2);
                    T v[L::Q];
#pragma unroll
                    for (int j = 0; j < L::Q; j++) v[j] = Store<S>::load(P.src, j * P.plane + sp);
                    outlet_equilibrium<L, T>(P, v, gout);
#pragma unroll
                    for (int j = 0; j < L::Q; j++) gout[j] = store_round<L, S>(j, gout[j]);
                    have_out = true;
                }
                g[i] = gout[i];
                continue;
            } else if (kind == BC_OUTLET_COPY) {
                // zero-gradient outflow: the column beyond the side is a copy
                // of the side column; the y and obstacle rules then apply
                sx = x;
            } else {
                g[i] = Store<S>::load(P.src, L::opp(i) * P.plane + s0);
                continue;
            }
        }
        if (sy < 0 || sy >= P.ny) {
            const int kind = sy < 0 ? P.bc[2] : P.bc[3];
            if (kind == BC_PERIODIC) {
                sy = sy < 0 ? sy + P.ny : sy - P.ny;
            } else if (kind == BC_FREESLIP) {
                g[i] = Store<S>::load(P.src, L::mir_y(i) * P.plane + (long long)y * P.nxp + sx);
                continue;
            } else {
                g[i] = Store<S>::load(P.src, L::opp(i) * P.plane + s0);
                continue;
            }
        }
        if (is_solid(P, sx, sy)) {
            g[i] = Store<S>::load(P.src, L::opp(i) * P.plane + s0);
            if (P.wall == WALL_DIFFUSE) wall_mask |= 1u << i;
            continue;
        }
        g[i] = Store<S>::load(P.src, i * P.plane + (long long)sy * P.nxp + sx);
    }
    if (wall_mask) diffuse_wall<L, T>(wall_mask, g);
}

// ---------------------------------------------------------------------------
// Block-wide top-k by radix select.
// Elements e in [0, n) with keys key[e] (uint64, larger = better) and unique
// indices idx[e]; total order (key descending, idx ascending).  The function
// finds the threshold so that exactly k (< n) elements are selected:
// selected(e) <=> (key & kmask) > kpre, or (key & kmask) == kpre and
// (all_tied or (~idx & imask) >= ipre).  Digits of 8 bits from the most
// significant differing bit down; the idx phase runs only when more than the
// needed number of elements share the exact threshold key.
// key/idx may point to shared or global memory.  All threads of the block
// must call it; scratch is shared memory supplied by the caller.
// ---------------------------------------------------------------------------
struct TopkScratch {
    unsigned hist[256];
    unsigned long long red_or[32], red_and[32];
    unsigned long long kpre, kmask;
    unsigned ipre, imask;
    int need;           // elements still to take among the tied group
    int all_tied;
    int digit;          // result of the last radix pass
    unsigned above;     // elements in digits above it
    int hi;             // most significant bit where keys differ (-1: none)
    unsigned long long diff;
};

struct Thresh {
    unsigned long long kpre, kmask;
    unsigned ipre, imask;
    int all_tied;
    __device__ __forceinline__ bool selected(unsigned long long key, unsigned id) const {
        const unsigned long long km = key & kmask;
        if (km != kpre) return km > kpre;
        if (all_tied) return true;
        return ((~id) & imask) >= ipre;
    }
};

// one radix pass over a digit [lo, lo+width) of the value returned by getv
// for elements matching the current prefix; updates prefix/need.
template <typename GetV, typename Match>
__device__ void radix_pass(TopkScratch& sc, int n, int lo, int width, GetV getv, Match match) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int b = tid; b < 256; b += nt) sc.hist[b] = 0;
    __syncthreads();
    const unsigned dmask = (1u << width) - 1u;
    if (tid == 0) { sc.digit = 0; sc.above = 0; }
    for (int e = tid; e < n; e += nt) {
        if (match(e)) atomicAdd(&sc.hist[(unsigned)(getv(e) >> lo) & dmask], 1u);
    }
    __syncthreads();
    if (tid < 32) {
        // bins b = 255..0 scanned from the top: lane l owns bins 8l..8l+7
        unsigned c[8], tot = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) { c[j] = sc.hist[tid * 8 + j]; tot += c[j]; }
        // inclusive suffix sum over lanes (lane 31 holds the top bins)
        unsigned suf = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_down_sync(0xffffffffu, suf, o);
            if (tid + o < 32) suf += v;
        }
        unsigned above = suf - tot;   // elements in bins above this lane's bins
        const unsigned need = (unsigned)sc.need;
        // the lane whose range contains the need-th element from the top
        const bool mine = above < need && need <= suf;
        if (mine) {
            unsigned acc = above;
            for (int j = 7; j >= 0; j--) {
                if (acc + c[j] >= need) {
                    sc.digit = tid * 8 + j;
                    sc.above = acc;
                    break;
                }
                acc += c[j];
            }
        }
    }
    __syncthreads();
}

template <typename KeyAt, typename IdAt>
__device__ Thresh block_topk(TopkScratch& sc, int n, int k, KeyAt keyat, IdAt idat) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    // common bits of all keys: skip digits where every key agrees
    unsigned long long o = 0, a = ~0ull;
    for (int e = tid; e < n; e += nt) { const unsigned long long v = keyat(e); o |= v; a &= v; }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, s);
        a &= __shfl_xor_sync(0xffffffffu, a, s);
    }
    if (lane == 0) { sc.red_or[warp] = o; sc.red_and[warp] = a; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long oo = 0, aa = ~0ull;
        for (int w = 0; w < (nt + 31) / 32; w++) { oo |= sc.red_or[w]; aa &= sc.red_and[w]; }
        const unsigned long long diff = oo ^ aa;
        const int hi = diff ? 63 - __clzll(diff) : -1;
        const unsigned long long above_hi = hi >= 63 ? 0ull : (~0ull << (hi + 1));
        sc.kmask = above_hi;
        sc.kpre = aa & above_hi;
        sc.need = k;
        sc.all_tied = 0;
        sc.ipre = 0;
        sc.imask = 0;
        sc.hi = hi;
        sc.diff = diff;
    }
    __syncthreads();
    const int hi = sc.hi;
    const unsigned long long diff = sc.diff;
    const int lo_bit = diff ? __ffsll((long long)diff) - 1 : 0;
    bool done = (hi < 0);   // all keys equal: go to the idx phase
    for (int top = hi; !done && top >= lo_bit; top -= 8) {
        const int lo = top - 7 > lo_bit ? top - 7 : lo_bit;
        const int width = top - lo + 1;
        const unsigned long long kpre = sc.kpre, kmask = sc.kmask;
        radix_pass(sc, n, lo, width, keyat,
                   [&](int e) { return (keyat(e) & kmask) == kpre; });
        if (tid == 0) {
            const unsigned long long dm = ((1ull << width) - 1ull) << lo;
            sc.kpre |= (unsigned long long)sc.digit << lo;
            sc.kmask |= dm;
            sc.need -= (int)sc.above;
            if (sc.hist[sc.digit] == (unsigned)sc.need) sc.all_tied = 1;
        }
        __syncthreads();
        if (sc.all_tied) done = true;
    }
    if (!sc.all_tied) {
        // the threshold key is fully determined; lower bits are common to all
        if (tid == 0) {
            // complete kpre with the common low bits
            unsigned long long low = (lo_bit > 0) ? ((1ull << lo_bit) - 1ull) : 0ull;
            sc.kpre = (sc.kpre & ~low) | (keyat(0) & low);
            sc.kmask = ~0ull;
        }
        __syncthreads();
        const unsigned long long T = sc.kpre;
        // idx phase on ~idx (larger ~idx = smaller idx) among key == T
        for (int top = 31; top >= 0; top -= 8) {
            const int lo = top - 7;
            const unsigned ipre = sc.ipre, imask = sc.imask;
            radix_pass(sc, n, lo, 8, [&](int e) { return (unsigned long long)(~idat(e)); },
                       [&](int e) { return keyat(e) == T && ((~idat(e)) & imask) == ipre; });
            if (tid == 0) {
                sc.ipre |= (unsigned)sc.digit << lo;
                sc.imask |= 0xffu << lo;
                sc.need -= (int)sc.above;
                if (sc.hist[sc.digit] == (unsigned)sc.need) sc.all_tied = 2;
            }
            __syncthreads();
            if (sc.all_tied) break;
        }
    }
    Thresh t;
    t.kpre = sc.kpre;
    t.kmask = sc.kmask;
    t.ipre = sc.ipre;
    t.imask = sc.imask;
    t.all_tied = sc.all_tied == 1;
    __syncthreads();
    return t;
}

}  // namespace lbm
