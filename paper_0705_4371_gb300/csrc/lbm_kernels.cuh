// lbm_kernels.cuh -- kernels of one time step (template definitions; each
// storage type is instantiated in its own translation unit).
//
//   k_collide_d2q9   fused pull-stream + moments + f* + dS + LBGK + per-block
//                    top-k of the Ehrenfests' candidates (the HBM-bound
//                    kernel; 4 sites per thread, aligned vector loads and
//                    warp shuffles for the x-shifted planes in the interior)
//   k_collide_site   the same update, one site per thread (D1Q3 runs)
//   The last block of each stream-collide launch runs the global radix
//   select of the k sites with the largest dS > delta over the block
//   candidates and the Ehrenfests' step f <- f* at those sites (Sec. 3.2;
//   (ESLB)), so one time step is one launch.
//   k_select         the same selection as a stand-alone kernel (test hook)
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kSelectThreads = 1024;
constexpr int kSiteBlock = 256;      // one-site-per-thread kernels

template <int N>
struct BlockCand {
    unsigned long long key[N];
    unsigned idx[N];
    unsigned count;
    unsigned base;
    unsigned cnt2;
    int is_last;
    int nsel;
    TopkScratch sc;
};

// Append (dS, site) to the block's candidate list.
template <int N>
__device__ __forceinline__ void push_candidate(BlockCand<N>& sh, double ds, unsigned site) {
    const unsigned slot = atomicAdd(&sh.count, 1u);
    sh.key[slot] = ds_key(ds);
    sh.idx[slot] = site;
}

// Block stage of the selection: keep at most k candidates per block (all of
// them if there are no more than k), appended to the global candidate list.
template <int N>
__device__ void block_emit(const Params& P, BlockCand<N>& sh) {
    __syncthreads();
    const int n = (int)sh.count;
    if (n == 0) return;
    const int tid = threadIdx.x;
    if (n <= P.k) {
        if (tid == 0) sh.base = atomicAdd(P.cand_count, (unsigned)n);
        __syncthreads();
        for (int e = tid; e < n; e += blockDim.x) {
            P.cand_key[sh.base + e] = sh.key[e];
            P.cand_idx[sh.base + e] = sh.idx[e];
        }
        return;
    }
    const Thresh th = block_topk(sh.sc, n, P.k, [&](int e) { return sh.key[e]; },
                                 [&](int e) { return sh.idx[e]; });
    if (tid == 0) {
        sh.base = atomicAdd(P.cand_count, (unsigned)P.k);
        sh.cnt2 = 0;
    }
    __syncthreads();
    for (int e = tid; e < n; e += blockDim.x) {
        if (th.selected(sh.key[e], sh.idx[e])) {
            const unsigned s = atomicAdd(&sh.cnt2, 1u);
            if (s < (unsigned)P.k) {   // exactly k are selected; the check only bounds the write
                P.cand_key[sh.base + s] = sh.key[e];
                P.cand_idx[sh.base + s] = sh.idx[e];
            }
        }
    }
}

template <typename L, typename T, int EQ>
__device__ __forceinline__ void equilibrium(const Params& P, T drho, T rho, T ux, T uy, T* gs) {
    if constexpr (EQ == EQ_POLY) feq_poly<L, T>(drho, rho, ux, uy, gs);
    else feq_entropic<L, T>(rho, ux, uy, T(P.rho0), gs);
}

template <typename L, typename T>
__device__ __forceinline__ void moments(const T* g, T rho0, T& drho, T& rho, T& jx, T& jy) {
    drho = T(0); jx = T(0); jy = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        drho += g[i];
        if (L::cx(i) == 1) jx += g[i];
        if (L::cx(i) == -1) jx -= g[i];
        if (L::cy(i) == 1) jy += g[i];
        if (L::cy(i) == -1) jy -= g[i];
    }
    rho = rho0 + drho;
}

// u = j / rho: FP64 divides (as the oracle does); FP32 multiplies by the
// correctly rounded reciprocal.
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

// Quasiequilibrium of a gathered site (shared by the collision, the
// Ehrenfests' step and the exports so that all round identically).
template <typename L, typename T, int EQ>
__device__ __forceinline__ void site_equilibrium(const Params& P, const T* g, T* gs, T& rho, T& ux,
                                                 T& uy) {
    T drho, jx, jy;
    moments<L, T>(g, T(P.rho0), drho, rho, jx, jy);
    velocity<T>(jx, jy, rho, ux, uy);
    equilibrium<L, T, EQ>(P, drho, rho, ux, uy, gs);
}

// FP64 recomputation of dS from the stored populations (precision form).
template <typename L, typename T, int EQ>
__device__ __noinline__ double delta_s_fp64(PopArr<L::Q, T> g, double rho0) {
    double gd[L::Q], gs[L::Q], drho, rho, jx, jy, ux, uy;
#pragma unroll
    for (int i = 0; i < L::Q; i++) gd[i] = (double)g.v[i];
    moments<L, double>(gd, rho0, drho, rho, jx, jy);
    velocity<double>(jx, jy, rho, ux, uy);
    if constexpr (EQ == EQ_POLY) feq_poly<L, double>(drho, rho, ux, uy, gs);
    else feq_entropic<L, double>(rho, ux, uy, rho0, gs);
    return delta_s_exact<L, double>(gd, gs, rho0);
}

// Per-site update after the gather: moments, f*, dS, LBGK.
// g: pre-collision deviations in, post-collision deviations out.
// Returns dS (negative: cleared by the bound, not a candidate).
template <typename L, typename T, int EQ>
__device__ __forceinline__ double update_site(const Params& P, T* g, int x, int y, long long t,
                                              bool& nonfinite) {
    T gs[L::Q], rho, ux, uy;
    site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
    nonfinite |= !isfinite(rho + ux + uy);
    if (x == P.probe_x && y == P.probe_y && P.probe_ring)
        P.probe_ring[t % P.ring_cap] = (double)ux;
    T d[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; i++) d[i] = g[i] - gs[i];
    double ds = -1.0;
    if (P.k > 0 && !ds_cleared<L, T, EQ>(d, gs, rho, ux, uy, T(P.rho0), T(P.delta))) {
        PopArr<L::Q, T> ga, gsa;
#pragma unroll
        for (int i = 0; i < L::Q; i++) { ga.v[i] = g[i]; gsa.v[i] = gs[i]; }
        ds = (double)delta_s_slow<L, T>(ga, gsa, T(P.rho0));
        if (P.recheck && isfinite(ds) && fabs(ds - P.delta) <= 1e-3 * fabs(P.delta))
            ds = delta_s_fp64<L, T, EQ>(ga, P.rho0);
    }
    const T nb2 = T(-2) * T(P.beta);
#pragma unroll
    for (int i = 0; i < L::Q; i++) g[i] = dfma<T>(nb2, d[i], g[i]);
    return ds;
}

// ---------------------------------------------------------------------------
// Global selection and Ehrenfests' step, run by one block: the last
// stream-collide block of a step, or the stand-alone select kernel.
//   mode 0: select among the candidates (or replay a given list), overwrite
//           the LBGK output of the selected sites with f* (Sec. 3.2; (ESLB)),
//           log the count and advance the step counter;
//   mode 1: select only (test hook).
// stage_key/stage_idx: shared memory for up to stage_cap candidates (larger
// candidate sets are ranked in place in global memory).
// ---------------------------------------------------------------------------
template <typename L, typename S, int EQ>
__device__ void select_and_fix(const Params& P, TopkScratch& sc, int& nsel_sh, unsigned& cnt_sh,
                               unsigned long long* stage_key, unsigned* stage_idx, int stage_cap,
                               int mode) {
    using T = typename Store<S>::T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long t = __ldcg(P.step);
    const long long r = t - P.replay_t0;
    const bool replay = P.replay_cnt && r >= 0 && r < P.replay_n;
    if (replay) {
        const int c = P.replay_cnt[r];
        const long long off = P.replay_off[r];
        for (int j = tid; j < c; j += nt) P.sel_idx[j] = P.replay_idx[off + j];
        if (tid == 0) nsel_sh = c;
    } else if (P.k <= 0) {
        if (tid == 0) nsel_sh = 0;
    } else {
        const int n = (int)__ldcg(P.cand_count);
        if (n <= P.k) {
            for (int j = tid; j < n; j += nt) P.sel_idx[j] = (int)__ldcg(P.cand_idx + j);
            if (tid == 0) nsel_sh = n;
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
            const Thresh th = block_topk(sc, n, P.k, keyat, idat);
            if (tid == 0) cnt_sh = 0;
            __syncthreads();
            for (int j = tid; j < n; j += nt) {
                const unsigned id = idat(j);
                if (th.selected(keyat(j), id)) {
                    const unsigned s = atomicAdd(&cnt_sh, 1u);
                    if (s < (unsigned)P.k) P.sel_idx[s] = (int)id;
                }
            }
            if (tid == 0) nsel_sh = P.k;
        }
    }
    __syncthreads();
    const int m = nsel_sh;
    if (mode == 0) {
        const long long nsites = (long long)P.nx * P.ny;
        for (int j = tid; j < m; j += nt) {
            const int site = P.sel_idx[j];
            if (site < 0 || site >= nsites) { atomicOr(P.err, ERR_REPLAY); continue; }
            const int x = site % P.nx, y = site / P.nx;
            if (is_solid(P, x, y)) { atomicOr(P.err, ERR_REPLAY); continue; }
            T g[L::Q], gs[L::Q], rho, ux, uy;
            gather_site<L, S>(P, x, y, g);
            site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
            const long long o = (long long)y * P.nxp + x;
#pragma unroll
            for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, gs[i]);
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

// End of a stream-collide block: publish this block's writes, take a ticket;
// the block that takes the last ticket runs the global selection and the
// Ehrenfests' step for the whole grid.  No block ever waits for another.
template <typename L, typename S, int EQ, int N>
__device__ __forceinline__ void finish_block(const Params& P, BlockCand<N>& sh) {
    // the barrier makes the block's writes visible to thread 0, whose
    // device-scope fence then orders all of them before the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nb = gridDim.x * gridDim.y;
        const unsigned tk = atomicAdd(P.ticket, 1u);
        __threadfence();
        sh.is_last = (tk == nb - 1);
    }
    __syncthreads();
    if (sh.is_last) {
        select_and_fix<L, S, EQ>(P, sh.sc, sh.nsel, sh.cnt2, sh.key, sh.idx, N, 0);
        if (threadIdx.x == 0) *P.ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// Vector loads and stores of VEC consecutive populations (aligned).
// ---------------------------------------------------------------------------
template <typename S, int VEC> struct VecIO;
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

template <typename S> struct VecIO<S, 1> {
    __device__ static void load(const void* p, long long i, typename Store<S>::T* v) {
        v[0] = Store<S>::load(p, i);
    }
    __device__ static void store(void* p, long long i, const typename Store<S>::T* v) {
        Store<S>::store(p, i, v[0]);
    }
};

// A tile [x0, x0 + TX) x [y0, y0 + TY) is interior when every site of the
// tile and of its one-site halo is fluid and inside the grid: its gather is
// then a pure shift with no boundary rule.
template <int TX, int TY>
__device__ __forceinline__ bool tile_interior(const Params& P, int x0, int y0) {
    if (x0 < 1 || x0 + TX > P.nx - 1 || y0 < 1 || y0 + TY > P.ny - 1) return false;
    if (P.ow > 0) {
        const bool apart = (x0 + TX + 1 <= P.ox0) || (x0 - 1 >= P.ox0 + P.ow) ||
                           (y0 + TY + 1 <= P.oy0) || (y0 - 1 >= P.oy0 + P.oh);
        if (!apart) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// K1 for D2Q9: one warp per row segment of 32 * VEC sites, ROWS rows per
// block.  Interior tiles: aligned VEC-wide loads per population plane, the
// x-shifted planes completed by one warp shuffle and one halo load per warp.
// Boundary tiles (and the first step after a state upload): per-site gather.
// ---------------------------------------------------------------------------
template <typename S, int EQ, int VEC, int ROWS, int MINB>
__global__ void __launch_bounds__(32 * ROWS, MINB) k_collide_d2q9(Params P) {
    using L = D2Q9;
    using T = typename Store<S>::T;
    constexpr int TX = 32 * VEC;
    constexpr int NS = 32 * ROWS * VEC;
    __shared__ BlockCand<NS> sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * ROWS;
    const int y = y0 + warp, xs = x0 + lane * VEC;
    if (threadIdx.x == 0) sh.count = 0;
    __syncthreads();
    const long long t = *P.step;
    bool nonfinite = false;
    if (!P.prestream && tile_interior<TX, ROWS>(P, x0, y0)) {
        T g[VEC][L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            const long long row = i * P.plane + (long long)(y - L::cy(i)) * P.nxp;
            T v[VEC];
            VecIO<S, VEC>::load(P.src, row + xs, v);
            if (L::cx(i) == 0) {
#pragma unroll
                for (int s = 0; s < VEC; s++) g[s][i] = v[s];
            } else if (L::cx(i) == 1) {
                // source x - 1: the previous lane's last element
                T prev = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
                if (lane == 0) prev = Store<S>::load(P.src, row + xs - 1);
                g[0][i] = prev;
#pragma unroll
                for (int s = 1; s < VEC; s++) g[s][i] = v[s - 1];
            } else {
                // source x + 1: the next lane's first element
                T next = __shfl_down_sync(0xffffffffu, v[0], 1);
                if (lane == 31) next = Store<S>::load(P.src, row + xs + VEC);
#pragma unroll
                for (int s = 0; s < VEC - 1; s++) g[s][i] = v[s + 1];
                g[VEC - 1][i] = next;
            }
        }
#pragma unroll
        for (int s = 0; s < VEC; s++) {
            const int x = xs + s;
            const double ds = update_site<L, T, EQ>(P, g[s], x, y, t, nonfinite);
            if (ds > P.delta) push_candidate(sh, ds, (unsigned)(y * P.nx + x));
        }
        const long long base = (long long)y * P.nxp + xs;
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            T v[VEC];
#pragma unroll
            for (int s = 0; s < VEC; s++) v[s] = g[s][i];
            VecIO<S, VEC>::store(P.dst, i * P.plane + base, v);
        }
    } else {
        // boundary tile (or the first step after a state upload): one site at
        // a time with the boundary rules
#pragma unroll 1
        for (int s = 0; s < VEC; s++) {
            const int x = xs + s;
            if (x >= P.nx || y >= P.ny) continue;
            const long long o = (long long)y * P.nxp + x;
            T g[L::Q];
            if (is_solid(P, x, y)) {
#pragma unroll
                for (int i = 0; i < L::Q; i++) g[i] = T(0);
            } else {
                gather_site<L, S>(P, x, y, g);
                const double ds = update_site<L, T, EQ>(P, g, x, y, t, nonfinite);
                if (ds > P.delta) push_candidate(sh, ds, (unsigned)(y * P.nx + x));
            }
#pragma unroll
            for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, g[i]);
        }
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if (P.k > 0) block_emit(P, sh);
    finish_block<L, S, EQ>(P, sh);
}

// ---------------------------------------------------------------------------
// K1, one site per thread (D1Q3).
// ---------------------------------------------------------------------------
template <typename L, typename S, int EQ>
__global__ void __launch_bounds__(kSiteBlock) k_collide_site(Params P) {
    using T = typename Store<S>::T;
    __shared__ BlockCand<kSiteBlock> sh;
    if (threadIdx.x == 0) sh.count = 0;
    const long long t = *P.step;
    const long long sid = (long long)blockIdx.x * kSiteBlock + threadIdx.x;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    const bool inside = sid < (long long)P.nx * P.ny;
    const bool valid = inside && !is_solid(P, x, y);
    bool nonfinite = false;
    T g[L::Q];
    if (valid) gather_site<L, S>(P, x, y, g);
    __syncthreads();
    if (valid) {
        const double ds = update_site<L, T, EQ>(P, g, x, y, t, nonfinite);
        if (ds > P.delta) push_candidate(sh, ds, (unsigned)sid);
    }
    if (inside) {
        const long long o = (long long)y * P.nxp + x;
#pragma unroll
        for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, valid ? g[i] : T(0));
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if (P.k > 0) block_emit(P, sh);
    finish_block<L, S, EQ>(P, sh);
}

// Stand-alone selection (select-only test hook).
template <typename L, typename S, int EQ>
__global__ void __launch_bounds__(kSelectThreads) k_select(Params P, int stage_cap, int mode) {
    extern __shared__ unsigned long long dyn[];
    __shared__ TopkScratch sc;
    __shared__ int nsel;
    __shared__ unsigned cnt;
    select_and_fix<L, S, EQ>(P, sc, nsel, cnt, dyn, reinterpret_cast<unsigned*>(dyn + stage_cap),
                             stage_cap, mode);
}

#ifdef LBM_DEFINE_EMIT_FROM_DS
// Candidates from a given dS array (select-only test hook): the same block
// stage as K1, 1024 values per block.
__global__ void __launch_bounds__(256) k_emit_from_ds(Params P, const double* ds, int n) {
    __shared__ BlockCand<1024> sh;
    if (threadIdx.x == 0) sh.count = 0;
    __syncthreads();
    const long long b = (long long)blockIdx.x * 1024;
    for (int s = threadIdx.x; s < 1024; s += 256) {
        const long long i = b + s;
        if (i < n && ds[i] > P.delta) push_candidate(sh, ds[i], (unsigned)i);
    }
    if (P.k > 0) block_emit(P, sh);
}
#endif

// ---------------------------------------------------------------------------
// State import / export and field kernels (one site per thread).
// ---------------------------------------------------------------------------

// Quasiequilibrium of given (rho, u) at every fluid site; zero elsewhere.
template <typename L, typename S, int EQ>
__global__ void k_init_eq(Params P, const double* rho, const double* ux, const double* uy) {
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
        const T r = T(rho[sid]), u = T(ux[sid]), v = uy ? T(uy[sid]) : T(0);
        equilibrium<L, T, EQ>(P, r - T(P.rho0), r, u, v, gs);
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++) Store<S>::store(P.dst, i * P.plane + o, gs[i]);
}

// FP64 populations [Q][ny][nx] -> deviation storage.
template <typename L, typename S>
__global__ void k_import(Params P, const double* f) {
    const long long N = (long long)P.nx * P.ny;
    const long long sid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= N) return;
    const int x = (int)(sid % P.nx), y = (int)(sid / P.nx);
    const long long o = (long long)y * P.nxp + x;
    const bool solid = is_solid(P, x, y);
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const double v = solid ? 0.0 : f[i * N + sid] - L::w(i) * P.rho0;
        Store<S>::store(P.dst, i * P.plane + o, (typename Store<S>::T)v);
    }
}

// Pre-collision state of the current step (gather of src), exported as
// mode 0: populations f [Q][ny][nx]; 1: rho, ux, uy, 2E; 2: exact dS.
template <typename L, typename S, int EQ>
__global__ void k_export(Params P, int mode, double* o0, double* o1, double* o2, double* o3) {
    using T = typename Store<S>::T;
    const long long N = (long long)P.nx * P.ny;
    const long long sid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= N) return;
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
        for (int i = 0; i < L::Q; i++) o0[i * N + sid] = (double)g[i] + L::w(i) * P.rho0;
    } else if (mode == 1) {
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
    } else {
        T gs[L::Q], rho, ux, uy;
        site_equilibrium<L, T, EQ>(P, g, gs, rho, ux, uy);
        o0[sid] = (double)delta_s_exact<L, T>(g, gs, T(P.rho0));
    }
}

// ---------------------------------------------------------------------------
// Launchers for one storage type.  Tile shapes of the D2Q9 kernel (sites per
// thread in x, rows per block = warps, minimum resident blocks per SM):
//   0: 1 x 8, 3     1: 1 x 8, 4     2: 2 x 8, 2     3: 4 x 8, 1
// ---------------------------------------------------------------------------

template <typename S, int EQ, int VEC, int ROWS, int MINB>
cudaError_t launch_d2q9(const Params& P, cudaStream_t st) {
    dim3 grid((P.nx + 32 * VEC - 1) / (32 * VEC), (P.ny + ROWS - 1) / ROWS);
    k_collide_d2q9<S, EQ, VEC, ROWS, MINB><<<grid, 32 * ROWS, 0, st>>>(P);
    return cudaGetLastError();
}

template <typename L, typename S, int EQ>
struct LaunchImpl {
    static cudaError_t collide(const Params& P, int shape, cudaStream_t st) {
        if constexpr (L::Q == 9) {
            switch (shape) {
                case 1: return launch_d2q9<S, EQ, 1, 8, 4>(P, st);
                case 2: return launch_d2q9<S, EQ, 2, 8, 2>(P, st);
                case 3: return launch_d2q9<S, EQ, 4, 8, 1>(P, st);
                default: return launch_d2q9<S, EQ, 1, 8, 3>(P, st);
            }
        } else {
            const long long N = (long long)P.nx * P.ny;
            const unsigned blocks = (unsigned)((N + kSiteBlock - 1) / kSiteBlock);
            k_collide_site<L, S, EQ><<<blocks, kSiteBlock, 0, st>>>(P);
            return cudaGetLastError();
        }
    }
    static cudaError_t select(const Params& P, int stage_cap, int mode, cudaStream_t st) {
        const size_t smem = (size_t)stage_cap * (sizeof(unsigned long long) + sizeof(unsigned));
        k_select<L, S, EQ><<<1, kSelectThreads, smem, st>>>(P, stage_cap, mode);
        return cudaGetLastError();
    }
    static cudaError_t init_eq(const Params& P, const double* rho, const double* ux,
                               const double* uy, const double*, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        k_init_eq<L, S, EQ><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, rho, ux, uy);
        return cudaGetLastError();
    }
    static cudaError_t import_state(const Params& P, const double* f, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        k_import<L, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, f);
        return cudaGetLastError();
    }
    static cudaError_t export_state(const Params& P, int mode, double* o0, double* o1, double* o2,
                                    double* o3, cudaStream_t st) {
        const long long N = (long long)P.nx * P.ny;
        k_export<L, S, EQ><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, mode, o0, o1, o2, o3);
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
        return l;
    }
};

template <typename S>
Launchers launchers_for(int lattice, int eq) {
    if (lattice == 0) {
        if (eq == EQ_POLY) return LaunchImpl<D1Q3, S, EQ_POLY>::get();
        return LaunchImpl<D1Q3, S, EQ_ENTROPIC>::get();
    }
    if (eq == EQ_POLY) return LaunchImpl<D2Q9, S, EQ_POLY>::get();
    return LaunchImpl<D2Q9, S, EQ_ENTROPIC>::get();
}

}  // namespace lbm
