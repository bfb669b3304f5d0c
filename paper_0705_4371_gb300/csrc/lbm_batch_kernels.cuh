// lbm_batch_kernels.cuh -- the batched form: one launch advances every run
// of a batch by one time step.
//
// The runs' work items (their x = 0 and x = nx - 1 columns, then their block
// tiles of R rows x 128 sites, staged in shared memory by bulk tensor copies
// exactly as in the single-run staged kernel: each plane's window is the R
// rows the tile pulls from it) form one flat list; a persistent grid takes
// items from a global counter, so small and large runs share the GPU without
// idle tails per run.  A tile's sites go through the same per-site update
// as a single run (tma_tile); the sites the dS bound does not clear are
// resolved in place, and the candidates go straight to their run's global
// list.  One block barrier per item.  A second launch (k_batch_select, one
// block per run) then runs every run's selection and Ehrenfests' step
// (Sec. 3.2) and resets the step's item counter.
#pragma once

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kBatchStage = 512;   // candidates a select stages in shared memory
constexpr int kBatchSmemRuns = 256;   // tile bases kept in shared memory (more runs: global)

struct BatchShared {
    int abort;
    int tile[4];   // per stage: item of its run (-1: none left; -2 - e: edge item e)
    int base[kBatchSmemRuns + 1];   // first item of each run (batches of up to kBatchSmemRuns runs)
    int dims[kBatchSmemRuns][2];    // nx, ny of each run
};
static_assert(sizeof(Params) % 16 == 0, "Params is copied by a bulk copy (16-byte multiples)");

// Bulk copy of bytes (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <typename S, int R, int STAGES>
constexpr size_t batch_params_offset() {
    return ((size_t)STAGES * TmaLayout<S, R>::STAGE_BYTES + 8 * STAGES + sizeof(BatchShared) + 15) / 16 * 16;
}

template <typename S, int R, int STAGES>
constexpr size_t batch_smem_bytes() {
    return 128 + batch_params_offset<S, R, STAGES>() + (size_t)STAGES * sizeof(Params);
}

template <typename S, int EQ, int R, int STAGES>
__global__ void __launch_bounds__(32 * R, 16 / R) k_collide_batch(const __grid_constant__ BatchArgs A) {
    using L = D2Q9;
    using LY = TmaLayout<S, R>;
    constexpr int TX = kTmaTX;
    static_assert(STAGES <= 4, "at most 4 stages");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    S* stages = reinterpret_cast<S*>(smem);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + STAGES * LY::STAGE_BYTES);
    BatchShared& sh = *reinterpret_cast<BatchShared*>(smem + STAGES * LY::STAGE_BYTES + 8 * STAGES);
    Params* sp = reinterpret_cast<Params*>(smem + batch_params_offset<S, R, STAGES>());
    MlpSlot<EQ> mslot;   // empty: the batch runs the polynomial and entropic forms
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; st++) mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.abort = 0;
    }
    const bool base_in_smem = A.nruns <= kBatchSmemRuns;
    if (base_in_smem)
        for (int q = threadIdx.x; q <= A.nruns; q += blockDim.x) {
            sh.base[q] = A.tile_base[q];
            if (q < A.nruns) {
                sh.dims[q][0] = A.P[q].nx;
                sh.dims[q][1] = A.P[q].ny;
            }
        }
    __syncthreads();
    const int* tile_base = base_in_smem ? sh.base : A.tile_base;
    int run_hint = 0;   // tiles are claimed in increasing order: runs only move forward

    // Thread 0 takes the item it claimed at the previous refill and claims
    // the next (the atomic's latency then overlaps an item's computation),
    // issues a bulk copy of the item's run parameters into the stage's slot
    // and the tile's copies, all completing on the stage's mbarrier (-1: no
    // item left; the phase then completes by a plain arrive).  The run's nx
    // and ny, which place the tile, come from a table in shared memory.
    int next_item = 0;   // claimed at the previous refill (the atomic's latency overlaps an item)
    auto fill = [&](int st) {
        unsigned long long* bar = &full[st];
        const int tile = next_item;
        if (tile >= A.total_tiles) {
            sh.tile[st] = -1;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
            return;
        }
        next_item = (int)atomicAdd(A.tile_counter, 1u);
        int lo = run_hint;   // the last run whose first tile is <= tile
        while (tile_base[lo + 1] <= tile) lo++;
        run_hint = lo;
        // a run's work: its edge items (the x = 0 and x = nx - 1 columns,
        // 32 R sites each), then its tiles
        const int nx = base_in_smem ? sh.dims[lo][0] : A.P[lo].nx;
        const int ny = base_in_smem ? sh.dims[lo][1] : A.P[lo].ny;
        const int edge_items = ((nx > 1 ? 2 : 1) * ny + 32 * R - 1) / (32 * R);
        int lt = tile - tile_base[lo];
        if (lt < edge_items) {
            sh.tile[st] = -2 - lt;
            mbar_expect_tx(bar, (unsigned)sizeof(Params));
            bulk_copy_g2s(sp + st, A.P + lo, (unsigned)sizeof(Params), bar);
            return;
        }
        lt -= edge_items;
        sh.tile[st] = lt;
        const int tiles_x = (nx + TX - 1) / TX;
        const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
        mbar_expect_tx(bar, (unsigned)(LY::TX_BYTES + sizeof(Params)));
        bulk_copy_g2s(sp + st, A.P + lo, (unsigned)sizeof(Params), bar);
        S* base = stages + (size_t)st * (LY::STAGE_BYTES / sizeof(S));
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            tma_load_3d(base + i * LY::PLANE, A.tm + lo, tx * TX - LY::H, ty * R - L::cy(i), i, bar);
    };
    if (threadIdx.x == 0) {
        next_item = (int)atomicAdd(A.tile_counter, 1u);
        for (int st = 0; st < STAGES - 1; st++) fill(st);
    }
    int jj = 0;
    for (;; jj++) {
        const int st = jj % STAGES;
        const unsigned parity = (unsigned)((jj / STAGES) & 1);
        // the barrier also ends every warp's reads of the stage and the
        // parameter slot that thread 0 refills next
        if (__syncthreads_or(!mbar_wait(&full[st], parity))) {
            if (threadIdx.x == 0) {
                for (int q = 0; q < A.nruns; q++) atomicOr(A.P[q].err, ERR_TIMEOUT);
                sh.abort = 1;
            }
            break;
        }
        const int lt = sh.tile[st];
        if (lt == -1) break;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fill((jj + STAGES - 1) % STAGES);
        }
        const Params& P = sp[st];
        const int tiles_x = (P.nx + TX - 1) / TX;
        const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
        const long long t = __ldcg(P.step);
        bool nonfinite = false;
        NewtonCount nc = {0, 0, 0, 0};
        const S* box = stages + (size_t)st * (LY::STAGE_BYTES / sizeof(S));
        GlobalCandSink sink;
        if (lt <= -2) edge_item<S, EQ, R>(P, -2 - lt, t, sink, mslot, nonfinite, nc);
        else tma_tile<S, EQ, R, kTmaTX, true>(P, box, tx * TX, ty * R, t, sink, mslot, nonfinite, nc, P);
        if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    }
    __syncthreads();
    if (sh.abort && threadIdx.x == 0) {
        // wait (bounded) for copies still in flight into every stage
        for (int k2 = 0; k2 < STAGES; k2++) {
            const int j2 = jj + k2;
            mbar_wait(&full[j2 % STAGES], (unsigned)((j2 / STAGES) & 1));
        }
    }
}

// Every run's selection and Ehrenfests' step after the batched stream-collide
// launch (block r: run r; the parameters staged in shared memory); block 0
// resets the step's item counter.
template <typename S, int EQ>
__global__ void __launch_bounds__(256) k_batch_select(const __grid_constant__ BatchArgs A) {
    __shared__ SelectShared ss;
    __shared__ unsigned long long skey[kBatchStage];
    __shared__ unsigned sidx[kBatchStage];
    __shared__ __align__(16) Params ps;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(A.P + blockIdx.x);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&ps);
    for (int k = threadIdx.x; k < (int)(sizeof(Params) / 8); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    select_and_fix<D2Q9, S, EQ>(ps, ss, skey, sidx, kBatchStage, 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.tile_counter = 0u;
}

template <typename S, int EQ, int R, int STAGES>
cudaError_t launch_batch(const BatchArgs& A, int grid, cudaStream_t st) {
    k_collide_batch<S, EQ, R, STAGES><<<grid, 32 * R, batch_smem_bytes<S, R, STAGES>(), st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_batch_select<S, EQ><<<A.nruns, 256, 0, st>>>(A);
    return cudaGetLastError();
}

template <typename S, int EQ, int R, int STAGES>
cudaError_t setup_batch(int* per_sm) {
    constexpr size_t smem = batch_smem_bytes<S, R, STAGES>();
    cudaError_t e = cudaFuncSetAttribute(k_collide_batch<S, EQ, R, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_collide_batch<S, EQ, R, STAGES>, 32 * R,
                                                         smem);
}

template <typename S, int EQ>
BatchLaunchers batch_launchers_of(int variant) {
    BatchLaunchers b;
    if (variant == 1) {
        b.launch = &launch_batch<S, EQ, 4, 3>;
        b.setup = &setup_batch<S, EQ, 4, 3>;
        b.rows = 4;
    } else {
        b.launch = &launch_batch<S, EQ, 8, 2>;
        b.setup = &setup_batch<S, EQ, 8, 2>;
        b.rows = 8;
    }
    return b;
}

}  // namespace lbm
