// lbm_internal.h -- launcher table between the C-ABI host code and the
// per-storage-type kernel translation units (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

struct lb_handle;

namespace lbm {

struct Params;

struct Launchers {
    cudaError_t (*collide)(const Params&, int tile_shape, const void* tensor_map, cudaStream_t);
    cudaError_t (*select)(const Params&, int stage_cap, int mode, cudaStream_t);
    cudaError_t (*init_eq)(const Params&, const double* rho, const double* ux, const double* uy,
                           const double* e2, cudaStream_t);
    // planes [i0, i1) of an FP64 state [Q][ny][nx] -> storage
    cudaError_t (*import_state)(const Params&, const double* f, int i0, int i1, cudaStream_t);
    // sites [s0, s1) (index y nx + x) of the pre-collision state, exported
    cudaError_t (*export_state)(const Params&, int mode, double*, double*, double*, double*,
                                long long s0, long long s1, cudaStream_t);
    cudaError_t (*set_smem)(int stage_cap);
    // slab ghost exchange: column col of field <-> packed buffer [3][ny]
    cudaError_t (*ghost)(const Params&, void* field, int col, int right, void* buf, int dir, cudaStream_t);
    cudaError_t (*occupancy)(int tile_shape, int* blocks_per_sm);
};

// storage: FP64, FP32 deviation, FP16 deviation, plain FP32 (f32p)
Launchers launchers_f64(int lattice, int eq);
Launchers launchers_f32(int lattice, int eq);
Launchers launchers_f16(int lattice, int eq);
Launchers launchers_f32p(int lattice, int eq);
// energy-constrained equilibria (D2Q9), one translation unit per storage
Launchers launchers_f64_energy(int eq);
Launchers launchers_f32_energy(int eq);
Launchers launchers_f16_energy(int eq);
Launchers launchers_f32p_energy(int eq);

constexpr int kTileShapes = 7;   // tile shapes of the D2Q9 stream-collide kernel

// Candidates the stand-alone select kernel stages in shared memory (its
// dynamic shared-memory limit is set from this one value by every caller).
constexpr int kSelectStageCap = 8192;

// Rows and columns per block tile of the shared-memory-staged shapes
// (rows 0: not staged).
inline int staged_rows(int tile_shape) {
    return tile_shape == 4 || tile_shape == 6 ? 8 : (tile_shape == 5 ? 6 : 0);
}
inline int staged_cols(int tile_shape) { return tile_shape == 6 ? 64 : 128; }

// message returned by lb_last_error on this thread
void set_last_error(const char* msg);

// select-only test hook: candidates from a device dS array
cudaError_t launch_emit_from_ds(const Params& P, const double* ds, int n, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batched form: many D2Q9 runs advanced by one kernel launch per step.
// ---------------------------------------------------------------------------

// Arguments of one batched step (device pointers).  The run parameters,
// tensor maps and counters of a step are selected by its buffer parity.
struct BatchArgs {
    const Params* P;               // [nruns] the runs' parameters for this step
    const CUtensorMap* tm;         // [nruns] tensor maps of the source buffers (64-byte aligned)
    const int* tile_base;          // [nruns + 1] first work item of each run in the flat list
    int nruns, total_tiles;        // total_tiles: work items (edge items and tiles) of all runs
    unsigned* tile_counter;        // this step's item counter (reset by the step's select launch)
};

struct BatchLaunchers {
    cudaError_t (*launch)(const BatchArgs&, int grid, cudaStream_t);
    cudaError_t (*setup)(int* blocks_per_sm);
    int rows;                      // tile rows (the tile is 128 sites wide)
};

// Launch strategies of a batch step: 0 and 1 = the batched kernel with
// 8-row tiles and 2 stages, or 4-row tiles and 3 stages; 2 = every run's own
// stream-collide kernel, in concurrent branches (one stream per run).
constexpr int kBatchVariants = 3;
constexpr int kBatchKernelVariants = 2;
// storage: 0 = FP64, 1 = FP32 deviation, 2 = FP16 deviation, 3 = plain
// FP32; eq: EQ_POLY or EQ_ENTROPIC
BatchLaunchers batch_launchers(int storage, int eq, int variant);
BatchLaunchers batch_launchers_f64(int eq, int variant);
BatchLaunchers batch_launchers_f32(int eq, int variant);
BatchLaunchers batch_launchers_f16(int eq, int variant);
BatchLaunchers batch_launchers_f32p(int eq, int variant);

// A run as the batch sees it (lbm_api.cu).
struct RunView {
    int lattice, nx, ny, eq, prec, cur;
    bool prestream, replaying;
    long long step;
    cudaStream_t stream;
};
RunView run_view(const lb_handle* h);
Params run_params(const lb_handle* h, int src, bool prestream);
int run_tensor_map(const lb_handle* h, int buf, int rows, CUtensorMap* out);
void run_advance(lb_handle* h, long long n);
// One step of the run on stream st (its own kernel and tile shape).
int run_queue_step(lb_handle* h, int src, bool prestream, cudaStream_t st);
int run_check(lb_handle* h);
int run_queue_err(lb_handle* h);
int run_fail(int code, const char* msg);

}  // namespace lbm
