// lbm_internal.h -- launcher table between the C-ABI host code and the
// per-storage-type kernel translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct Params;

struct Launchers {
    cudaError_t (*collide)(const Params&, int tile_shape, const void* tensor_map, cudaStream_t);
    cudaError_t (*select)(const Params&, int stage_cap, int mode, cudaStream_t);
    cudaError_t (*init_eq)(const Params&, const double* rho, const double* ux, const double* uy,
                           const double* e2, cudaStream_t);
    cudaError_t (*import_state)(const Params&, const double* f, cudaStream_t);
    cudaError_t (*export_state)(const Params&, int mode, double*, double*, double*, double*,
                                cudaStream_t);
    cudaError_t (*set_smem)(int stage_cap);
    cudaError_t (*occupancy)(int tile_shape, int* blocks_per_sm);
};

// storage: 0 = FP64, 1 = FP32 (plain and deviation), 2 = FP16 deviation
Launchers launchers_f64(int lattice, int eq);
Launchers launchers_f32(int lattice, int eq);
Launchers launchers_f16(int lattice, int eq);
// energy-constrained equilibria (D2Q9), one translation unit per storage
Launchers launchers_f64_energy(int eq);
Launchers launchers_f32_energy(int eq);
Launchers launchers_f16_energy(int eq);

constexpr int kTileShapes = 6;   // tile shapes of the D2Q9 stream-collide kernel

// Rows per block tile of the shared-memory-staged shapes (0: not staged).
inline int staged_rows(int tile_shape) { return tile_shape == 4 ? 8 : (tile_shape == 5 ? 4 : 0); }

// message returned by lb_last_error on this thread
void set_last_error(const char* msg);

// select-only test hook: candidates from a device dS array
cudaError_t launch_emit_from_ds(const Params& P, const double* ds, int n, cudaStream_t st);

}  // namespace lbm
