// Kernel instantiations for storage type double.
#define LBM_DEFINE_EMIT_FROM_DS
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f64(int lattice, int eq) {
    if (lattice == 1 && eq >= EQ_ENERGY) return launchers_f64_energy(eq);
    return launchers_basic<double>(lattice, eq);
}
}  // namespace lbm

namespace lbm {
cudaError_t launch_emit_from_ds(const Params& P, const double* ds, int n, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + kEmitPerBlock - 1) / kEmitPerBlock);
    k_emit_from_ds<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(P, ds, n);
    return cudaGetLastError();
}
}  // namespace lbm
