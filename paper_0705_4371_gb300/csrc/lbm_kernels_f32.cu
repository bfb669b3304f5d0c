// Kernel instantiations for storage type float.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f32(int lattice, int eq) { return launchers_for<float>(lattice, eq); }
}  // namespace lbm
