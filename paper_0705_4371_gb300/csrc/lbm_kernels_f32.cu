// Kernel instantiations for storage type float.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f32(int lattice, int eq) {
    if (lattice == 1 && eq >= EQ_ENERGY) return launchers_f32_energy(eq);
    return launchers_basic<float>(lattice, eq);
}
}  // namespace lbm
