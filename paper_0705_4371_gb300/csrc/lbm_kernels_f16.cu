// Kernel instantiations for storage type __half.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f16(int lattice, int eq) {
    if (lattice == 1 && eq >= EQ_ENERGY) return launchers_f16_energy(eq);
    return launchers_basic<__half>(lattice, eq);
}
}  // namespace lbm
