// Kernel instantiations for plain FP32 storage (plain32).
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f32p(int lattice, int eq) {
    if (lattice == 1 && eq >= EQ_ENERGY) return launchers_f32p_energy(eq);
    return launchers_basic<plain32>(lattice, eq);
}
}  // namespace lbm
