// Kernel instantiations of the energy-constrained equilibria for storage
// type __half.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f16_energy(int eq) { return launchers_energy<__half>(eq); }
}  // namespace lbm
