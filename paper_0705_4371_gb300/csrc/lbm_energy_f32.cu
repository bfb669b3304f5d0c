// Kernel instantiations of the energy-constrained equilibria for storage
// type float.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f32_energy(int eq) { return launchers_energy<float>(eq); }
}  // namespace lbm
