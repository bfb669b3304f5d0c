// Kernel instantiations of the energy-constrained equilibria for storage
// type double.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f64_energy(int eq) { return launchers_energy<double>(eq); }
}  // namespace lbm
