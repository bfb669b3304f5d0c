// Kernel instantiations of the energy-constrained equilibria for plain FP32
// storage (plain32).
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f32p_energy(int eq) { return launchers_energy<plain32>(eq); }
}  // namespace lbm
