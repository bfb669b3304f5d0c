// Kernel instantiations for storage type __half.
#include "lbm_kernels.cuh"

namespace lbm {
Launchers launchers_f16(int lattice, int eq) { return launchers_for<__half>(lattice, eq); }
}  // namespace lbm
