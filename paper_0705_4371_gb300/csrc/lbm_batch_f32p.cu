// lbm_batch_f32p.cu -- batched stream-collide kernels, plain FP32 storage.
#include "lbm_batch_kernels.cuh"

namespace lbm {

BatchLaunchers batch_launchers_f32p(int eq, int variant) {
    if (eq == EQ_ENTROPIC) return batch_launchers_of<plain32, EQ_ENTROPIC>(variant);
    return batch_launchers_of<plain32, EQ_POLY>(variant);
}

}  // namespace lbm
