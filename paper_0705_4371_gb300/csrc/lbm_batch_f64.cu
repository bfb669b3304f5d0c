// lbm_batch_f64.cu -- batched stream-collide kernels, FP64 storage.
#include "lbm_batch_kernels.cuh"

namespace lbm {

BatchLaunchers batch_launchers_f64(int eq, int variant) {
    if (eq == EQ_ENTROPIC) return batch_launchers_of<double, EQ_ENTROPIC>(variant);
    return batch_launchers_of<double, EQ_POLY>(variant);
}

}  // namespace lbm
