// lbm_batch_f32.cu -- batched stream-collide kernels, FP32 storage.
#include "lbm_batch_kernels.cuh"

namespace lbm {

BatchLaunchers batch_launchers_f32(int eq, int variant) {
    if (eq == EQ_ENTROPIC) return batch_launchers_of<float, EQ_ENTROPIC>(variant);
    return batch_launchers_of<float, EQ_POLY>(variant);
}

}  // namespace lbm
