// lbm_batch_f16.cu -- batched stream-collide kernels, FP16 deviation storage.
#include "lbm_batch_kernels.cuh"

namespace lbm {

BatchLaunchers batch_launchers_f16(int eq, int variant) {
    if (eq == EQ_ENTROPIC) return batch_launchers_of<__half, EQ_ENTROPIC>(variant);
    return batch_launchers_of<__half, EQ_POLY>(variant);
}

}  // namespace lbm
