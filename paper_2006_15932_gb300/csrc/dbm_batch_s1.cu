// dbm_batch_s1.cu -- batched step kernels instantiated for 1 species.
#include "dbm_batch_impl.cuh"

namespace dbm {
template BatchKernel batch_kernel_s<1>(int);
}  // namespace dbm
