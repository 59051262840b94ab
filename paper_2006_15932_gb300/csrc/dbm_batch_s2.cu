// dbm_batch_s2.cu -- batched step kernels instantiated for 2 species.
#include "dbm_batch_impl.cuh"

namespace dbm {
template BatchKernel batch_kernel_s<2>(int);
}  // namespace dbm
