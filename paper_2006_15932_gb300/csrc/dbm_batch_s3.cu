// dbm_batch_s3.cu -- batched step kernels instantiated for 3 species.
#include "dbm_batch_impl.cuh"

namespace dbm {
template BatchKernel batch_kernel_s<3>(int);
}  // namespace dbm
