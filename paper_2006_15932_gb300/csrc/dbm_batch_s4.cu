// dbm_batch_s4.cu -- batched step kernels instantiated for 4 species.
#include "dbm_batch_impl.cuh"

namespace dbm {
template BatchKernel batch_kernel_s<4>(int);
}  // namespace dbm
