// dbm_step_s8.cu -- fused step instantiated for 8 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<8>(dbm_handle *, const void *, void *, cudaStream_t);
}  // namespace dbm
