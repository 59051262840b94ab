// dbm_step_s6.cu -- fused step instantiated for 6 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<6>(dbm_handle *, const void *, void *, cudaStream_t);
}  // namespace dbm
