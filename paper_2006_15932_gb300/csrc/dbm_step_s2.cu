// dbm_step_s2.cu -- fused step instantiated for 2 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<2>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<2, 64, 8>(dbm_handle *, const CUtensorMap *, void *, cudaStream_t);
}  // namespace dbm
