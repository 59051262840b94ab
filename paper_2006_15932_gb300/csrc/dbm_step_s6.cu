// dbm_step_s6.cu -- fused step instantiated for 6 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<6>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<6, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
