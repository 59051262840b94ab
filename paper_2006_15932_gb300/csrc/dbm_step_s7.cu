// dbm_step_s7.cu -- fused step instantiated for 7 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<7>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<7, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
