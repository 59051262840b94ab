// dbm_step_s5.cu -- fused step instantiated for 5 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<5>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<5, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
