// dbm_step_s3.cu -- fused step instantiated for 3 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<3>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<3, tma_tile_x(3), tma_tile_y(3), 1, false>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<3, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
