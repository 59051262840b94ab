// dbm_step_s4.cu -- fused step instantiated for 4 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<4>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<4, tma_tile_x(4), tma_tile_y(4), 1, false>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<4, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
