// dbm_step_s2.cu -- fused step instantiated for 2 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<2>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<2, tma_tile_x(2), tma_tile_y(2), 1, false>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<2, PAIR_TX, PAIR_TY, 2, false>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
template int launch_step_staged_t<2, STAGED_TX, STAGED_TY>(dbm_handle *, const CUtensorMap *, const CUtensorMap *,
                                                                const void *, void *, cudaStream_t);
}  // namespace dbm
