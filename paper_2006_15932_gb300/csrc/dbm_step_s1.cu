// dbm_step_s1.cu -- fused step instantiated for 1 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_t<1>(dbm_handle *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<1, tma_tile_x(1), tma_tile_y(1), 1, false>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
}  // namespace dbm
