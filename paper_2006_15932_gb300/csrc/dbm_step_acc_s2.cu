// dbm_step_acc_s2.cu -- the fused step with the FP32 arithmetic options
// (FP64 thermo, stochastic rounding) instantiated for 2 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_tma_t<2, tma_tile_x(2), tma_tile_y(2), 1, true>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
template int launch_step_tma_t<2, PAIR_TX, PAIR_TY, 2, true>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
}  // namespace dbm
