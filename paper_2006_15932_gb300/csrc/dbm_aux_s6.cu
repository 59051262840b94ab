// dbm_aux_s6.cu -- the output and initialisation launches for 6 species.
#include "dbm_aux_impl.cuh"

namespace dbm {
template void aux_set_state<6>(dbm_handle *, void *, const double *, const double *, const double *, const double *,
                                cudaStream_t);
template void aux_moments<6>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_noneq<6>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_cons<6>(dbm_handle *, const void *, double *, double *, cudaStream_t);
}  // namespace dbm
