// dbm_aux_s2.cu -- the output and initialisation launches for 2 species.
#include "dbm_aux_impl.cuh"

namespace dbm {
template void aux_set_state<2>(dbm_handle *, void *, const double *, const double *, const double *, const double *,
                                cudaStream_t);
template void aux_moments<2>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_noneq<2>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_cons<2>(dbm_handle *, const void *, double *, double *, cudaStream_t);
}  // namespace dbm
