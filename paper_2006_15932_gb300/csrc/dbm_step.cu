// dbm_step.cu -- dispatch of the fused step on precision and species count;
// the kernel itself is in dbm_step_impl.cuh, instantiated once per species
// count in dbm_step_s<S>.cu so that the units compile in parallel.
#include "dbm_internal.h"

namespace dbm {

template <typename real, int S>
int launch_step_t(dbm_handle *h, const void *fin, void *fout, cudaStream_t st);

template <typename real>
static int launch_step_p(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: return launch_step_t<real, 1>(h, fin, fout, st);
    case 2: return launch_step_t<real, 2>(h, fin, fout, st);
    case 3: return launch_step_t<real, 3>(h, fin, fout, st);
    case 4: return launch_step_t<real, 4>(h, fin, fout, st);
    case 5: return launch_step_t<real, 5>(h, fin, fout, st);
    case 6: return launch_step_t<real, 6>(h, fin, fout, st);
    case 7: return launch_step_t<real, 7>(h, fin, fout, st);
    case 8: return launch_step_t<real, 8>(h, fin, fout, st);
    }
    return DBM_ERR_INVALID;
}

int launch_step(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) return launch_step_p<double>(h, fin, fout, st);
    if (h->p.precision == DBM_FP32) return launch_step_p<float>(h, fin, fout, st);
    return DBM_ERR_INVALID;
}

}  // namespace dbm
