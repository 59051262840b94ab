// dbm_aux.cu -- initialisation, raw state transfer and FP64 output calls
// of the D2V16 DBM: f = f^eq from macroscopic fields, checkpoint load/read,
// the macroscopic fields, the nonequilibrium moments (Eqs. Delta2, Delta31,
// Delta3, Delta42) and the conserved totals.  The kernels and their
// per-species-count launches are in dbm_aux_impl.cuh (instantiated in
// dbm_aux_s<S>.cu); this unit dispatches on S.
#include <stdio.h>

#include <mutex>

#include "dbm_aux_impl.cuh"

namespace dbm {

template <int S>
void aux_set_state(dbm_handle *, void *, const double *, const double *, const double *, const double *, cudaStream_t);
template <int S>
void aux_moments(dbm_handle *, const void *, double *, cudaStream_t);
template <int S>
void aux_noneq(dbm_handle *, const void *, double *, cudaStream_t);
template <int S>
void aux_cons(dbm_handle *, const void *, double *, double *, cudaStream_t);

template <typename real>
__global__ void __launch_bounds__(256)
    k_set_f(real *__restrict__ f, const double *__restrict__ src, int nplanes, int nx, int ny,
            int pitch, long long plane, int bc_x, int bc_y)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const long long d = (long long)y * nx + x;
    const long long cell = (long long)(y + GY) * pitch + (x + GX);
    const Images im = cell_images(x, y, nx, ny, bc_x, bc_y);
    for (int p = 0; p < nplanes; ++p)
        store_with_images(f + p * plane, cell, x, y, pitch, im, (real)src[p * N + d]);
}

template <typename real>
__global__ void __launch_bounds__(256)
    k_get_f(const real *__restrict__ f, double *__restrict__ dst, int nplanes, int nx, int ny,
            int pitch, long long plane)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const long long d = (long long)y * nx + x;
    const long long cell = (long long)(y + GY) * pitch + (x + GX);
    for (int p = 0; p < nplanes; ++p) dst[p * N + d] = (double)f[p * plane + cell];
}

#define DBM_DISPATCH_S(S_, CALL)             \
    switch (S_) {                            \
    case 1: { constexpr int S = 1; CALL; } break; \
    case 2: { constexpr int S = 2; CALL; } break; \
    case 3: { constexpr int S = 3; CALL; } break; \
    case 4: { constexpr int S = 4; CALL; } break; \
    case 5: { constexpr int S = 5; CALL; } break; \
    case 6: { constexpr int S = 6; CALL; } break; \
    case 7: { constexpr int S = 7; CALL; } break; \
    case 8: { constexpr int S = 8; CALL; } break; \
    default: return DBM_ERR_INVALID;         \
    }

int launch_set_state(dbm_handle *h, void *f, const double *rho_s, const double *ux,
                     const double *uy, const double *T, cudaStream_t st)
{
    if (h->p.precision == DBM_BF16DEV) return launch_set_state_bf16(h, f, rho_s, ux, uy, T, st);
    DBM_DISPATCH_S(h->p.nspecies, (aux_set_state<S>(h, f, rho_s, ux, uy, T, st)));
    return set_cuda_error(h, cudaGetLastError(), "set_state kernel launch");
}

int launch_set_f(dbm_handle *h, void *f, const double *src, cudaStream_t st)
{
    dim3 b(32, 8);
    const int np = h->p.nspecies * Q;
    if (h->p.precision == DBM_FP64)
        k_set_f<double><<<cell_grid(h, b), b, 0, st>>>((double *)f, src, np, h->p.nx, h->p.ny,
                                                       h->lay.pitch, h->lay.plane, h->p.bc_x, h->p.bc_y);
    else if (h->p.precision == DBM_FP32)
        k_set_f<float><<<cell_grid(h, b), b, 0, st>>>((float *)f, src, np, h->p.nx, h->p.ny,
                                                      h->lay.pitch, h->lay.plane, h->p.bc_x, h->p.bc_y);
    else
        return launch_set_f_bf16(h, f, src, st);
    return set_cuda_error(h, cudaGetLastError(), "set_f kernel launch");
}

int launch_get_f(dbm_handle *h, const void *f, double *dst, cudaStream_t st)
{
    dim3 b(32, 8);
    const int np = h->p.nspecies * Q;
    if (h->p.precision == DBM_FP64)
        k_get_f<double><<<cell_grid(h, b), b, 0, st>>>((const double *)f, dst, np, h->p.nx, h->p.ny,
                                                       h->lay.pitch, h->lay.plane);
    else if (h->p.precision == DBM_FP32)
        k_get_f<float><<<cell_grid(h, b), b, 0, st>>>((const float *)f, dst, np, h->p.nx, h->p.ny,
                                                      h->lay.pitch, h->lay.plane);
    else
        return launch_get_f_bf16(h, f, dst, st);
    return set_cuda_error(h, cudaGetLastError(), "get_f kernel launch");
}

static bool bf_ok(const dbm_handle *h) { return h->p.precision != DBM_BF16DEV || h->p.nspecies <= 4; }

int launch_moments(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (!bf_ok(h)) return DBM_ERR_INVALID;
    DBM_DISPATCH_S(h->p.nspecies, (aux_moments<S>(h, f, out, st)));
    return set_cuda_error(h, cudaGetLastError(), "moments kernel launch");
}

int launch_noneq(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (!bf_ok(h)) return DBM_ERR_INVALID;
    DBM_DISPATCH_S(h->p.nspecies, (aux_noneq<S>(h, f, out, st)));
    return set_cuda_error(h, cudaGetLastError(), "nonequilibrium kernel launch");
}

// Conserved totals into `out` with the block partials in `partial`.
static int conservation_into(dbm_handle *h, const void *f, double *partial, double *out, cudaStream_t st)
{
    if (!bf_ok(h)) return DBM_ERR_INVALID;
    DBM_DISPATCH_S(h->p.nspecies, (aux_cons<S>(h, f, partial, out, st)));
    return DBM_OK;
}

int launch_conservation(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    double *partial = (double *)((char *)h->scratch + SCRATCH_HEAD);
    const int rc = conservation_into(h, f, partial, out, st);
    if (rc) return rc;
    return set_cuda_error(h, cudaGetLastError(), "conservation kernel launch");
}

// ---------------------------------------------------------------------------
// Conserved totals without a caller-provided scratch buffer.
//
// Some callers cannot allocate device memory at the point where they need
// the totals (for example a plug-in that runs inside a host application
// which owns all of the GPU's memory and forbids further allocations).  For
// them the block partials of the reduction live in this file-scope device
// array instead of the caller's scratch buffer.  Every GPU that loads the
// library holds the array until the process exits.  Host code must not
// pass the array's name to a kernel (on the host it is only a stand-in):
// its device address is looked up once per device with cudaGetSymbolAddress
// and cached.
// ---------------------------------------------------------------------------

static __device__ __align__(256) double g_noalloc_partials[DBM_NOALLOC_SCRATCH_DOUBLES];

static const int NOALLOC_MAX_DEVICES = 64;
static double *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Device address of g_noalloc_partials on the current device (looked up on
// the first call per device, with that device current).
static int noalloc_scratch(dbm_handle *h, double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(h, e, "conservation_noalloc: current device");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        snprintf(h->err, sizeof(h->err),
                 "conservation_noalloc: device ordinal %d outside the %d devices whose array address is cached", dev,
                 NOALLOC_MAX_DEVICES);
        return DBM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return set_cuda_error(h, e, "conservation_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = (double *)ptr;
    }
    *out = g_noalloc_addr[dev];
    return DBM_OK;
}

int launch_conservation_noalloc(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    const size_t need = (size_t)CONS_BLOCKS * (h->p.nspecies + 4);
    if (need > DBM_NOALLOC_SCRATCH_DOUBLES) return DBM_ERR_INVALID;
    double *partial = nullptr;
    int rc = noalloc_scratch(h, &partial);
    if (rc) return rc;
    // every block overwrites all of its partials, so nothing needs clearing
    rc = conservation_into(h, f, partial, out, st);
    if (rc) return rc;
    return set_cuda_error(h, cudaGetLastError(), "conservation_noalloc kernel launch");
}

}  // namespace dbm
