// dbm_step.cu -- dispatch of the fused step on precision, species count and
// kernel variant, and the TMA descriptors of the state buffers.  The
// kernels are in dbm_step_impl.cuh, instantiated once per species count in
// dbm_step_s<S>.cu so that the units compile in parallel.
#include <string.h>

#include "dbm_internal.h"

namespace dbm {

template <int S>
int launch_step_t(dbm_handle *h, const void *fin, void *fout, cudaStream_t st);
template <int S, int TX, int TY, int CW, bool ACC>
int launch_step_tma_t(dbm_handle *h, const CUtensorMap *tmap, const void *fin, void *fout, cudaStream_t st);
template <int S, int TX, int TY>
int launch_step_staged_t(dbm_handle *h, const CUtensorMap *tmap, const CUtensorMap *tmap_in, const void *fin,
                         void *fout, cudaStream_t st);

// The species-staged step of the handle's tile (no arithmetic options).
static int launch_staged(dbm_handle *h, int cur, const void *fin, void *fout, cudaStream_t st)
{
    const CUtensorMap *tm = &h->tmap[cur], *ti = &h->tmap_in[cur];
    switch (h->p.nspecies) {
    case 2: return launch_step_staged_t<2, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 3: return launch_step_staged_t<3, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 4: return launch_step_staged_t<4, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 5: return launch_step_staged_t<5, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 6: return launch_step_staged_t<6, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 7: return launch_step_staged_t<7, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    case 8: return launch_step_staged_t<8, STAGED_TX, STAGED_TY>(h, tm, ti, fin, fout, st);
    }
    return DBM_ERR_INVALID;
}

// The TMA-staged step of the handle's tile, with (ACC) or without the FP32
// arithmetic options.
template <bool ACC>
static int launch_tma(dbm_handle *h, const CUtensorMap *tm, const void *fin, void *fout, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: return launch_step_tma_t<1, tma_tile_x(1), tma_tile_y(1), 1, ACC>(h, tm, fin, fout, st);
    case 2:
        if (h->tma_cw == 2) return launch_step_tma_t<2, PAIR_TX, PAIR_TY, 2, ACC>(h, tm, fin, fout, st);
        return launch_step_tma_t<2, tma_tile_x(2), tma_tile_y(2), 1, ACC>(h, tm, fin, fout, st);
    case 3: return launch_step_tma_t<3, tma_tile_x(3), tma_tile_y(3), 1, ACC>(h, tm, fin, fout, st);
    case 4: return launch_step_tma_t<4, tma_tile_x(4), tma_tile_y(4), 1, ACC>(h, tm, fin, fout, st);
    }
    return DBM_ERR_INVALID;
}

// The all-species TMA-staged kernels exist for FP32 with up to four species;
// the species-staged one for two to eight species without the arithmetic
// options.
bool tma_supported(const dbm_params &p) { return p.precision == DBM_FP32 && p.nspecies <= 4; }
static bool staged_supported(const dbm_params &p)
{
    return p.precision == DBM_FP32 && p.nspecies >= 2 && p.nspecies <= DBM_MAX_SPECIES && !uses_acc(p);
}

// The tile of the TMA-staged step.  Two species: two cells per thread when
// asked for, or (DBM_KERNEL_AUTO / DBM_KERNEL_TMA) on grids of at least
// PAIR_MIN_TILES pair tiles, else the one-cell tile.  Three and four
// species: the one-cell tile (faster than the species-staged kernel on every
// grid measured), the species-staged one when two cells per thread are asked
// for.  Five or more: the species-staged kernel, the only TMA-staged one.
static void choose_tile(dbm_handle *h)
{
    const dbm_params &p = h->p;
    const int want = p.step_kernel;
    h->tma_staged = 0;
    const bool staged_by_default = p.nspecies > 4 && want != DBM_KERNEL_TMA_CELL;
    const bool staged_asked = want == DBM_KERNEL_TMA_STAGED || (p.nspecies >= 3 && want == DBM_KERNEL_TMA_PAIR);
    if (staged_supported(p) && (staged_by_default || staged_asked)) {
        h->tma_staged = 1;
        h->tma_tx = STAGED_TX;
        h->tma_ty = STAGED_TY;
        h->tma_cw = 2;
        return;
    }
    bool pair = false;
    if (p.nspecies == 2 && want != DBM_KERNEL_TMA_CELL) {
        const long long tiles = (long long)((p.nx + PAIR_TX - 1) / PAIR_TX) * ((p.ny + PAIR_TY - 1) / PAIR_TY);
        pair = want == DBM_KERNEL_TMA_PAIR || tiles >= PAIR_MIN_TILES;
    }
    h->tma_tx = pair ? PAIR_TX : tma_tile_x(p.nspecies);
    h->tma_ty = pair ? PAIR_TY : tma_tile_y(p.nspecies);
    h->tma_cw = pair ? 2 : 1;
}

typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

// One 3-D descriptor per state buffer: (column, row, plane) with the whole
// padded geometry; out-of-range boxes are zero-filled by the copy engine.
int make_tensor_maps(dbm_handle *h)
{
    h->tma_ok = 0;
    h->tma_tx = h->tma_ty = h->tma_cw = h->tma_staged = 0;
    if (!tma_supported(h->p) && !staged_supported(h->p)) return DBM_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return DBM_OK;  // no TMA descriptors: the generic kernel runs
    }
    encode_tiled_fn encode = (encode_tiled_fn)fn;
    const dbm_layout &L = h->lay;
    cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)(16 * h->p.nspecies)};
    cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
    choose_tile(h);
    if (!h->tma_staged && !tma_supported(h->p)) {  // no all-species kernel for this species count
        h->tma_tx = h->tma_ty = h->tma_cw = 0;
        return DBM_OK;
    }
    // the box: the tile, its halo and every plane (one species' planes for
    // the species-staged kernel)
    const cuuint32_t planes = (cuuint32_t)(h->tma_staged ? Q : Q * h->p.nspecies);
    cuuint32_t box[3] = {(cuuint32_t)(h->tma_tx + 8), (cuuint32_t)(h->tma_ty + 4), planes};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        CUresult r = encode(&h->tmap[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->f[k], dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS && h->tma_staged) {  // interior box of one species: the moment-sum copies
            cuuint32_t box_in[3] = {(cuuint32_t)h->tma_tx, (cuuint32_t)h->tma_ty, (cuuint32_t)Q};
            r = encode(&h->tmap_in[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->f[k], dims, strides, box_in, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
        if (r != CUDA_SUCCESS) {
            h->tma_tx = h->tma_ty = h->tma_cw = h->tma_staged = 0;
            return DBM_OK;
        }
    }
    h->tma_ok = 1;
    return DBM_OK;
}

static int launch_generic(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: return launch_step_t<1>(h, fin, fout, st);
    case 2: return launch_step_t<2>(h, fin, fout, st);
    case 3: return launch_step_t<3>(h, fin, fout, st);
    case 4: return launch_step_t<4>(h, fin, fout, st);
    case 5: return launch_step_t<5>(h, fin, fout, st);
    case 6: return launch_step_t<6>(h, fin, fout, st);
    case 7: return launch_step_t<7>(h, fin, fout, st);
    case 8: return launch_step_t<8>(h, fin, fout, st);
    }
    return DBM_ERR_INVALID;
}

int launch_step(dbm_handle *h, int cur, cudaStream_t st)
{
    const void *fin = h->f[cur];
    void *fout = h->f[cur ^ 1];
    const int want = h->p.step_kernel;
    if (h->tma_ok && want != DBM_KERNEL_GENERIC) {
        const CUtensorMap *tm = &h->tmap[cur];
        if (h->tma_staged) return launch_staged(h, cur, fin, fout, st);
        return uses_acc(h->p) ? launch_tma<true>(h, tm, fin, fout, st) : launch_tma<false>(h, tm, fin, fout, st);
    }
    if (uses_acc(h->p)) return DBM_ERR_INVALID;  // the options exist in the TMA-staged kernel only
    if (want != DBM_KERNEL_AUTO && want != DBM_KERNEL_GENERIC) return DBM_ERR_INVALID;
    if (h->p.precision == DBM_BF16DEV) return launch_step_bf16(h, cur, st);
    if (h->p.precision == DBM_FP64) return launch_step_f64(h, cur, st);
    if (h->p.precision == DBM_FP32) return launch_generic(h, fin, fout, st);
    return DBM_ERR_INVALID;
}

}  // namespace dbm
