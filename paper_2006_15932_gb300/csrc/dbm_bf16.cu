// dbm_bf16.cu -- the step and the state transfers of the BF16-deviation
// storage (see dbm_bf16.cuh).
//
// One CTA steps a TX x TY tile.  Phase A rebuilds f (FP32) of the tile and
// its radius-2 halo in shared memory from the stored moments and bfloat16
// deviations (a halo cell outside the domain from its periodic or outflow
// source cell); phase B runs the same per-cell FP32 arithmetic as the FP32
// kernels (step_cell) on that tile and stores delta^{n+1} and the
// reference moments, and no ghost cells.  Reactions and forces are not supported in this
// storage (their equilibrium is not the one of the stored moments); init
// rejects them.
#include "dbm_bf16.cuh"

namespace dbm {

// CTAs of the BF16 step's TX x TY tile that fit on one SM (shared memory for
// the rebuilt FP32 tile plus its radius-2 halo, at least 64 registers per
// cell), at most four.
constexpr int bf16_ctas_per_sm(int S, int TX, int TY)
{
    const int by_smem = (227 * 1024) / ((TX + 4) * (TY + 4) * S * 64 + 1024);
    const int by_regs = 65536 / (TX * TY * 64);
    const int n = by_smem < by_regs ? by_smem : by_regs;
    return n > 4 ? 4 : n < 1 ? 1 : n;
}

template <int S, int TX, int TY, int CW>
__global__ void __launch_bounds__(TX / CW * TY, bf16_ctas_per_sm(S, TX, TY))
    k_step_bf16(const __grid_constant__ StepConsts<float, S> c, BfState in, BfState out,
                unsigned *__restrict__ flag)
{
    constexpr int BX = TX + 4, BY = TY + 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);  // [16 S][BY][BX], column 0 = x0 - 2
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nthr = TX / CW * TY, tid = ty * (TX / CW) + tx;
    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;

    // phase A: rebuild f for the tile and its halo, one cell per iteration
    // (two cells per iteration in packed FP32x2 measured slower: 18.7
    // against 23.8 G/s on KH 4096^2); a halo cell outside the domain is
    // rebuilt from its source cell (periodic wrap, or the edge cell for
    // outflow), so the stored ghost cells are neither read nor written
    for (int k = tid; k < BX * BY; k += nthr) {
        const int rr = k / BX, cc = k % BX;
        const int x = bx0 - 2 + cc, y = by0 - 2 + rr;
        const bool ok = x <= c.nx + 1 && y <= c.ny + 1;  // within reach of the stencil
        const int xs = x >= 0 && x < c.nx ? x
                       : c.bc_x == DBM_BC_PERIODIC ? ((x % c.nx) + c.nx) % c.nx : min(max(x, 0), c.nx - 1);
        const int ys = y >= 0 && y < c.ny ? y
                       : c.bc_y == DBM_BC_PERIODIC ? ((y % c.ny) + c.ny) % c.ny : min(max(y, 0), c.ny - 1);
        const long long cell = (long long)(ys + GY) * c.pitch + (xs + GX);
        float *dst = tile + rr * BX + cc;
        const bool src_ok = ok && in_bounds(cell, in.P, flag);
#pragma unroll 1
        for (int s = 0; s < S; ++s) {
            float f[Q];
            if (src_ok) bf_cell_f<S>(c, in, s, cell, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) dst[(s * Q + i) * (BY * BX)] = src_ok ? f[i] : 0.0f;
        }
    }
    __syncthreads();

    // phase B: the step from shared memory, CW adjacent cells per thread
    const int x = bx0 + CW * tx, y = by0 + ty;
    if (x >= c.nx || y >= c.ny) return;
    const float *base = tile + (ty + 2) * BX + (CW * tx + 2);
    BfOut o{out, S, flag};
    if constexpr (CW == 2) {
        const SmemTile2 t{base, BY * BX, BX, tile, S * Q * BY * BX, flag};
        step_cell<S>(c, c, t, x, y, x + 1 < c.nx, o, flag);
    } else {
        const SmemTile t{base, BY * BX, BX, tile, S * Q * BY * BX, flag};
        step_cell<S>(c, c, t, x, y, true, o, flag);
    }
}

// State from macroscopic fields: reference moments n^s = rho^s/m^s, u, T
// and zero deviations.
template <int S>
__global__ void __launch_bounds__(256)
    k_set_state_bf16(BfState st, int nx, int ny, int pitch, int bc_x, int bc_y, const double *__restrict__ rho_s,
                     const double *__restrict__ ux, const double *__restrict__ uy, const double *__restrict__ T,
                     const __grid_constant__ OutConsts<S> oc)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny, d = (long long)y * nx + x;
    const long long cell = (long long)(y + GY) * pitch + (x + GX);
    const Images im = cell_images(x, y, nx, ny, bc_x, bc_y);
    for (int s = 0; s < S; ++s) {
        store_with_images(st.mom + (long long)s * st.P, cell, x, y, pitch, im, (float)(rho_s[s * N + d] / oc.m[s]));
        for (int i = 0; i < Q; ++i)
            store_with_images(st.d + (long long)(s * Q + i) * st.P, cell, x, y, pitch, im, __float2bfloat16_rn(0.0f));
    }
    store_with_images(st.mom + (long long)S * st.P, cell, x, y, pitch, im, (float)ux[d]);
    store_with_images(st.mom + (long long)(S + 1) * st.P, cell, x, y, pitch, im, (float)uy[d]);
    store_with_images(st.mom + (long long)(S + 2) * st.P, cell, x, y, pitch, im, (float)T[d]);
}

// State from raw distributions (FP64 dense): reference moments are the
// moments of f (species n^s; mixture u, T as the collision defines them,
// in FP64), deviations f - f^eq(moments) rounded to bfloat16.
template <int S>
__global__ void __launch_bounds__(128)
    k_set_f_bf16(const __grid_constant__ StepConsts<float, S> k, const __grid_constant__ OutConsts<S> oc, BfState st,
                 const double *__restrict__ src)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= oc.nx || y >= oc.ny) return;
    const long long N = (long long)oc.nx * oc.ny, d = (long long)y * oc.nx + x;
    const long long cell = (long long)(y + GY) * oc.pitch + (x + GX);
    const Images im = cell_images(x, y, oc.nx, oc.ny, oc.bc_x, oc.bc_y);
    double n[S], w = 0, wx = 0, wy = 0, we = 0, wd = 0;
    for (int s = 0; s < S; ++s) {
        double sn = 0, sx = 0, sy = 0, se = 0;
        for (int i = 0; i < Q; ++i) {
            const double v = src[(s * Q + i) * N + d];
            const int r = i >> 2;
            sn += v;
            sx += dir_x(i) * oc.vr[s][r] * v;
            sy += dir_y(i) * oc.vr[s][r] * v;
            se += oc.qr[s][r] * v;
        }
        n[s] = sn;
        const double mt = oc.m[s] * oc.inv_tau[s];
        w += mt * sn;
        wx += mt * sx;
        wy += mt * sy;
        we += mt * se;
        wd += oc.dpi[s] * oc.inv_tau[s] * sn;
    }
    const double Ux = wx / w, Uy = wy / w;
    const double T = (we - (Ux * Ux + Uy * Uy) * w) / wd;
    const float ux = (float)Ux, uy = (float)Uy, Tf = (float)T;
    store_with_images(st.mom + (long long)S * st.P, cell, x, y, oc.pitch, im, ux);
    store_with_images(st.mom + (long long)(S + 1) * st.P, cell, x, y, oc.pitch, im, uy);
    store_with_images(st.mom + (long long)(S + 2) * st.P, cell, x, y, oc.pitch, im, Tf);
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        const float ns = (float)n[s];
        store_with_images(st.mom + (long long)s * st.P, cell, x, y, oc.pitch, im, ns);
        float fe[Q];
        feq_ref<S>(k, s, ns, ux, uy, Tf, fe);
        for (int i = 0; i < Q; ++i)
            store_with_images(st.d + (long long)(s * Q + i) * st.P, cell, x, y, oc.pitch, im,
                              __float2bfloat16_rn((float)(src[(s * Q + i) * N + d] - (double)fe[i])));
    }
}

template <int S>
__global__ void __launch_bounds__(128)
    k_get_f_bf16(const __grid_constant__ StepConsts<float, S> k, BfState st, double *__restrict__ dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const long long N = (long long)k.nx * k.ny, d = (long long)y * k.nx + x;
    const long long cell = (long long)(y + GY) * k.pitch + (x + GX);
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        float f[Q];
        bf_cell_f<S>(k, st, s, cell, f);
        for (int i = 0; i < Q; ++i) dst[(s * Q + i) * N + d] = (double)f[i];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// one cell per thread: 32 x 16 measured fastest of 64x8, 32x16, 32x8, 32x7
// and 64x4; BF_CW = 2: two adjacent cells per thread (packed FP32x2 step)
constexpr int BF_TX = 32, BF_TY = 16, BF_CW = 2;

template <int S>
static int step_bf16_t(dbm_handle *h, int cur, cudaStream_t st)
{
    constexpr size_t smem = (size_t)(BF_TX + 4) * (BF_TY + 4) * S * Q * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_bf16<S, BF_TX, BF_TY, BF_CW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(h, e, "BF16 step kernel shared-memory attribute");
        attr_set = true;
    }
    StepConsts<float, S> c;
    fill_step_consts<float, S>(h, c);
    dim3 block(BF_TX / BF_CW, BF_TY);
    dim3 grid((h->p.nx + BF_TX - 1) / BF_TX, (h->p.ny + BF_TY - 1) / BF_TY);
    k_step_bf16<S, BF_TX, BF_TY, BF_CW><<<grid, block, smem, st>>>(c, bf_state(h, h->f[cur]),
                                                                   bf_state(h, h->f[cur ^ 1]),
                                                                   (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "BF16 step kernel launch");
}

int launch_step_bf16(dbm_handle *h, int cur, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: return step_bf16_t<1>(h, cur, st);
    case 2: return step_bf16_t<2>(h, cur, st);
    case 3: return step_bf16_t<3>(h, cur, st);
    case 4: return step_bf16_t<4>(h, cur, st);
    }
    return DBM_ERR_INVALID;
}

static dim3 grid_of(const dbm_handle *h, dim3 b)
{
    return dim3((h->p.nx + b.x - 1) / b.x, (h->p.ny + b.y - 1) / b.y);
}

template <int S>
static void set_state_bf16_t(dbm_handle *h, void *f, const double *rho_s, const double *ux, const double *uy,
                             const double *T, cudaStream_t st)
{
    OutConsts<S> oc;
    fill_out_consts<S>(h, oc);
    dim3 b(32, 8);
    k_set_state_bf16<S><<<grid_of(h, b), b, 0, st>>>(bf_state(h, f), h->p.nx, h->p.ny, h->lay.pitch, h->p.bc_x,
                                                     h->p.bc_y, rho_s, ux, uy, T, oc);
}

int launch_set_state_bf16(dbm_handle *h, void *f, const double *rho_s, const double *ux, const double *uy,
                          const double *T, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: set_state_bf16_t<1>(h, f, rho_s, ux, uy, T, st); break;
    case 2: set_state_bf16_t<2>(h, f, rho_s, ux, uy, T, st); break;
    case 3: set_state_bf16_t<3>(h, f, rho_s, ux, uy, T, st); break;
    case 4: set_state_bf16_t<4>(h, f, rho_s, ux, uy, T, st); break;
    default: return DBM_ERR_INVALID;
    }
    return set_cuda_error(h, cudaGetLastError(), "BF16 set_state kernel launch");
}

template <int S>
static void set_f_bf16_t(dbm_handle *h, void *f, const double *src, cudaStream_t st)
{
    StepConsts<float, S> k;
    fill_step_consts<float, S>(h, k);
    OutConsts<S> oc;
    fill_out_consts<S>(h, oc);
    dim3 b(32, 4);
    k_set_f_bf16<S><<<grid_of(h, b), b, 0, st>>>(k, oc, bf_state(h, f), src);
}

int launch_set_f_bf16(dbm_handle *h, void *f, const double *src, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: set_f_bf16_t<1>(h, f, src, st); break;
    case 2: set_f_bf16_t<2>(h, f, src, st); break;
    case 3: set_f_bf16_t<3>(h, f, src, st); break;
    case 4: set_f_bf16_t<4>(h, f, src, st); break;
    default: return DBM_ERR_INVALID;
    }
    return set_cuda_error(h, cudaGetLastError(), "BF16 set_f kernel launch");
}

template <int S>
static void get_f_bf16_t(dbm_handle *h, const void *f, double *dst, cudaStream_t st)
{
    StepConsts<float, S> k;
    fill_step_consts<float, S>(h, k);
    dim3 b(32, 4);
    k_get_f_bf16<S><<<grid_of(h, b), b, 0, st>>>(k, bf_state(h, (void *)f), dst);
}

int launch_get_f_bf16(dbm_handle *h, const void *f, double *dst, cudaStream_t st)
{
    switch (h->p.nspecies) {
    case 1: get_f_bf16_t<1>(h, f, dst, st); break;
    case 2: get_f_bf16_t<2>(h, f, dst, st); break;
    case 3: get_f_bf16_t<3>(h, f, dst, st); break;
    case 4: get_f_bf16_t<4>(h, f, dst, st); break;
    default: return DBM_ERR_INVALID;
    }
    return set_cuda_error(h, cudaGetLastError(), "BF16 get_f kernel launch");
}

}  // namespace dbm
