// dbm_batch_impl.cuh -- the batched step kernel and its launch parameter
// block (see dbm_batch.cu for the batch itself).  The kernels are
// instantiated once per species count in dbm_batch_s<S>.cu, so that the
// units compile in parallel.
#pragma once

#include <stddef.h>
#include <string.h>

#include "dbm_step_impl.cuh"

namespace dbm {

// The constants of one instance that step_cell reads from the instance's
// own block (`g`: geometry, boundaries, reaction, force, wait limit); the
// rest of StepConsts is shared by every instance of a launch.
template <int S>
struct InstConsts {
    float tau_d[S], tau_a[S];  // tau^s, tau^s a^s
    float k_ov, Ea_over_R, Qheat, src;
    float accel_x, accel_y;
    int fuel, oxid, has_reaction, has_force;
    int nx, ny, pitch, bc_x, bc_y, wait_polls;
    long long plane;
};

template <int S>
InstConsts<S> inst_part(const StepConsts<float, S> &c)
{
    InstConsts<S> g;
    memset(&g, 0, sizeof(g));
    for (int s = 0; s < S; ++s) {
        g.tau_d[s] = c.tau_d[s];
        g.tau_a[s] = c.tau_a[s];
    }
    g.k_ov = c.k_ov;
    g.Ea_over_R = c.Ea_over_R;
    g.Qheat = c.Qheat;
    g.src = c.src;
    g.accel_x = c.accel_x;
    g.accel_y = c.accel_y;
    g.fuel = c.fuel;
    g.oxid = c.oxid;
    g.has_reaction = c.has_reaction;
    g.has_force = c.has_force;
    g.nx = c.nx;
    g.ny = c.ny;
    g.pitch = c.pitch;
    g.bc_x = c.bc_x;
    g.bc_y = c.bc_y;
    g.wait_polls = c.wait_polls;
    g.plane = c.plane;
    return g;
}

// One instance of a launch: its input descriptor at the launch's parity,
// own constants and outputs.
template <int S>
struct __align__(128) BatchInst {  // CUtensorMap is 128-byte aligned
    CUtensorMap tmap;
    InstConsts<S> c;
    const float *fin;  // the input buffer (interior cells for a boundary tile's halo)
    float *fout;
    unsigned *flag;
};

// Bytes a launch's parameter block may use (the kernel-parameter limit is
// 32764 bytes; the tile-list pointer follows the block).
constexpr int BATCH_PARAM_BYTES = 32 * 1024 - 256;

// Parameter block of one launch: n instances that share the constants the
// step uses many times per cell (`hot`: equilibrium blocks, ring speeds,
// weights, advection numbers), and their tiles t0 .. t0+nt-1 of the device
// tile list.  The shared constants stay constant-bank operands in the
// kernel; each instance's own block supplies only geometry, boundaries,
// reaction and force.
template <int S>
struct BatchChunk {
    static constexpr int HOT_BYTES = ((int)sizeof(StepConsts<float, S>) + 127) / 128 * 128;
    static constexpr int CAP = (BATCH_PARAM_BYTES - 128 - HOT_BYTES) / (int)sizeof(BatchInst<S>);
    int n, t0, nt, pad;
    StepConsts<float, S> hot;
    BatchInst<S> e[CAP];
};
// The constants of a block that instances must share to go into one
// launch: everything but geometry, boundaries, reaction and force, which
// step_cell reads from the instance's own block.
template <int S>
void hot_part(StepConsts<float, S> &c)
{
    for (int s = 0; s < S; ++s) c.tau_d[s] = c.tau_a[s] = 0.f;
    c.k_ov = c.Ea_over_R = c.Qheat = c.src = 0.f;
    c.fuel = c.oxid = c.has_reaction = c.has_force = 0;
    c.accel_x = c.accel_y = 0.f;
    c.nx = c.ny = c.pitch = c.bc_x = c.bc_y = 0;
    c.wait_polls = 0;
    c.plane = 0;
}

static_assert(sizeof(BatchChunk<1>) <= BATCH_PARAM_BYTES && sizeof(BatchChunk<4>) <= BATCH_PARAM_BYTES,
              "parameter block too large");

// One tile of one instance, as a single 16-byte load.
struct __align__(16) BatchTile {
    int k;         // instance (index in its launch's parameter block)
    int bx0, by0;  // first interior cell of the tile
    int pad;
};

// PERSIST: the grid holds only the CTAs resident at once, each walking a
// contiguous range of tiles; else one CTA per tile (compiled without the
// loop, so that no loop state stays live across the step).
template <int S, int TX, int TY, int CW, bool PERSIST>
__global__ void __launch_bounds__(TX / CW * TY, tma_ctas_per_sm(S, TX, TY))
    k_step_batch(const __grid_constant__ BatchChunk<S> P, const BatchTile *__restrict__ tiles)
{
    constexpr int BX = TX + 8, BY = TY + 4, NP = S * Q, NT = TX / CW * TY;
    constexpr unsigned BYTES = (unsigned)(BX * BY * NP * sizeof(float));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool leader = tx == 0 && ty == 0;
    const unsigned b = smem_u32(&bar);
    if (leader) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    const int t0 = P.t0 + (PERSIST ? (int)((long long)P.nt * blockIdx.x / gridDim.x) : (int)blockIdx.x);
    const int t1 = PERSIST ? P.t0 + (int)((long long)P.nt * (blockIdx.x + 1) / gridDim.x) : t0 + 1;
    unsigned phase = 0;
    BatchTile next = tiles[t0];
    for (int t = t0; t < t1; ++t, phase ^= 1u) {
        const BatchTile cur = next;
        if (t + 1 < t1) next = tiles[t + 1];
        const BatchInst<S> &e = P.e[cur.k];
        const InstConsts<S> &g = e.c;
        __syncthreads();  // barrier initialised / previous tile no longer read
        if (leader) {
            // the previous tile's halo fill and stencil reads went through the
            // generic proxy; order them before the async-proxy copy that
            // overwrites the same shared memory
            if (t > t0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_tile_load(tile, reinterpret_cast<unsigned long long>(&e.tmap), cur.bx0, cur.by0, b, BYTES);
        }
        const int tid = ty * (TX / CW) + tx;
        const HaloSides hs = halo_sides<TX, TY>(cur.bx0, cur.by0, g.nx, g.ny);
        HaloRegs<NP, TX, TY, NT> hr;
        if (hs.any())
            halo_load(hr, hs, e.fin, cur.bx0, cur.by0, g.nx, g.ny, g.pitch, g.plane, g.bc_x, g.bc_y, tid, e.flag);
        const bool ok = mbar_wait(b, phase, g.wait_polls);
        if (__syncthreads_or(!ok)) {
            // the copy did not land: report, give it one more bounded wait so
            // that no copy is left writing into shared memory, leave together
            if (leader) raise_flag(e.flag, DBM_HEALTH_TIMEOUT);
            mbar_wait(b, phase, TMA_WAIT_LIMIT);
            return;
        }
        if (hs.any()) halo_store(hr, hs, tile, cur.bx0, cur.by0, g.nx, g.ny, tid, e.flag);
        const int x = cur.bx0 + CW * tx, y = cur.by0 + ty;
        if (x < g.nx && y < g.ny) {
            StateOutNoImages o{e.fout, g.plane, (long long)NP * g.plane, e.flag};
            const float *base = tile + (ty + 2) * BX + (CW * tx + 4);
            if constexpr (CW == 2) {
                const SmemTile2 st{base, BY * BX, BX, tile, NP * BY * BX, e.flag};
                step_cell<S>(P.hot, g, st, x, y, x + 1 < g.nx, o, e.flag);
            } else {
                const SmemTile st{base, BY * BX, BX, tile, NP * BY * BX, e.flag};
                step_cell<S>(P.hot, g, st, x, y, true, o, e.flag);
            }
        }
    }
}

// The compiled kernel of species count S and tile shape TX x TY (cells;
// bx = TX / CW threads per row).
struct BatchKernel {
    const void *fn;  // one CTA per tile; fn_persist: CTAs walking tile ranges
    const void *fn_persist;
    int tx, ty, bx;
    size_t smem;
    size_t chunk_bytes;
    int cap;
};

template <int S, int TX, int TY, int CW>
BatchKernel batch_kernel()
{
    const void *fn = (const void *)k_step_batch<S, TX, TY, CW, false>;
    const void *fn_persist = (const void *)k_step_batch<S, TX, TY, CW, true>;
    return BatchKernel{fn, fn_persist, TX, TY, TX / CW, (size_t)(TX + 8) * (TY + 4) * S * Q * sizeof(float),
                       sizeof(BatchChunk<S>), BatchChunk<S>::CAP};
}

// The kernel of tile shape `shape` (an index into the compiled shapes
// 32x10, 32x8, 32x16, 32x7, 64x4 at one cell per thread, 64x8, 32x16 at
// two), instantiated for each species count in dbm_batch_s<S>.cu.
template <int S>
BatchKernel batch_kernel_s(int shape)
{
    switch (shape) {
    case 0: return batch_kernel<S, 32, 10, 1>();
    case 1: return batch_kernel<S, 32, 8, 1>();
    case 2: return batch_kernel<S, 32, 16, 1>();
    case 3: return batch_kernel<S, 32, 7, 1>();
    case 4: return batch_kernel<S, 64, 4, 1>();
    case 5: return batch_kernel<S, 64, 8, 2>();
    default: return batch_kernel<S, 32, 16, 2>();
    }
}

}  // namespace dbm
