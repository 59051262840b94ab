// dbm_batch.cu -- many independent D2V16 problems stepped together.
//
// A batch groups bound FP32 handles with the same species count.  Instances
// may differ in grid size, boundaries, species constants, reaction and time
// step.  The instances are split into chunks; per time step each chunk is
// one kernel launch whose parameter block (the kernel's constant bank)
// holds, for every instance of the chunk, its step constants, the TMA
// descriptor of its input buffer and its output pointers.  A CTA takes one
// tile (or a contiguous range of tiles) from the device tile list, stages
// the tile plus halo with one TMA copy through its instance's descriptor
// and runs the same per-cell arithmetic as the single-problem kernel, with
// the constants read from the constant bank (shared-memory copies of them
// would compete with the stencil reads).  Pairs of steps are replayed from
// a CUDA graph in which each chunk is an independent two-launch chain; the
// tile shape, launch form and L2 promotion are chosen by timing
// (dbm_batch_tune).  Like the single-problem TMA kernel, the batched kernel
// takes a boundary tile's halo from the interior cells and writes no ghost
// cells.  The kernel and the parameter block are in dbm_batch_impl.cuh.
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dbm_batch_impl.cuh"

namespace dbm {
// instantiated in dbm_batch_s1.cu .. dbm_batch_s4.cu
extern template BatchKernel batch_kernel_s<1>(int);
extern template BatchKernel batch_kernel_s<2>(int);
extern template BatchKernel batch_kernel_s<3>(int);
extern template BatchKernel batch_kernel_s<4>(int);
}  // namespace dbm

using namespace dbm;

typedef CUresult (*encode_tiled_fn_b)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);

// Tile shapes compiled for the batched kernel (cells) and the cells each
// thread updates (1, or 2 adjacent cells of a row in packed FP32x2).
static const int N_SHAPES = 7;
static const int SHAPE_TX[N_SHAPES] = {32, 32, 32, 32, 64, 64, 32};
static const int SHAPE_TY[N_SHAPES] = {10, 8, 16, 7, 4, 8, 16};
static const int SHAPE_CW[N_SHAPES] = {1, 1, 1, 1, 1, 2, 2};

static BatchKernel batch_kernel_for(int S, int shape)
{
    return S == 1 ? batch_kernel_s<1>(shape) : S == 2 ? batch_kernel_s<2>(shape)
           : S == 3 ? batch_kernel_s<3>(shape) : batch_kernel_s<4>(shape);
}

struct dbm_batch {
    std::vector<dbm_handle *> h;
    int S;
    int shape;       // index into SHAPE_TX / SHAPE_TY
    int persistent;  // 1: a launch has at most the CTAs resident at once; 0: one CTA per tile
    int promote;     // 1: the tile copies promote L2 fills to 256 B; 0: no promotion
    int parity;      // steps taken mod 2 since the parameter blocks were written
    int total_tiles;
    int resident;    // CTAs of the current kernel resident at once on the device
    BatchKernel k;
    void *table;  // caller's device buffer: the tile list
    size_t table_bytes;
    std::vector<BatchTile> tiles;  // host copy of the tile list
    unsigned char *chunks;         // parameter blocks [chunk][parity], 128-byte aligned
    int nchunks;
    std::vector<long long> expected_steps;  // each handle's step count the blocks assume
    cudaGraphExec_t graph[2];               // two steps starting at parity 0 / 1
    char err[512];
};

static int bfail(dbm_batch *b, int code, const char *msg)
{
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return code;
}

// Tiles per step of these handles with a TX x TY tile.
static long long count_tiles(dbm_handle *const *h, int n, int TX, int TY)
{
    long long t = 0;
    for (int k = 0; k < n; ++k) t += (long long)((h[k]->p.nx + TX - 1) / TX) * ((h[k]->p.ny + TY - 1) / TY);
    return t;
}

// Device table: the tile list for the tile shape with the most tiles.
static size_t table_size(dbm_handle *const *h, int n)
{
    long long most = 0;
    for (int sh = 0; sh < N_SHAPES; ++sh) {
        const long long t = count_tiles(h, n, SHAPE_TX[sh], SHAPE_TY[sh]);
        if (t > most) most = t;
    }
    return (size_t)most * sizeof(BatchTile) + 256;
}

static unsigned char *chunk_block(dbm_batch *b, int j, int parity)
{
    return b->chunks + (size_t)(2 * j + parity) * b->k.chunk_bytes;
}

// Write the tile list (to the device, then synchronise the stream) and the
// host parameter blocks of every chunk at both parities; parity 0 reads
// each handle's current buffer.
template <int S>
static int write_tables(dbm_batch *b, cudaStream_t st)
{
    const int n = (int)b->h.size();
    const int TX = b->k.tx, TY = b->k.ty;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return bfail(b, DBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode_tiled_fn_b encode = (encode_tiled_fn_b)fn;
    // group the instances by their shared ("hot") constants, then cut each
    // group into launches of at most CAP instances
    const int cap = BatchChunk<S>::CAP;
    std::vector<StepConsts<float, S>> cs(n), hot(n);
    for (int k = 0; k < n; ++k) {
        fill_step_consts<float, S>(b->h[k], cs[k]);
        memcpy(&hot[k], &cs[k], sizeof(hot[k]));  // all bytes, padding included, for memcmp
        hot_part<S>(hot[k]);
    }
    std::vector<std::vector<int>> chunks;
    std::vector<int> rep;  // an instance of each chunk's group
    for (int k = 0; k < n; ++k) {
        int j = -1;
        for (size_t q = 0; q < chunks.size() && j < 0; ++q)
            if ((int)chunks[q].size() < cap && !memcmp(&hot[rep[q]], &hot[k], sizeof(hot[k]))) j = (int)q;
        if (j < 0) {
            chunks.emplace_back();
            rep.push_back(k);
            j = (int)chunks.size() - 1;
        }
        chunks[j].push_back(k);
    }
    const int nchunks = (int)chunks.size();
    const size_t bytes_all = (size_t)2 * nchunks * sizeof(BatchChunk<S>);
    if (nchunks != b->nchunks || !b->chunks) {
        free(b->chunks);
        b->chunks = (unsigned char *)aligned_alloc(128, (bytes_all + 127) / 128 * 128);
        b->nchunks = b->chunks ? nchunks : 0;
        if (!b->chunks) return bfail(b, DBM_ERR_INVALID, "out of host memory");
    }
    memset(b->chunks, 0, bytes_all);
    b->expected_steps.assign(n, 0);
    b->tiles.clear();
    for (int j = 0; j < nchunks; ++j) {
        const int t0 = (int)b->tiles.size();
        BatchChunk<S> *blk[2] = {reinterpret_cast<BatchChunk<S> *>(chunk_block(b, j, 0)),
                                 reinterpret_cast<BatchChunk<S> *>(chunk_block(b, j, 1))};
        for (int local = 0; local < (int)chunks[j].size(); ++local) {
            const int k = chunks[j][local];
            dbm_handle *h = b->h[k];
            b->expected_steps[k] = h->steps;
            const int tiles_x = (h->p.nx + TX - 1) / TX, nt = tiles_x * ((h->p.ny + TY - 1) / TY);
            for (int u = 0; u < nt; ++u)
                b->tiles.push_back(BatchTile{local, (u % tiles_x) * TX, (u / tiles_x) * TY, 0});
            for (int par = 0; par < 2; ++par) {
                BatchInst<S> &e = blk[par]->e[local];
                void *in = h->f[h->cur ^ par];
                const dbm_layout &L = h->lay;
                cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)(16 * S)};
                cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
                cuuint32_t box[3] = {(cuuint32_t)(TX + 8), (cuuint32_t)(TY + 4), (cuuint32_t)(16 * S)};
                cuuint32_t estr[3] = {1, 1, 1};
                if (encode(&e.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, in, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           b->promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return bfail(b, DBM_ERR_CUDA, "tensor map encoding failed");
                e.c = inst_part<S>(cs[k]);
                e.fin = (const float *)in;
                e.fout = (float *)h->f[h->cur ^ par ^ 1];
                e.flag = (unsigned *)h->scratch;
            }
        }
        for (int par = 0; par < 2; ++par) {
            blk[par]->n = (int)chunks[j].size();
            blk[par]->t0 = t0;
            blk[par]->nt = (int)b->tiles.size() - t0;
            blk[par]->hot = cs[rep[j]];
        }
    }
    b->total_tiles = (int)b->tiles.size();
    const size_t bytes = b->tiles.size() * sizeof(BatchTile);
    if (bytes > b->table_bytes) return bfail(b, DBM_ERR_INVALID, "tile list larger than the table");
    cudaError_t er = cudaMemcpyAsync(b->table, b->tiles.data(), bytes, cudaMemcpyHostToDevice, st);
    if (er != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(er));
    er = cudaStreamSynchronize(st);  // the host list may change on the next write
    if (er != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(er));
    return DBM_OK;
}

// Tiles of chunk j (the count sits in the block header: n, t0, nt).
static int chunk_tiles(const dbm_batch *b, int j)
{
    return reinterpret_cast<const int *>(b->chunks + (size_t)(2 * j) * b->k.chunk_bytes)[2];
}

static int chunk_grid(const dbm_batch *b, int j)
{
    const int nt = chunk_tiles(b, j);
    return b->persistent && b->resident < nt ? b->resident : nt;
}

// Launch arguments of chunk j at a parity (the block is copied at launch).
struct ChunkArgs {
    const BatchTile *tiles;
    void *args[2];
};

static void chunk_args(dbm_batch *b, int j, int parity, ChunkArgs &a)
{
    a.tiles = (const BatchTile *)b->table;
    a.args[0] = chunk_block(b, j, parity);
    a.args[1] = &a.tiles;
}

// One time step of every chunk, launched in turn on the stream.
static int launch_step_all(dbm_batch *b, int parity, cudaStream_t st)
{
    for (int j = 0; j < b->nchunks; ++j) {
        ChunkArgs a;
        chunk_args(b, j, parity, a);
        cudaError_t e =
            cudaLaunchKernel(b->k.fn, dim3(chunk_grid(b, j)), dim3(b->k.bx, b->k.ty), a.args, b->k.smem, st);
        if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
    }
    return DBM_OK;
}

// Two steps from `parity`: per chunk a chain of two kernel nodes; the
// chunks' chains are independent of each other.
static int build_graph(dbm_batch *b, int parity, cudaGraphExec_t *out)
{
    cudaGraph_t g;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
    for (int j = 0; j < b->nchunks && e == cudaSuccess; ++j) {
        cudaGraphNode_t prev = nullptr;
        for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
            ChunkArgs a;
            chunk_args(b, j, parity ^ s, a);
            cudaKernelNodeParams kp;
            memset(&kp, 0, sizeof(kp));
            kp.func = const_cast<void *>(b->k.fn);
            kp.gridDim = dim3(chunk_grid(b, j));
            kp.blockDim = dim3(b->k.bx, b->k.ty);
            kp.sharedMemBytes = (unsigned)b->k.smem;
            kp.kernelParams = a.args;
            cudaGraphNode_t node;
            e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            prev = node;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? DBM_OK : bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
}

static void drop_graphs(dbm_batch *b)
{
    for (int g = 0; g < 2; ++g)
        if (b->graph[g]) {
            cudaGraphExecDestroy(b->graph[g]);
            b->graph[g] = nullptr;
        }
}

// Select the kernel of the current shape and rewrite every table for the
// handles' current states.
static int rebuild(dbm_batch *b, cudaStream_t st)
{
    drop_graphs(b);
    b->k = batch_kernel_for(b->S, b->shape);
    if (b->persistent) b->k.fn = b->k.fn_persist;
    cudaError_t e = cudaFuncSetAttribute(b->k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->k.smem);
    if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, b->k.fn, b->k.bx * b->k.ty, b->k.smem);
    b->resident = sms * (per > 0 ? per : 1);
    const int rc = b->S == 1   ? write_tables<1>(b, st)
                   : b->S == 2 ? write_tables<2>(b, st)
                   : b->S == 3 ? write_tables<3>(b, st)
                               : write_tables<4>(b, st);
    if (rc) return rc;
    b->parity = 0;  // the blocks map each handle's current buffer to parity 0
    return DBM_OK;
}

extern "C" {

int dbm_batch_table_bytes(dbm_handle *const *handles, int n, size_t *bytes)
{
    if (!handles || n < 1 || !bytes || !handles[0]) return DBM_ERR_INVALID;
    const int S = handles[0]->p.nspecies;
    if (S > 4) return DBM_ERR_INVALID;
    for (int k = 0; k < n; ++k)
        if (!handles[k]) return DBM_ERR_INVALID;
    *bytes = table_size(handles, n);
    return DBM_OK;
}

int dbm_batch_create(dbm_handle *const *handles, int n, void *table, size_t table_bytes, void *stream,
                     dbm_batch **out)
{
    if (!handles || n < 1 || !out || !table) return DBM_ERR_INVALID;
    *out = nullptr;
    const int S = handles[0] ? handles[0]->p.nspecies : 0;
    for (int k = 0; k < n; ++k) {
        const dbm_handle *h = handles[k];
        if (!h || !h->bound || h->p.precision != DBM_FP32 || h->p.nspecies != S || S > 4 || !h->tma_ok ||
            uses_acc(h->p))
            return DBM_ERR_INVALID;
    }
    if (table_bytes < table_size(handles, n) || ((uintptr_t)table & 127)) return DBM_ERR_INVALID;
    dbm_batch *b = new dbm_batch();
    b->h.assign(handles, handles + n);
    b->S = S;
    b->shape = 0;
    b->persistent = 0;
    b->promote = 1;
    b->table = table;
    b->table_bytes = table_bytes;
    b->chunks = nullptr;
    b->nchunks = 0;
    b->graph[0] = b->graph[1] = nullptr;
    b->err[0] = 0;
    const int rc = rebuild(b, (cudaStream_t)stream);
    if (rc) {
        free(b->chunks);
        delete b;
        return rc;
    }
    *out = b;
    return DBM_OK;
}

// Hand each instance's step count and current buffer back to its handle.
static void sync_handles(dbm_batch *b, int nsteps)
{
    for (size_t k = 0; k < b->h.size(); ++k) {
        dbm_handle *h = b->h[k];
        h->cur ^= (nsteps & 1);
        h->steps += nsteps;
        b->expected_steps[k] = h->steps;
    }
}

int dbm_batch_tune(dbm_batch *b, void *stream, int reps)
{
    if (!b) return DBM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (reps < 1) reps = 3;
    float best = 1e30f;
    int best_shape = 0, best_mode = 0, best_promote = 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = DBM_OK;
    for (int trial = 0; trial < 4 * N_SHAPES && !rc; ++trial) {
        b->shape = trial >> 2;
        b->persistent = trial & 1;
        b->promote = (trial >> 1) & 1;
        rc = rebuild(b, st);
        // a trial step reads the current states and writes the other
        // buffers, which the next real step overwrites: no state advances
        if (!rc) rc = launch_step_all(b, 0, st);
        if (rc) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc; ++r) rc = launch_step_all(b, 0, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && ms < best) {
            best = ms;
            best_shape = b->shape;
            best_mode = b->persistent;
            best_promote = b->promote;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->shape = best_shape;
    b->persistent = best_mode;
    b->promote = best_promote;
    return rebuild(b, st);
}

static int batch_step(dbm_batch *b, int nsteps, cudaStream_t st);

int dbm_batch_step(dbm_batch *b, int nsteps, void *stream)
{
    if (!b || nsteps < 0) return DBM_ERR_INVALID;
    nvtxRangePushA("dbm_batch_step");  // host-side range over the enqueueing of the steps
    const int rc = batch_step(b, nsteps, (cudaStream_t)stream);
    nvtxRangePop();
    return rc;
}

static int batch_step(dbm_batch *b, int nsteps, cudaStream_t st)
{
    for (size_t k = 0; k < b->h.size(); ++k)
        if (b->h[k]->steps != b->expected_steps[k]) {  // a handle was reset or stepped alone
            const int rc = rebuild(b, st);
            if (rc) return rc;
            break;
        }
    int left = nsteps;
    // graphs run on a created stream; on the legacy default stream the
    // steps are launched one by one
    const bool graphs = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    while (left >= 2 && !graphs) {
        int rc = launch_step_all(b, b->parity, st);
        if (!rc) rc = launch_step_all(b, b->parity ^ 1, st);
        if (rc) return rc;
        left -= 2;
    }
    while (left >= 2) {
        cudaGraphExec_t &g = b->graph[b->parity];
        if (!g) {
            const int rc = build_graph(b, b->parity, &g);
            if (rc) return rc;
        }
        cudaError_t e = cudaGraphLaunch(g, st);
        if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
        left -= 2;
    }
    if (left == 1) {
        const int rc = launch_step_all(b, b->parity, st);
        if (rc) return rc;
        b->parity ^= 1;
    }
    sync_handles(b, nsteps);
    return DBM_OK;
}

int dbm_batch_info(const dbm_batch *b, int *tile_x, int *tile_y, int *tiles, int *ctas)
{
    if (!b) return DBM_ERR_INVALID;
    if (tile_x) *tile_x = SHAPE_TX[b->shape];
    if (tile_y) *tile_y = SHAPE_TY[b->shape];
    if (tiles) *tiles = b->total_tiles;
    if (ctas) {
        int c = 0;
        for (int j = 0; j < b->nchunks; ++j) c += chunk_grid(b, j);
        *ctas = c;
    }
    return DBM_OK;
}

int dbm_batch_get_config(const dbm_batch *b, int *tile_x, int *tile_y, int *cells_per_thread, int *persistent,
                         int *promote)
{
    if (!b) return DBM_ERR_INVALID;
    if (tile_x) *tile_x = SHAPE_TX[b->shape];
    if (tile_y) *tile_y = SHAPE_TY[b->shape];
    if (cells_per_thread) *cells_per_thread = SHAPE_CW[b->shape];
    if (persistent) *persistent = b->persistent;
    if (promote) *promote = b->promote;
    return DBM_OK;
}

int dbm_batch_set_config(dbm_batch *b, int tile_x, int tile_y, int cells_per_thread, int persistent, int promote,
                         void *stream)
{
    if (!b || (persistent != 0 && persistent != 1) || (promote != 0 && promote != 1)) return DBM_ERR_INVALID;
    int shape = -1;
    for (int sh = 0; sh < N_SHAPES; ++sh)
        if (SHAPE_TX[sh] == tile_x && SHAPE_TY[sh] == tile_y && SHAPE_CW[sh] == cells_per_thread) shape = sh;
    if (shape < 0) return bfail(b, DBM_ERR_INVALID, "tile shape not compiled for batches");
    b->shape = shape;
    b->persistent = persistent;
    b->promote = promote;
    return rebuild(b, (cudaStream_t)stream);
}

const char *dbm_batch_last_error(const dbm_batch *b) { return b ? b->err : "null batch"; }

void dbm_batch_destroy(dbm_batch *b)
{
    if (!b) return;
    drop_graphs(b);
    free(b->chunks);
    delete b;
}

}  // extern "C"
