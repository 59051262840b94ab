// dbm_batch.cu -- many independent D2V16 problems stepped together.
//
// A batch groups bound FP32 handles with the same species count.  One
// persistent kernel launch per time step walks the tiles of every instance
// (instances may differ in grid size, boundaries, species constants,
// reaction and time step): each CTA takes a contiguous range of tiles, looks
// up each tile's instance in a table, copies that instance's step constants
// into shared memory when the instance changes, stages the tile plus halo
// with one TMA copy through the instance's own tensor map, and runs the
// same per-cell arithmetic as the single-problem kernel.  Steps are replayed from captured CUDA graphs, and
// the tile shape is chosen by timing each compiled shape (dbm_batch_tune).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "dbm_step_impl.cuh"

namespace dbm {

// One instance as the batched kernel sees it (device table entry).
template <int S>
struct __align__(128) BatchEntry {
    CUtensorMap tmap[2];  // input descriptor at parity 0 and parity 1
    StepConsts<float, S> c;
    float *f[2];          // input buffer at parity 0 and parity 1
    unsigned *flag;
    int tiles_x, tile_begin;
};

template <int S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2)
    k_step_batch(const BatchEntry<S> *__restrict__ tab, const int *__restrict__ tile_inst, int total, int parity)
{
    constexpr int BX = TX + 8, BY = TY + 4, NP = S * Q;
    constexpr unsigned BYTES = (unsigned)(BX * BY * NP * sizeof(float));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ StepConsts<float, S> sc;
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y, nthr = TX * TY, tid = ty * TX + tx;
    const bool leader = tid == 0;
    const unsigned b = smem_u32(&bar);
    if (leader) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // a contiguous range of tiles per CTA: consecutive tiles mostly belong
    // to the same instance, so its constants stay in shared memory
    const int t0 = (int)((long long)total * blockIdx.x / gridDim.x);
    const int t1 = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
    int k_loaded = -1;
    unsigned phase = 0;
    for (int t = t0; t < t1; ++t, phase ^= 1u) {
        const int k = tile_inst[t];
        const BatchEntry<S> &e = tab[k];
        __syncthreads();  // the previous tile is done with the shared tile and constants
        const int local = t - e.tile_begin;
        const int bx0 = (local % e.tiles_x) * TX, by0 = (local / e.tiles_x) * TY;
        if (leader) {
            const unsigned long long tm = reinterpret_cast<unsigned long long>(&e.tmap[parity]);
            // the descriptor lives in global memory: acquire it for the tensor-map proxy
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
            tma_tile_load(tile, tm, bx0, by0, b, BYTES);
        }
        if (k != k_loaded) {  // this instance's constants into shared memory
            const unsigned *src = reinterpret_cast<const unsigned *>(&e.c);
            unsigned *dst = reinterpret_cast<unsigned *>(&sc);
            for (int j = tid; j < (int)(sizeof(sc) / 4); j += nthr) dst[j] = src[j];
            k_loaded = k;
            __syncthreads();
        }
        if (!mbar_wait(b, phase, TMA_WAIT_LIMIT)) {
            if (leader) raise_flag(e.flag, DBM_HEALTH_TIMEOUT);
            mbar_wait(b, phase, TMA_WAIT_LIMIT);
            return;
        }
        const int x = bx0 + tx, y = by0 + ty;
        if (x < sc.nx && y < sc.ny) {
            SmemTile st;
            st.base = tile + (ty + 2) * BX + (tx + 4);
            st.P = BY * BX;
            st.py = BX;
            StateOut o{e.f[parity ^ 1], sc.plane, sc.nx, sc.ny, sc.pitch};
            step_cell<S>(sc, st, x, y, o, e.flag);
        }
    }
}

}  // namespace dbm

using namespace dbm;

typedef CUresult (*encode_tiled_fn_b)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);

// Tile shapes compiled for the batched kernel.
static const int N_SHAPES = 3;
static const int SHAPE_TX[N_SHAPES] = {64, 32, 32};
static const int SHAPE_TY[N_SHAPES] = {8, 8, 16};

struct dbm_batch {
    std::vector<dbm_handle *> h;
    int S;
    int shape;                 // index into SHAPE_TX / SHAPE_TY
    int persistent;            // 1: as many CTAs as fit at once; 0: one CTA per tile
    int parity;                // steps taken mod 2
    int total_tiles, ctas;
    void *table;               // caller's device buffer
    size_t table_bytes;
    unsigned char *host;       // staging copy of the table (128-byte aligned)
    size_t host_bytes;
    std::vector<long long> expected_steps;  // each handle's step count the table assumes
    cudaGraphExec_t graph[2];         // two steps starting at parity 0 / 1
    char err[512];
};

static int bfail(dbm_batch *b, int code, const char *msg)
{
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return code;
}

template <int S>
static size_t entry_bytes()
{
    return sizeof(BatchEntry<S>);
}

// Tiles per step of these handles with a TX x TY tile.
static long long count_tiles(dbm_handle *const *h, int n, int TX, int TY)
{
    long long t = 0;
    for (int k = 0; k < n; ++k) t += (long long)((h[k]->p.nx + TX - 1) / TX) * ((h[k]->p.ny + TY - 1) / TY);
    return t;
}

// Table: n entries, then the instance of every tile (for the tile shape
// with the most tiles).
static size_t table_size(dbm_handle *const *h, int n)
{
    const int S = h[0]->p.nspecies;
    const size_t e = S == 1 ? entry_bytes<1>() : S == 2 ? entry_bytes<2>() : entry_bytes<3>();
    long long most = 0;
    for (int sh = 0; sh < N_SHAPES; ++sh) {
        const long long t = count_tiles(h, n, SHAPE_TX[sh], SHAPE_TY[sh]);
        if (t > most) most = t;
    }
    return e * n + (size_t)most * sizeof(int) + 256;
}

template <int S>
static int write_table(dbm_batch *b, cudaStream_t st)
{
    const int n = (int)b->h.size();
    const int TX = SHAPE_TX[b->shape], TY = SHAPE_TY[b->shape];
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return bfail(b, DBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode_tiled_fn_b encode = (encode_tiled_fn_b)fn;
    const size_t bytes = table_size(b->h.data(), n);
    if (b->host_bytes < bytes) {
        free(b->host);
        b->host = (unsigned char *)aligned_alloc(128, (bytes + 127) / 128 * 128);
        if (!b->host) return bfail(b, DBM_ERR_INVALID, "out of host memory");
        b->host_bytes = bytes;
    }
    memset(b->host, 0, bytes);
    b->expected_steps.assign(n, 0);
    BatchEntry<S> *ent = reinterpret_cast<BatchEntry<S> *>(b->host);
    int *tile_inst = reinterpret_cast<int *>(b->host + sizeof(BatchEntry<S>) * n);
    int tiles = 0;
    for (int k = 0; k < n; ++k) {
        dbm_handle *h = b->h[k];
        BatchEntry<S> &e = ent[k];
        fill_step_consts<float, S>(h, e.c);
        const int cur = h->cur;
        b->expected_steps[k] = h->steps;
        for (int par = 0; par < 2; ++par) {
            void *in = h->f[cur ^ par];  // parity 0 reads the current state
            e.f[par] = (float *)in;
            const dbm_layout &L = h->lay;
            cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)(16 * S)};
            cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
            cuuint32_t box[3] = {(cuuint32_t)(TX + 8), (cuuint32_t)(TY + 4), (cuuint32_t)(16 * S)};
            cuuint32_t estr[3] = {1, 1, 1};
            if (encode(&e.tmap[par], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, in, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return bfail(b, DBM_ERR_CUDA, "tensor map encoding failed");
        }
        e.flag = (unsigned *)h->scratch;
        e.tiles_x = (h->p.nx + TX - 1) / TX;
        e.tile_begin = tiles;
        const int nt = e.tiles_x * ((h->p.ny + TY - 1) / TY);
        for (int j = 0; j < nt; ++j) tile_inst[tiles + j] = k;
        tiles += nt;
    }
    b->total_tiles = tiles;
    // the table is rewritten while its parity layout is "current input at parity 0"
    cudaError_t er = cudaMemcpyAsync(b->table, b->host, bytes, cudaMemcpyHostToDevice, st);
    if (er != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(er));
    er = cudaStreamSynchronize(st);  // the staging buffer may change on the next write
    if (er != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(er));
    return DBM_OK;
}

static int grid_size(const dbm_batch *b)
{
    return b->persistent && b->ctas < b->total_tiles ? b->ctas : b->total_tiles;
}

template <int S, int TX, int TY>
static int launch_batch_t(dbm_batch *b, int parity, cudaStream_t st, bool set_attr)
{
    constexpr size_t smem = (size_t)(TX + 8) * (TY + 4) * S * Q * sizeof(float);
    if (set_attr) {
        cudaError_t e = cudaFuncSetAttribute(k_step_batch<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_batch<S, TX, TY>, TX * TY, smem);
        b->ctas = sms * (per > 0 ? per : 1);
        return DBM_OK;
    }
    const int n = (int)b->h.size();
    const BatchEntry<S> *tab = reinterpret_cast<const BatchEntry<S> *>(b->table);
    const int *tile_inst = reinterpret_cast<const int *>((const char *)b->table + sizeof(BatchEntry<S>) * n);
    const int grid = grid_size(b);
    k_step_batch<S, TX, TY><<<grid, dim3(TX, TY), smem, st>>>(tab, tile_inst, b->total_tiles, parity);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DBM_OK : bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
}

template <int S>
static int launch_batch_s(dbm_batch *b, int parity, cudaStream_t st, bool set_attr)
{
    switch (b->shape) {
    case 0: return launch_batch_t<S, 64, 8>(b, parity, st, set_attr);
    case 1: return launch_batch_t<S, 32, 8>(b, parity, st, set_attr);
    case 2: return launch_batch_t<S, 32, 16>(b, parity, st, set_attr);
    }
    return DBM_ERR_INVALID;
}

static int launch_batch(dbm_batch *b, int parity, cudaStream_t st, bool set_attr = false)
{
    switch (b->S) {
    case 1: return launch_batch_s<1>(b, parity, st, set_attr);
    case 2: return launch_batch_s<2>(b, parity, st, set_attr);
    case 3: return launch_batch_s<3>(b, parity, st, set_attr);
    }
    return DBM_ERR_INVALID;
}

static int rebuild(dbm_batch *b, cudaStream_t st)
{
    for (int g = 0; g < 2; ++g)
        if (b->graph[g]) {
            cudaGraphExecDestroy(b->graph[g]);
            b->graph[g] = nullptr;
        }
    int rc = b->S == 1 ? write_table<1>(b, st) : b->S == 2 ? write_table<2>(b, st) : write_table<3>(b, st);
    if (rc) return rc;
    b->parity = 0;  // the table now maps the current inputs to parity 0
    return launch_batch(b, 0, st, true);
}

extern "C" {

int dbm_batch_table_bytes(dbm_handle *const *handles, int n, size_t *bytes)
{
    if (!handles || n < 1 || !bytes || !handles[0]) return DBM_ERR_INVALID;
    const int S = handles[0]->p.nspecies;
    if (S > 3) return DBM_ERR_INVALID;
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
        if (!h || !h->bound || h->p.precision != DBM_FP32 || h->p.nspecies != S || S > 3 || !h->tma_ok)
            return DBM_ERR_INVALID;
    }
    if (table_bytes < table_size(handles, n) || ((uintptr_t)table & 127)) return DBM_ERR_INVALID;
    dbm_batch *b = new dbm_batch();
    b->host = nullptr;
    b->host_bytes = 0;
    b->h.assign(handles, handles + n);
    b->S = S;
    b->shape = 0;
    b->persistent = 1;
    b->table = table;
    b->table_bytes = table_bytes;
    b->graph[0] = b->graph[1] = nullptr;
    const int rc = rebuild(b, (cudaStream_t)stream);
    if (rc) {
        free(b->host);
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
    int best_shape = 0, best_mode = 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int trial = 0; trial < 2 * N_SHAPES; ++trial) {
        const int sh = trial >> 1;
        b->shape = sh;
        b->persistent = trial & 1;
        int rc = rebuild(b, st);
        // a trial launch reads the current states and writes the other
        // buffers, which the next real step overwrites: no state advances
        if (!rc) rc = launch_batch(b, 0, st);
        if (!rc) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && !rc; ++r) rc = launch_batch(b, 0, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
        if (ms < best) {
            best = ms;
            best_shape = sh;
            best_mode = b->persistent;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape = best_shape;
    b->persistent = best_mode;
    return rebuild(b, st);
}

int dbm_batch_step(dbm_batch *b, int nsteps, void *stream)
{
    if (!b || nsteps < 0) return DBM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t k = 0; k < b->h.size(); ++k)
        if (b->h[k]->steps != b->expected_steps[k]) {  // a handle was reset or stepped alone
            const int rc = rebuild(b, st);
            if (rc) return rc;
            break;
        }
    int left = nsteps;
    // graphs are captured on a created stream; on the legacy default stream
    // the steps are launched one by one
    const bool graphs = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    while (left >= 2 && !graphs) {
        int rc = launch_batch(b, b->parity, st);
        if (!rc) rc = launch_batch(b, b->parity ^ 1, st);
        if (rc) return rc;
        left -= 2;
    }
    while (left >= 2) {
        cudaGraphExec_t &g = b->graph[b->parity];
        if (!g) {  // capture two steps starting at this parity
            cudaGraph_t graph;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
            int rc = launch_batch(b, b->parity, st);
            if (!rc) rc = launch_batch(b, b->parity ^ 1, st);
            e = cudaStreamEndCapture(st, &graph);
            if (rc) return rc;
            if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
            e = cudaGraphInstantiate(&g, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
        }
        cudaError_t e = cudaGraphLaunch(g, st);
        if (e != cudaSuccess) return bfail(b, DBM_ERR_CUDA, cudaGetErrorString(e));
        left -= 2;
    }
    if (left == 1) {
        const int rc = launch_batch(b, b->parity, st);
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
    if (ctas) *ctas = grid_size(b);
    return DBM_OK;
}

const char *dbm_batch_last_error(const dbm_batch *b) { return b ? b->err : "null batch"; }

void dbm_batch_destroy(dbm_batch *b)
{
    if (!b) return;
    for (int g = 0; g < 2; ++g)
        if (b->graph[g]) cudaGraphExecDestroy(b->graph[g]);
    free(b->host);
    delete b;
}

}  // extern "C"
