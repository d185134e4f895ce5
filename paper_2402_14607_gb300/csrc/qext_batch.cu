// Batched extraction: many stream pairs of uneven length and mixed block size
// (q = n/n_p in {1, 2, 4, 8, 16, 32, 64}) in ONE persistent kernel launch.
//
// Each stream's blocks are cut into tiles (T blocks; for q <= 16, T = 128 *
// blocks-per-thread).  The tiles of all streams form a table on the device,
// sorted by estimated cost, largest first; persistent CTAs take tiles from an
// atomic counter (reset by a memset node before the kernel), so long q = 64
// tiles start early and short tiles fill the end.  A tile arrives in shared
// memory by two TMA bulk copies (mbarrier, bounded wait) when its stream is
// 16-byte aligned, else by plain loads; threads compute blocks (Ext_IP,
// Definition 3.2) exactly as the single-stream kernel does and warps assemble
// the m-bit outputs of 32 consecutive blocks.
//
// Tile shape (blocks per thread for q = 4 and q = 16) and CTAs per SM are the
// tunables; qext_batch_autotune times the candidates on the batch itself.
// qext_batch_capture records memset + kernel into a CUDA graph.
//
// Streams of raw b-bit samples (qext_batch_create_samples) are packed by the
// CTA from global memory straight into the tile buffer (the fused ingest of
// qext_extract_samples), so a batch of ADC streams is one launch with no
// packed copy in device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "qext_block.cuh"
#include "qext_wide.cuh"
#include "qext_internal.h"
#include "qext_nvtx.h"

using namespace qxd;

namespace {

constexpr int kThreads = 128;
constexpr int kSmemBytes = 64 * 1024;  // one tile buffer (x and y)

struct BatchStreamDev {
    StreamArgs s;
    uint32_t q;
    uint32_t tma;  // x, y 16-byte aligned
    // raw samples (b = 8, 12 or 16; b = 0: packed words in s.x, s.y)
    const uint16_t *sx;
    const uint16_t *sy;
    uint64_t nsamples;
    uint32_t b;
};

struct BatchTileDev {
    uint32_t item;
    uint32_t nb;     // blocks in the tile
    uint64_t first;  // first block
};

// no_copy (test of failure detection): the barrier is armed but no copy is
// issued, so the bounded wait gives up.
__device__ __forceinline__ void load_tile(const StreamArgs &s, uint64_t first, uint32_t nb, int tma, uint32_t *xs,
                                          uint32_t *ys, uint64_t *bar, uint32_t &uses, bool &ok, uint32_t max_polls,
                                          int no_copy) {
    const uint32_t words = nb * s.wpb;
    const uint32_t tid = threadIdx.x;
    if (tma && (words % 4u) == 0) {
        if (tid == 0) {
            mbar_expect_tx(bar, 8u * words);
            if (!no_copy) {
                tma_load_1d(xs, s.x + first * s.wpb, 4u * words, bar);
                tma_load_1d(ys, s.y + first * s.wpb, 4u * words, bar);
            }
        }
        ok = mbar_wait_bounded(bar, uses & 1u, max_polls);
        ++uses;
    } else {
        for (uint32_t i = tid; i < words; i += blockDim.x) {
            xs[i] = __ldg(s.x + first * s.wpb + i);
            ys[i] = __ldg(s.y + first * s.wpb + i);
        }
        ok = true;
    }
}

template <int Q>
__device__ __forceinline__ void compute_tile(const StreamArgs &s, uint64_t first, uint32_t nb, uint32_t *xs,
                                             uint32_t *ys, uint64_t *vals) {
    const uint32_t tid = threadIdx.x;
    if constexpr (Q == 64) {
        // two threads per block, 64 blocks per pass
        for (uint32_t base = 0; base < nb; base += kThreads / 2) {
            const uint32_t lb = base + tid / 2, part = tid & 1u;
            uint64_t A = 0, B = 0, C = 0;
            if (lb < nb) {
                uint32_t *xb = xs + lb * s.wpb, *yb = ys + lb * s.wpb;
                if (s.wpb % 4 == 0)
                    half_products64_inplace(xb, yb, s.wpb, tid, part, 2, A, B, C, s);
                else
                    half_products64(xb, yb, s.wpb, 0, tid, part, 2, A, B, C, s);
            }
            A ^= __shfl_xor_sync(0xffffffffu, A, 1);
            B ^= __shfl_xor_sync(0xffffffffu, B, 1);
            C ^= __shfl_xor_sync(0xffffffffu, C, 1);
            if (lb < nb && part == 0) vals[lb] = combine_q64(A, B, C, s) & mask_m(s.m);
        }
        fence_proxy_async_smem();  // slices written over the tile, which a bulk copy refills later
    } else {
        for (uint32_t lb = tid; lb < nb; lb += kThreads)
            vals[lb] = block_small_q<Q>(xs + lb * s.wpb, ys + lb * s.wpb, s.wpb, s.wpb % 4 == 0, tid, s) &
                       mask_m(s.m);
    }
}

__global__ void __launch_bounds__(kThreads) batch_kernel(const BatchStreamDev *__restrict__ items,
                                                         const BatchTileDev *__restrict__ tiles, uint32_t ntiles,
                                                         unsigned long long *counter, uint32_t max_polls,
                                                         int no_copy) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long next_tile;
    __shared__ uint64_t vals[512];
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses = 0;
    for (;;) {
        if (tid == 0) next_tile = atomicAdd(counter, 1ull);
        __syncthreads();
        const uint64_t t = next_tile;
        if (t >= ntiles) return;
        const BatchTileDev tl = tiles[t];
        const BatchStreamDev it = items[tl.item];
        const StreamArgs &s = it.s;
        const uint32_t words = tl.nb * s.wpb;
        uint32_t *xs = smem, *ys = smem + words;
        bool ok = true;
        if (it.b) {
            // fused ingest: the tile's samples packed from global memory into the buffer
            const uint64_t w0 = tl.first * s.wpb;
            if (it.b == 8)
                pack_tile<8>(it.sx, it.sy, it.nsamples, w0, words, xs, ys, tid, kThreads);
            else if (it.b == 12)
                pack_tile<12>(it.sx, it.sy, it.nsamples, w0, words, xs, ys, tid, kThreads);
            else
                pack_tile<16>(it.sx, it.sy, it.nsamples, w0, words, xs, ys, tid, kThreads);
        } else {
            load_tile(s, tl.first, tl.nb, it.tma, xs, ys, &bar, uses, ok, max_polls, no_copy);
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                record_status(s.status, QEXT_E_TIMEOUT);
                if (!no_copy) mbar_wait_bounded(&bar, (uses - 1) & 1u, max_polls);  // let the copy in flight land
            }
            return;
        }
        for (uint32_t i = tid; i < ((tl.nb + 31u) & ~31u); i += kThreads) vals[i] = 0;
        __syncthreads();
        switch (it.q) {
            case 1: compute_tile<1>(s, tl.first, tl.nb, xs, ys, vals); break;
            case 2: compute_tile<2>(s, tl.first, tl.nb, xs, ys, vals); break;
            case 4: compute_tile<4>(s, tl.first, tl.nb, xs, ys, vals); break;
            case 8: compute_tile<8>(s, tl.first, tl.nb, xs, ys, vals); break;
            case 16: compute_tile<16>(s, tl.first, tl.nb, xs, ys, vals); break;
            case 32: compute_tile<32>(s, tl.first, tl.nb, xs, ys, vals); break;
            default: compute_tile<64>(s, tl.first, tl.nb, xs, ys, vals); break;
        }
        __syncthreads();
        // warps assemble 32 consecutive blocks at a time (tiles start at
        // multiples of 32 blocks within their stream)
        for (uint32_t g = tid >> 5; g * 32 < tl.nb; g += kThreads / 32)
            store_warp(vals[32 * g + (tid & 31u)], tl.first + 32 * g, s.nblocks, s.m, s.out);
        __syncthreads();
    }
}

// relative cost of one block (ALU work), for ordering tiles
double block_cost(uint32_t q, uint32_t wpb) {
    const double per_word = q <= 4 ? 4.0 : q <= 16 ? 14.0 : q <= 32 ? 30.0 : 64.0;
    return per_word * wpb;
}

}  // namespace

struct qext_batch {
    std::vector<BatchStreamDev> items;
    std::vector<uint64_t> nblocks;
    qext_batch_config cfg;
    BatchStreamDev *d_items = nullptr;
    BatchTileDev *d_tiles = nullptr;
    unsigned long long *d_counter = nullptr;  // 64-bit: every CTA takes one index past the last tile
    uint32_t ntiles = 0;
    size_t tiles_cap = 0;
    int sms = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_def = nullptr;
};

namespace {

uint32_t tile_blocks(const qext_batch_config &c, uint32_t q, uint32_t wpb) {
    uint32_t T;
    if (q == 64)
        T = 64;
    else if (q == 32)
        T = 128;
    else if (q <= 4)
        T = 128 * c.blocks_per_thread_small;
    else
        T = 128 * c.blocks_per_thread_mid;
    // one tile (x and y) must fit the shared-memory buffer; keep T a multiple of 32
    while (T > 32 && uint64_t(T) * wpb * 8 > uint64_t(kSmemBytes)) T /= 2;
    if (T > 512) T = 512;
    return T;
}

int build_tiles(qext_batch *b) {
    struct HostTile {
        BatchTileDev t;
        double cost;
    };
    std::vector<HostTile> tiles;
    for (uint32_t i = 0; i < b->items.size(); ++i) {
        const BatchStreamDev &it = b->items[i];
        const uint32_t T = tile_blocks(b->cfg, it.q, it.s.wpb);
        if (uint64_t(T) * it.s.wpb * 8 > uint64_t(kSmemBytes)) return QEXT_E_UNSUPPORTED;
        for (uint64_t f = 0; f < it.s.nblocks; f += T) {
            HostTile h;
            h.t.item = i;
            h.t.first = f;
            h.t.nb = uint32_t(std::min<uint64_t>(T, it.s.nblocks - f));
            h.cost = h.t.nb * block_cost(it.q, it.s.wpb) * (it.b ? 1.25 : 1.0);  // the ingest adds ~a quarter
            tiles.push_back(h);
        }
    }
    if (b->cfg.order == 0)
        std::stable_sort(tiles.begin(), tiles.end(), [](const HostTile &a, const HostTile &c) { return a.cost > c.cost; });
    if (tiles.size() > 0xFFFFFFFFull) return QEXT_E_INVAL;
    b->ntiles = uint32_t(tiles.size());
    if (b->ntiles > b->tiles_cap) {
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        if (cudaMalloc(&b->d_tiles, sizeof(BatchTileDev) * b->ntiles) != cudaSuccess) return QEXT_E_CUDA;
        b->tiles_cap = b->ntiles;
    }
    std::vector<BatchTileDev> flat(b->ntiles);
    for (uint32_t i = 0; i < b->ntiles; ++i) flat[i] = tiles[i].t;
    if (b->ntiles && cudaMemcpy(b->d_tiles, flat.data(), sizeof(BatchTileDev) * b->ntiles,
                                cudaMemcpyHostToDevice) != cudaSuccess)
        return QEXT_E_CUDA;
    return QEXT_OK;
}

int enqueue(qext_batch *b, cudaStream_t st, uint32_t flags = 0) {
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(*b->d_counter), st) != cudaSuccess) return QEXT_E_CUDA;
    if (!b->ntiles) return QEXT_OK;
    const uint64_t cap = uint64_t(b->sms) * b->cfg.ctas_per_sm;
    const int grid = int(std::min<uint64_t>(cap, b->ntiles));
    const int no_copy = (flags & QEXT_F_TEST_TIMEOUT) ? 1 : 0;
    batch_kernel<<<grid, kThreads, kSmemBytes, st>>>(b->d_items, b->d_tiles, b->ntiles, b->d_counter,
                                                     no_copy ? 256u : kMaxPolls, no_copy);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

void drop_graph(qext_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_def) cudaGraphDestroy(b->graph_def);
    b->graph = nullptr;
    b->graph_def = nullptr;
}

}  // namespace

namespace {

// The device descriptor of one stream (pointers filled by the caller).
BatchStreamDev stream_dev(const qext_plan *plan, uint64_t nblocks, uint32_t *out) {
    BatchStreamDev d;
    std::memset(&d, 0, sizeof d);
    d.s.out = out;
    d.s.nblocks = nblocks;
    d.s.wpb = plan->n / 32;
    d.s.m = plan->m;
    d.s.ntaps = plan->ntaps;
    for (int k = 0; k < 4; ++k) d.s.taps[k] = plan->taps[k];
    d.s.set_multipliers();
    d.s.status = qext::device_status_ptr();
    d.q = plan->q;
    return d;
}

// Device tables and tiles for validated descriptors.
int create_batch(const std::vector<BatchStreamDev> &devs, qext_batch **out) {
    static qext::DeviceSlots attr_set;
    const int dev = qext::current_device();
    if (dev < 0 || attr_set.get(dev, [] {
            return cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) ==
                           cudaSuccess ? 1 : 0;
        }) <= 0)
        return QEXT_E_CUDA;
    qext_batch *b = new (std::nothrow) qext_batch();
    if (!b) return QEXT_E_INVAL;
    b->cfg.blocks_per_thread_small = 4;
    b->cfg.blocks_per_thread_mid = 1;
    b->cfg.ctas_per_sm = 3;
    b->cfg.order = 0;
    b->sms = qext::sm_count(dev);
    b->items = devs;
    const size_t nitems = devs.size();
    if (b->sms <= 0 || cudaMalloc(&b->d_counter, sizeof(*b->d_counter)) != cudaSuccess ||
        (nitems && cudaMalloc(&b->d_items, sizeof(BatchStreamDev) * nitems) != cudaSuccess) ||
        (nitems && cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchStreamDev) * nitems,
                              cudaMemcpyHostToDevice) != cudaSuccess)) {
        qext_batch_destroy(b);
        return QEXT_E_CUDA;
    }
    const int rc = build_tiles(b);
    if (rc != QEXT_OK) {
        qext_batch_destroy(b);
        return rc;
    }
    *out = b;
    return QEXT_OK;
}

}  // namespace

extern "C" {

int qext_batch_create(const qext_batch_item *items, uint32_t nitems, qext_batch **out) {
    if (!out || (nitems && !items)) return QEXT_E_INVAL;
    *out = nullptr;
    std::vector<BatchStreamDev> devs;
    devs.reserve(nitems);
    for (uint32_t i = 0; i < nitems; ++i) {
        const qext_batch_item &it = items[i];
        if (!it.plan) return QEXT_E_INVAL;
        if (!it.plan->gpu_supported) return QEXT_E_UNSUPPORTED;
        const uintptr_t al = reinterpret_cast<uintptr_t>(it.x) | reinterpret_cast<uintptr_t>(it.y);
        if (it.nblocks && (!it.x || !it.y || !it.out || al % 4 || reinterpret_cast<uintptr_t>(it.out) % 4))
            return QEXT_E_INVAL;
        BatchStreamDev d = stream_dev(it.plan, it.nblocks, it.out);
        d.s.x = it.x;
        d.s.y = it.y;
        d.tma = al % 16 == 0;
        devs.push_back(d);
    }
    return create_batch(devs, out);
}

int qext_batch_create_samples(const qext_batch_samples_item *items, uint32_t nitems, qext_batch **out) {
    if (!out || (nitems && !items)) return QEXT_E_INVAL;
    *out = nullptr;
    std::vector<BatchStreamDev> devs;
    devs.reserve(nitems);
    for (uint32_t i = 0; i < nitems; ++i) {
        const qext_batch_samples_item &it = items[i];
        if (!it.plan) return QEXT_E_INVAL;
        if (it.b != 8 && it.b != 12 && it.b != 16) return QEXT_E_UNSUPPORTED;
        if (!it.plan->gpu_supported) return QEXT_E_UNSUPPORTED;
        const uintptr_t al = reinterpret_cast<uintptr_t>(it.x_samples) | reinterpret_cast<uintptr_t>(it.y_samples);
        if (it.nblocks && (!it.x_samples || !it.y_samples || !it.out || al % 16 ||
                           reinterpret_cast<uintptr_t>(it.out) % 4))
            return QEXT_E_INVAL;
        if (it.nsamples > UINT64_MAX / 16 || it.nblocks > (it.nsamples * it.b) / it.plan->n) return QEXT_E_INVAL;
        BatchStreamDev d = stream_dev(it.plan, it.nblocks, it.out);
        d.sx = it.x_samples;
        d.sy = it.y_samples;
        d.nsamples = it.nsamples;
        d.b = it.b;
        devs.push_back(d);
    }
    return create_batch(devs, out);
}

int qext_batch_destroy(qext_batch *b) {
    if (!b) return QEXT_OK;
    drop_graph(b);
    cudaFree(b->d_items);
    cudaFree(b->d_tiles);
    cudaFree(b->d_counter);
    delete b;
    return QEXT_OK;
}

int qext_batch_get_config(const qext_batch *b, qext_batch_config *cfg, uint32_t *ntiles) {
    if (!b) return QEXT_E_INVAL;
    if (cfg) *cfg = b->cfg;
    if (ntiles) *ntiles = b->ntiles;
    return QEXT_OK;
}

int qext_batch_set_config(qext_batch *b, const qext_batch_config *cfg) {
    if (!b || !cfg) return QEXT_E_INVAL;
    const qext_batch_config &c = *cfg;
    const bool ok = (c.blocks_per_thread_small == 1 || c.blocks_per_thread_small == 2 ||
                     c.blocks_per_thread_small == 4) &&
                    (c.blocks_per_thread_mid == 1 || c.blocks_per_thread_mid == 2 ||
                     c.blocks_per_thread_mid == 4) &&
                    c.ctas_per_sm >= 1 && c.ctas_per_sm <= 3 && c.order <= 1;
    if (!ok) return QEXT_E_INVAL;
    b->cfg = c;
    drop_graph(b);
    return build_tiles(b);
}

int qext_batch_run(qext_batch *b, qext_cuda_stream stream) { return qext_batch_run_ex(b, stream, 0); }

int qext_batch_run_ex(qext_batch *b, qext_cuda_stream stream, uint32_t flags) {
    if (!b) return QEXT_E_INVAL;
    if (flags & ~uint32_t(QEXT_F_TEST_TIMEOUT)) return QEXT_E_INVAL;
    if (flags) {
        // the test needs every tile on the bulk-copy path (sample tiles take none)
        for (const BatchStreamDev &d : b->items)
            if (d.s.nblocks && (!d.tma || d.b)) return QEXT_E_INVAL;
    }
    const qext::NvtxRange range("qext batch run");
    return enqueue(b, reinterpret_cast<cudaStream_t>(stream), flags);
}

int qext_batch_capture(qext_batch *b, qext_cuda_stream stream) {
    if (!b) return QEXT_E_INVAL;
    drop_graph(b);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return QEXT_E_CUDA;
    const int rc = enqueue(b, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != QEXT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != QEXT_OK ? rc : QEXT_E_CUDA;
    }
    if (cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return QEXT_E_CUDA;
    }
    b->graph_def = g;
    return QEXT_OK;
}

int qext_batch_launch(qext_batch *b, qext_cuda_stream stream) {
    if (!b) return QEXT_E_INVAL;
    if (!b->graph) return QEXT_E_STATE;
    const qext::NvtxRange range("qext batch (graph launch)");
    return cudaGraphLaunch(b->graph, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

int qext_batch_autotune(qext_batch *b, uint32_t reps, qext_cuda_stream stream, float *best_ms) {
    if (!b || reps == 0) return QEXT_E_INVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QEXT_E_CUDA;
    qext_batch_config best = b->cfg;
    float best_t = 1e30f;
    int rc = QEXT_OK;
    for (uint32_t small : {1u, 2u, 4u})
        for (uint32_t mid : {1u, 2u})
            for (uint32_t ctas : {2u, 3u})
                for (uint32_t order : {0u, 1u}) {
                    qext_batch_config c{small, mid, ctas, order};
                    if ((rc = qext_batch_set_config(b, &c)) != QEXT_OK) goto done;
                    if ((rc = enqueue(b, st)) != QEXT_OK) goto done;  // warm-up
                    cudaEventRecord(e0, st);
                    for (uint32_t r = 0; r < reps; ++r)
                        if ((rc = enqueue(b, st)) != QEXT_OK) goto done;
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        rc = QEXT_E_CUDA;
                        goto done;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= float(reps);
                    if (ms < best_t) {
                        best_t = ms;
                        best = c;
                    }
                }
    rc = qext_batch_set_config(b, &best);
    if (best_ms) *best_ms = best_t;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batch run (qext_batch_run_noalloc).  Same per-tile work as
// batch_kernel, but the descriptors and the tile counter live in a fixed
// static device array instead of cudaMalloc'ed tables, and tiles are found
// from per-stream tile prefix counts rather than a tile table.
// ---------------------------------------------------------------------------
namespace {

struct NoallocScratch {
    unsigned long long counter;  // next tile; 0 at the start of every call (64-bit: cannot wrap)
    uint32_t nitems;
    uint64_t total_tiles;
    uint64_t tile_prefix[QEXT_NOALLOC_MAX_ITEMS + 1];  // tiles of the items before item i
    uint32_t tile_blocks[QEXT_NOALLOC_MAX_ITEMS];
    BatchStreamDev items[QEXT_NOALLOC_MAX_ITEMS];
};

// Scratch of the allocation-free entry point: one per device, held until the
// process exits, shared by every call (see qext_batch_run_noalloc).  The size
// quoted in the header (about 200 KB) is kept by this bound.
static_assert(sizeof(NoallocScratch) <= 200 * 1024, "the documented static scratch size");
static __device__ __align__(256) unsigned char qext_noalloc_scratch[sizeof(NoallocScratch)];

__global__ void __launch_bounds__(kThreads) batch_noalloc_kernel(NoallocScratch *sc) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long next_tile;
    __shared__ uint64_t vals[512];
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses = 0;
    for (;;) {
        if (tid == 0) next_tile = atomicAdd(&sc->counter, 1ull);
        __syncthreads();
        const uint64_t t = next_tile;
        if (t >= sc->total_tiles) return;
        uint32_t lo = 0, hi = sc->nitems;  // last item whose prefix <= t
        while (lo + 1 < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (sc->tile_prefix[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        const BatchStreamDev it = sc->items[lo];
        const StreamArgs &s = it.s;
        const uint32_t T = sc->tile_blocks[lo];
        const uint64_t first = (t - sc->tile_prefix[lo]) * T;
        const uint32_t nb = uint32_t(s.nblocks - first < T ? s.nblocks - first : T);
        const uint32_t words = nb * s.wpb;
        uint32_t *xs = smem, *ys = smem + words;
        bool ok;
        load_tile(s, first, nb, it.tma, xs, ys, &bar, uses, ok, kMaxPolls, 0);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                record_status(s.status, QEXT_E_TIMEOUT);
                mbar_wait_bounded(&bar, (uses - 1) & 1u);
            }
            return;
        }
        for (uint32_t i = tid; i < ((nb + 31u) & ~31u); i += kThreads) vals[i] = 0;
        __syncthreads();
        switch (it.q) {
            case 1: compute_tile<1>(s, first, nb, xs, ys, vals); break;
            case 2: compute_tile<2>(s, first, nb, xs, ys, vals); break;
            case 4: compute_tile<4>(s, first, nb, xs, ys, vals); break;
            case 8: compute_tile<8>(s, first, nb, xs, ys, vals); break;
            case 16: compute_tile<16>(s, first, nb, xs, ys, vals); break;
            case 32: compute_tile<32>(s, first, nb, xs, ys, vals); break;
            default: compute_tile<64>(s, first, nb, xs, ys, vals); break;
        }
        __syncthreads();
        for (uint32_t g = tid >> 5; g * 32 < nb; g += kThreads / 32)
            store_warp(vals[32 * g + (tid & 31u)], first + 32 * g, s.nblocks, s.m, s.out);
        __syncthreads();
    }
}

// Validates the items and fills the descriptor table h (header, per-item
// descriptors in the given order, tile prefix sums), as both table entry
// points need it: every item has a plan with GPU kernels, non-null 4-byte
// aligned pointers (when it has blocks) and a tile that fits the kernel's
// shared memory; at most QEXT_NOALLOC_MAX_ITEMS items and 2^32 - 1 tiles.
// order == nullptr keeps the caller's order.
int fill_table(const qext_batch_item *items, uint32_t nitems, const uint32_t *order, NoallocScratch *h) {
    if (nitems > QEXT_NOALLOC_MAX_ITEMS) return QEXT_E_LIMIT;
    if (nitems && !items) return QEXT_E_INVAL;
    h->counter = 0;
    h->nitems = nitems;
    const qext_batch_config cfg{4, 1, 3, 0};
    uint64_t tiles = 0;
    for (uint32_t k = 0; k < nitems; ++k) {
        const qext_batch_item &it = items[order ? order[k] : k];
        if (!it.plan) return QEXT_E_INVAL;
        if (!it.plan->gpu_supported) return QEXT_E_UNSUPPORTED;
        const uintptr_t al = reinterpret_cast<uintptr_t>(it.x) | reinterpret_cast<uintptr_t>(it.y);
        if (it.nblocks && (!it.x || !it.y || !it.out || al % 4 || reinterpret_cast<uintptr_t>(it.out) % 4))
            return QEXT_E_INVAL;
        BatchStreamDev &d = h->items[k];
        std::memset(&d, 0, sizeof d);
        d.s.x = it.x;
        d.s.y = it.y;
        d.s.out = it.out;
        d.s.nblocks = it.nblocks;
        d.s.wpb = it.plan->n / 32;
        d.s.m = it.plan->m;
        d.s.ntaps = it.plan->ntaps;
        for (int j = 0; j < 4; ++j) d.s.taps[j] = it.plan->taps[j];
        d.s.set_multipliers();
        d.s.status = qext::device_status_ptr();
        d.q = it.plan->q;
        d.tma = al % 16 == 0;
        const uint32_t T = tile_blocks(cfg, d.q, d.s.wpb);
        if (uint64_t(T) * d.s.wpb * 8 > uint64_t(kSmemBytes)) return QEXT_E_UNSUPPORTED;
        h->tile_blocks[k] = T;
        h->tile_prefix[k] = tiles;
        tiles += (it.nblocks + T - 1) / T;
    }
    if (tiles > 0xFFFFFFFFull) return QEXT_E_LIMIT;
    h->tile_prefix[nitems] = tiles;
    h->total_tiles = tiles;
    return QEXT_OK;
}

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_dev[kNoallocMaxDevices];                 // device address of the scratch, per device
unsigned char g_noalloc_stage[sizeof(NoallocScratch)];  // host staging (static: no heap)

}  // namespace

extern "C" int qext_batch_run_noalloc(const qext_batch_item *items, uint32_t nitems, qext_cuda_stream stream) {
    if (nitems > QEXT_NOALLOC_MAX_ITEMS) return QEXT_E_LIMIT;
    if (nitems && !items) return QEXT_E_INVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The descriptors are copied from a static host buffer that the next call
    // rewrites; a captured copy would read that buffer at replay time, so a
    // capturing stream is refused before anything is enqueued.
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap_status) != cudaSuccess) return QEXT_E_CUDA;
    if (cap_status != cudaStreamCaptureStatusNone) return QEXT_E_STATE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QEXT_E_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return QEXT_E_LIMIT;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    // one-time set-up on this device (the first call, with the device current)
    if (!g_noalloc_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, qext_noalloc_scratch) != cudaSuccess || !p) return QEXT_E_CUDA;
        if (cudaFuncSetAttribute(batch_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
            cudaSuccess)
            return QEXT_E_CUDA;
        g_noalloc_dev[dev] = p;
    }
    for (uint32_t i = 0; i < nitems; ++i)
        if (!items[i].plan) return QEXT_E_INVAL;
    // heavier streams first, so their tiles are taken first
    uint32_t order[QEXT_NOALLOC_MAX_ITEMS];
    for (uint32_t i = 0; i < nitems; ++i) order[i] = i;
    std::stable_sort(order, order + nitems,
                     [&](uint32_t a, uint32_t c) { return items[a].plan->q > items[c].plan->q; });
    NoallocScratch *h = reinterpret_cast<NoallocScratch *>(g_noalloc_stage);
    const int rc = fill_table(items, nitems, order, h);
    if (rc != QEXT_OK) return rc;
    // the whole header plus the used part of the item table; the copy from
    // pageable host memory is staged before cudaMemcpyAsync returns
    const size_t bytes = offsetof(NoallocScratch, items) + sizeof(BatchStreamDev) * nitems;
    if (cudaMemcpyAsync(g_noalloc_dev[dev], g_noalloc_stage, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return QEXT_E_CUDA;
    const uint64_t tiles = h->total_tiles;
    if (!tiles) return QEXT_OK;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QEXT_E_CUDA;
    const uint64_t cap = uint64_t(sms) * 3;
    const int grid = int(tiles < cap ? tiles : cap);
    batch_noalloc_kernel<<<grid, kThreads, kSmemBytes, st>>>(static_cast<NoallocScratch *>(g_noalloc_dev[dev]));
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

// ---------------------------------------------------------------------------
// Batch launch from caller-provided tables (the serving loop's rounds): the
// descriptors are written to a pinned host staging buffer, copied to the
// caller's device table asynchronously and consumed by the same kernel as the
// allocation-free entry point.  The staging buffer must not be reused until
// the copy has completed (the caller orders that with events).
// ---------------------------------------------------------------------------
namespace qext {

size_t batch_table_bytes() { return sizeof(NoallocScratch); }

int batch_launch_tables(const qext_batch_item *items, uint32_t nitems, void *d_table, void *h_stage,
                        qext_cuda_stream stream) {
    static qext::DeviceSlots attr_set;
    const int dev = qext::current_device();
    if (dev < 0 || attr_set.get(dev, [] {
            return cudaFuncSetAttribute(batch_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes) == cudaSuccess ? 1 : 0;
        }) <= 0)
        return QEXT_E_CUDA;
    if (!d_table || !h_stage) return QEXT_E_INVAL;
    NoallocScratch *h = static_cast<NoallocScratch *>(h_stage);
    const int rc = fill_table(items, nitems, nullptr, h);
    if (rc != QEXT_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = offsetof(NoallocScratch, items) + sizeof(BatchStreamDev) * nitems;
    if (cudaMemcpyAsync(d_table, h_stage, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return QEXT_E_CUDA;
    const uint64_t tiles = h->total_tiles;
    if (!tiles) return QEXT_OK;
    const int sms = qext::sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    const uint64_t cap = uint64_t(sms) * 3;
    const int grid = int(tiles < cap ? tiles : cap);
    batch_noalloc_kernel<<<grid, kThreads, kSmemBytes, st>>>(static_cast<NoallocScratch *>(d_table));
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

}  // namespace qext
