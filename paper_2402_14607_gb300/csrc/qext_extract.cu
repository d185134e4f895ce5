// Per-block extraction Ext_IP^{n_p,q} (Definition 3.2) inside Algorithm 1's
// block loop, for GB300 (sm_103a).  See qext_device.cuh for the sliced GF(2)
// formulation.
//
// Tiled kernel (qext_extract's path; with B != 0 the CTA-tile variant of
// qext_extract_samples, whose default for q = 4, 16 is the per-warp kernel
// of qext_extract_raw.cu).  A persistent CTA walks tiles of T consecutive
// blocks.  Each tile of x and y arrives in shared memory by two
// 1-D TMA bulk copies (cp.async.bulk, completion on an mbarrier); the copy of
// the next tile is issued before the current one is computed (two buffers).
// Each thread (two for q = 64) computes one block from shared memory, reading
// its 16-byte chunks in a lane-rotated order so that eight consecutive lanes
// hit eight different bank groups (q = 64 writes its slices back over its own
// part of the tile and reads them again: half_products64_inplace).  Block
// values go to shared memory and warps
// assemble m-bit outputs of 32 consecutive blocks into whole words.  From raw
// samples (B != 0) the tile's samples arrive by TMA and are packed in place.
//
// Direct kernel (fallback for blocks too long to stage): each thread loads its
// own block from global memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_block.cuh"
#include "qext_wide.cuh"
#include "qext_internal.h"

using namespace qxd;

namespace {

constexpr int kThreads = 128;
constexpr int kSmemBudget = 100 * 1024;  // per CTA: at least two CTAs per SM

struct TileArgs {
    StreamArgs s;
    const uint16_t *sx;  // raw ADC samples (fused ingest), else null
    const uint16_t *sy;
    uint64_t nsamples;
    uint64_t ntiles;
    uint32_t T;     // blocks per tile (multiple of 32)
    uint32_t nbuf;  // 1 or 2 tile buffers
    int tma;        // x, y 16-byte aligned: full tiles arrive by bulk copy
    int vec;        // wpb % 4 == 0: 16-byte shared-memory reads
    uint32_t max_polls;  // bound of every mbarrier wait
    int no_copy;         // test of the timeout path: arm the barrier, issue no copy
    uint32_t raw_periods;  // fused ingest: raw buffer capacity per source, in periods of 8 samples
    int raw_prefetch;      // fused ingest: two raw buffers, next tile's copy issued before computing
};

template <int Q>
struct QTraits {
    static constexpr int TPB = Q == 64 ? 2 : 1;  // threads per block
};

// ---------------------------------------------------------------------------
// Tiled kernel.  B = 0: packed words arrive by TMA; B = 8, 12, 16: the tile
// is packed from raw samples by the CTA (fused ingest).
// ---------------------------------------------------------------------------
template <int Q, int B>
__global__ void __launch_bounds__(kThreads) extract_tiled_kernel(const TileArgs ta) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ uint64_t vals[kThreads];
    constexpr int TPB = QTraits<Q>::TPB;
    const StreamArgs &s = ta.s;
    const uint32_t tid = threadIdx.x;
    const uint32_t T = ta.T;
    const uint32_t tw = T * s.wpb;  // words per tile per source
    const uint32_t nthreads = T * TPB;
    uint32_t *const buf1 = smem + (ta.nbuf > 1 ? 2 * tw : 0);  // second tile buffer

    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_prologue();

    auto full_tile = [&](uint64_t t) { return (t + 1) * uint64_t(T) <= s.nblocks; };
    auto issue = [&](uint64_t t, int b) {
        const uint32_t bytes = tw * 4u;
        mbar_expect_tx(&full[b], 2u * bytes);
        if (ta.no_copy) return;  // the completion never comes: the wait must give up
        uint32_t *dst = b ? buf1 : smem;
        tma_load_1d(dst, s.x + t * tw, bytes, &full[b]);
        tma_load_1d(dst + tw, s.y + t * tw, bytes, &full[b]);
    };

    uint64_t tile = blockIdx.x;
    uint32_t raw_uses0 = 0, raw_uses1 = 0;  // fused ingest: completed uses of full[0], full[1]
    bool prefetched = false;         // fused ingest (thread 0): this tile's copy was issued last iteration
    // fused ingest: the raw samples of tile t fit the raw buffer and lie in the array
    auto raw_tile_ok = [&](uint64_t t) {
        if (!ta.raw_periods || B == 0) return false;
        constexpr uint32_t WP = B == 12 ? 3u : B == 8 ? 2u : 4u;
        const uint64_t nbt = s.nblocks - t * T < T ? s.nblocks - t * T : T;
        const uint64_t w0t = t * tw, p0t = w0t / WP;
        const uint32_t np = uint32_t((w0t - p0t * WP + nbt * s.wpb + WP - 1) / WP);
        return np <= ta.raw_periods && 8 * (p0t + np) <= ta.nsamples;
    };
    auto issue_raw = [&](uint64_t t, int rbuf) {
        constexpr uint32_t WP = B == 12 ? 3u : B == 8 ? 2u : 4u;
        const uint64_t nbt = s.nblocks - t * T < T ? s.nblocks - t * T : T;
        const uint64_t w0t = t * tw, p0t = w0t / WP;
        const uint32_t np = uint32_t((w0t - p0t * WP + nbt * s.wpb + WP - 1) / WP);
        uint4 *rx = reinterpret_cast<uint4 *>(smem) + size_t(rbuf) * 2 * ta.raw_periods, *ry = rx + ta.raw_periods;
        mbar_expect_tx(&full[rbuf], 32u * np);
        tma_load_1d(rx, ta.sx + 8 * p0t, 16u * np, &full[rbuf]);
        tma_load_1d(ry, ta.sy + 8 * p0t, 16u * np, &full[rbuf]);
    };
    if (tid == 0 && ta.tma && tile < ta.ntiles && full_tile(tile)) issue(tile, 0);
    for (uint32_t k = 0; tile < ta.ntiles; ++k, tile += gridDim.x) {
        const int b = ta.nbuf > 1 ? int(k & 1u) : 0;
        const uint64_t next = tile + gridDim.x;
        if (tid == 0 && ta.tma) {
            if (ta.nbuf > 1) {
                if (next < ta.ntiles && full_tile(next)) issue(next, b ^ 1);  // prefetch
            } else if (k > 0 && full_tile(tile)) {
                issue(tile, 0);  // single buffer: free since the last __syncthreads
            }
        }
        uint32_t *xs = b ? buf1 : smem, *ys = xs + tw;
        if constexpr (B != 0) {
            // fused ingest: the tile's raw samples arrive by TMA and are packed
            // in place (one buffer per CTA), else they are packed from global
            // memory (the stream's last tiles)
            constexpr uint32_t WP = PeriodOf<B>::kWords;
            const uint64_t nb = s.nblocks - tile * T < T ? s.nblocks - tile * T : T;
            const uint32_t nw = uint32_t(nb * s.wpb);
            const uint64_t w0 = tile * tw, p0 = w0 / WP;
            const uint32_t phi = uint32_t(w0 - p0 * WP);
            // raw buffers of raw_periods periods each, or (no raw staging) the
            // packed tile's usual x / y halves
            const int rb = ta.raw_prefetch ? int(k & 1u) : 0;  // raw buffer of this tile
            uint4 *raw_x = reinterpret_cast<uint4 *>(smem) + size_t(rb) * 2 * ta.raw_periods;
            uint4 *raw_y = ta.raw_periods ? raw_x + ta.raw_periods : reinterpret_cast<uint4 *>(smem + tw);
            xs = reinterpret_cast<uint32_t *>(raw_x);
            ys = reinterpret_cast<uint32_t *>(raw_y);
            bool packed = false;
            if (raw_tile_ok(tile)) {
                if (tid == 0) {
                    if (!prefetched) issue_raw(tile, rb);
                    prefetched = ta.raw_prefetch && next < ta.ntiles && raw_tile_ok(next);
                    if (prefetched) issue_raw(next, rb ^ 1);
                }
                const uint32_t use = rb ? raw_uses1++ : raw_uses0++;
                const bool ok = mbar_wait_bounded(&full[rb], use & 1u, ta.max_polls);
                if (!__syncthreads_and(ok)) {
                    if (tid == 0) {
                        record_status(s.status, QEXT_E_TIMEOUT);
                        // give the copies in flight a bounded chance to land
                        mbar_wait_bounded(&full[rb], use & 1u, ta.max_polls);
                        if (prefetched) mbar_wait_bounded(&full[rb ^ 1], (rb ? raw_uses0 : raw_uses1) & 1u, ta.max_polls);
                    }
                    return;
                }
                pack_tile_in_place<B>(raw_x, raw_y, phi, nw, tid, nthreads);
                packed = true;
            }
            if (!packed) {
                pack_tile<B>(ta.sx, ta.sy, ta.nsamples, w0, nw, xs, ys, tid, nthreads);
                __syncthreads();
            }
        } else if (ta.tma && full_tile(tile)) {
            const uint32_t use = ta.nbuf > 1 ? (k >> 1) : k;
            const bool ok = mbar_wait_bounded(&full[b], use & 1u, ta.max_polls);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    record_status(s.status, QEXT_E_TIMEOUT);
                    // give the copies in flight a bounded chance to land
                    if (!ta.no_copy) {
                        mbar_wait_bounded(&full[b], use & 1u, ta.max_polls);
                        if (ta.nbuf > 1) mbar_wait_bounded(&full[b ^ 1], ((k + 1) >> 1) & 1u, ta.max_polls);
                    }
                }
                return;
            }
        } else {
            const uint64_t nb = s.nblocks - tile * T < T ? s.nblocks - tile * T : T;
            const uint64_t nw = nb * s.wpb;
            for (uint64_t i = tid; i < nw; i += nthreads) {
                xs[i] = __ldg(s.x + tile * tw + i);
                ys[i] = __ldg(s.y + tile * tw + i);
            }
            __syncthreads();
        }

        // compute: one block per thread (q = 64: two threads per block)
        const uint32_t lb = tid / TPB;
        const uint64_t blk = tile * T + lb;
        uint64_t v = 0;
        if constexpr (Q == 64) {
            const uint32_t part = tid % TPB;
            uint64_t A = 0, Bm = 0, C = 0;
            if (blk < s.nblocks) {
                uint32_t *xb = xs + lb * s.wpb, *yb = ys + lb * s.wpb;
                if (ta.vec)
                    half_products64_inplace(xb, yb, s.wpb, tid, part, TPB, A, Bm, C, s);
                else
                    half_products64(xb, yb, s.wpb, ta.vec, tid, part, TPB, A, Bm, C, s);
            }
            fence_proxy_async_smem();  // slices written over the tile, which a bulk copy refills later
            A ^= __shfl_xor_sync(0xffffffffu, A, 1);
            Bm ^= __shfl_xor_sync(0xffffffffu, Bm, 1);
            C ^= __shfl_xor_sync(0xffffffffu, C, 1);
            if (blk < s.nblocks) v = combine_q64(A, Bm, C, s) & mask_m(s.m);
            if (part == 0) vals[lb] = v;
        } else {
            if (blk < s.nblocks)
                v = block_small_q<Q>(xs + lb * s.wpb, ys + lb * s.wpb, s.wpb, ta.vec, tid, s) &
                    mask_m(s.m);
            vals[lb] = v;
        }
        __syncthreads();
        // output: warp w assembles blocks [32w, 32w + 32) of the tile
        const uint32_t w = tid >> 5;
        if (w < T / 32) store_warp(vals[32 * w + (tid & 31u)], tile * T + 32 * w, s.nblocks, s.m, s.out);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Direct kernel: each thread loads its own block from global memory (blocks
// too long to stage in shared memory).
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(kThreads) extract_direct_kernel(const StreamArgs s) {
    pdl_prologue();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < s.nblocks; base += nwarps * 32) {
        const uint64_t blk = base + lane;
        uint64_t v = 0;
        if (blk < s.nblocks) {
            const uint32_t *xb = s.x + blk * s.wpb, *yb = s.y + blk * s.wpb;
            if constexpr (Q == 64) {
                // scalar loads here: the per-part templates beat the one-copy loop
                const uint64_t A = half_product64<0>(xb, yb, s.wpb, 0, 0, 0, 1, s);
                const uint64_t B = half_product64<1>(xb, yb, s.wpb, 0, 0, 0, 1, s);
                const uint64_t C = half_product64<2>(xb, yb, s.wpb, 0, 0, 0, 1, s);
                v = combine_q64(A, B, C, s);
            } else {
                v = block_small_q<Q>(xb, yb, s.wpb, 0, 0, s);
            }
            v &= mask_m(s.m);
        }
        store_warp(v, base, s.nblocks, s.m, s.out);
    }
}


template <int Q, int B>
int launch_q(const StreamArgs &s, const uint16_t *sx, const uint16_t *sy, uint64_t nsamples, cudaStream_t st,
             uint32_t flags) {
    const bool force_direct = B == 0 && (flags & QEXT_F_DIRECT) && !(flags & QEXT_F_TEST_TIMEOUT);
    const uint32_t t_max = (flags & QEXT_F_TILE32) ? 32u : (flags & QEXT_F_TILE64) ? 64u : 128u;
    const uint32_t nb_max = (flags & QEXT_F_NBUF1) ? 1u : 2u;
    // per device: SM count, "attribute set", occupancies by tile shape
    static qext::DeviceSlots attr_set, occ_tiled[24], occ_direct;
    const int dev = qext::current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int sms = qext::sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    constexpr int TPB = QTraits<Q>::TPB;
    // tile size: the largest T (multiple of 32, T * TPB <= kThreads) whose
    // buffers fit the per-CTA budget, double-buffered if possible; the fused
    // ingest keeps one raw-sample buffer per source (packed in place)
    uint32_t raw_periods = 0;
    if constexpr (B != 0) {
        constexpr uint32_t WP = PeriodOf<B>::kWords;
        const uint32_t T0 = kThreads / TPB;
        raw_periods = (T0 * s.wpb + WP - 1) / WP + 2;
        const size_t smem = size_t(2) * 16 * raw_periods;
        if (smem > size_t(kSmemBudget)) raw_periods = 0;
    }
    uint32_t T = 0, nbuf = 0;
    for (uint32_t t = kThreads / TPB < t_max ? kThreads / TPB : t_max; t >= 32 && !T; t /= 2)
        for (uint32_t nb = nb_max; nb >= 1 && !T; --nb)
            if (uint64_t(nb) * 2 * t * s.wpb * 4 <= uint64_t(kSmemBudget)) {
                T = t;
                nbuf = nb;
            }
    if (T && !force_direct) {
        if (attr_set.get(dev, [] {
                return cudaFuncSetAttribute(extract_tiled_kernel<Q, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSmemBudget) == cudaSuccess ? 1 : 0;
            }) <= 0)
            return QEXT_E_CUDA;
        TileArgs ta;
        ta.s = s;
        ta.sx = sx;
        ta.sy = sy;
        ta.nsamples = nsamples;
        ta.T = T;
        ta.nbuf = nbuf;
        ta.ntiles = (s.nblocks + T - 1) / T;
        const uintptr_t al = reinterpret_cast<uintptr_t>(s.x) | reinterpret_cast<uintptr_t>(s.y);
        ta.tma = B == 0 && al % 16 == 0;
        ta.vec = s.wpb % 4 == 0;
        ta.no_copy = B == 0 && (flags & QEXT_F_TEST_TIMEOUT) ? 1 : 0;
        ta.max_polls = ta.no_copy ? 256u : kMaxPolls;
        if (ta.no_copy && !ta.tma) return QEXT_E_INVAL;  // the test needs the bulk-copy path
        ta.raw_periods = 0;
        size_t smem = size_t(nbuf) * 2 * T * s.wpb * 4;
        ta.raw_prefetch = 0;
        if constexpr (B != 0) {
            nbuf = 1;
            ta.nbuf = 1;
            T = kThreads / TPB;
            ta.T = T;
            ta.ntiles = (s.nblocks + T - 1) / T;
            ta.raw_periods = raw_periods;
            ta.raw_prefetch = raw_periods && (flags & QEXT_F_RAW_PREFETCH) &&
                              size_t(4) * 16 * raw_periods <= size_t(kSmemBudget);
            smem = raw_periods ? size_t(ta.raw_prefetch ? 4 : 2) * 16 * raw_periods : size_t(2) * T * s.wpb * 4;
        }
        const int ti = (T == 32 ? 0 : T == 64 ? 1 : 2) + 3 * int(nbuf - 1) + (B != 0 ? 6 : 0) + 12 * ta.raw_prefetch;
        const int occ = occ_tiled[ti].get(dev, [&] {
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, extract_tiled_kernel<Q, B>, int(T * TPB), smem) !=
                cudaSuccess)
                return 0;
            return o < 1 ? 1 : o;
        });
        if (occ <= 0) return QEXT_E_CUDA;
        const uint64_t cap = uint64_t(sms) * occ;
        const int grid = int(ta.ntiles < cap ? ta.ntiles : cap);
        return qext::launch_pdl(extract_tiled_kernel<Q, B>, grid, int(T * TPB), smem, st, ta);
    } else {
        if (B != 0) return QEXT_E_UNSUPPORTED;  // fused ingest needs a staged tile
        const int occd = occ_direct.get(dev, [] {
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, extract_direct_kernel<Q>, kThreads, 0) != cudaSuccess)
                return 0;
            return o < 1 ? 1 : o;
        });
        if (occd <= 0) return QEXT_E_CUDA;
        const uint64_t ctas = (s.nblocks + kThreads - 1) / kThreads;
        const uint64_t cap = uint64_t(sms) * occd;
        const int grid = int(ctas < cap ? ctas : cap);
        return qext::launch_pdl(extract_direct_kernel<Q>, grid, kThreads, 0, st, s);
    }
}

}  // namespace

namespace qext {

static StreamArgs stream_args(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out) {
    StreamArgs s;
    s.x = x;
    s.y = y;
    s.out = out;
    s.nblocks = nblocks;
    s.wpb = p->n / 32;
    s.m = p->m;
    s.ntaps = p->ntaps;
    for (int i = 0; i < 4; ++i) {
        s.taps[i] = p->taps[i];
    }
    s.set_multipliers();
    s.status = device_status_ptr();
    return s;
}

int launch_extract(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                   qext_cuda_stream stream, uint32_t flags) {
    const StreamArgs s = stream_args(p, x, y, nblocks, out);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // q = 16, n_p = 64, 16-byte aligned sources, default launch: per-warp
    // copy pipelines (qext_extract_raw.cu)
    const uintptr_t al = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y);
    if (p->q == 16 && p->n == 1024 && al % 16 == 0 && (flags & ~uint32_t(QEXT_F_TEST_TIMEOUT)) == 0)
        return launch_extract_packed16(s, stream, flags);
    switch (p->q) {
        case 1: return launch_q<1, 0>(s, nullptr, nullptr, 0, st, flags);
        case 2: return launch_q<2, 0>(s, nullptr, nullptr, 0, st, flags);
        case 4: return launch_q<4, 0>(s, nullptr, nullptr, 0, st, flags);
        case 8: return launch_q<8, 0>(s, nullptr, nullptr, 0, st, flags);
        case 16: return launch_q<16, 0>(s, nullptr, nullptr, 0, st, flags);
        case 32: return launch_q<32, 0>(s, nullptr, nullptr, 0, st, flags);
        case 64: return launch_q<64, 0>(s, nullptr, nullptr, 0, st, flags);
        default: return QEXT_E_UNSUPPORTED;
    }
}

template <int B>
static int launch_samples_b(const qext_plan *p, const StreamArgs &s, const uint16_t *sx, const uint16_t *sy,
                            uint64_t nsamples, cudaStream_t st, uint32_t flags) {
    switch (p->q) {
        case 4: return launch_q<4, B>(s, sx, sy, nsamples, st, flags);
        case 16: return launch_q<16, B>(s, sx, sy, nsamples, st, flags);
        case 64: return launch_q<64, B>(s, sx, sy, nsamples, st, flags);
        default: return QEXT_E_UNSUPPORTED;
    }
}

int launch_extract_samples(const qext_plan *p, uint32_t b, const uint16_t *sx, const uint16_t *sy,
                           uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream,
                           uint32_t flags) {
    const StreamArgs s = stream_args(p, nullptr, nullptr, nblocks, out);
    if ((flags & QEXT_F_WARP_SPECIALIZED) && (p->q == 4 || p->q == 16))
        return launch_fused_samples(p->q, b, s, sx, sy, nsamples, stream);
    if (!(flags & QEXT_F_CTA_TILES)) {
        const int rc = launch_raw_samples(p->q, b, s, sx, sy, nsamples, stream, flags);
        if (rc != QEXT_E_UNSUPPORTED) return rc;
        if (flags & QEXT_F_TEST_TIMEOUT) return QEXT_E_INVAL;  // no per-warp kernel for this shape
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (b) {
        case 8: return launch_samples_b<8>(p, s, sx, sy, nsamples, st, flags);
        case 12: return launch_samples_b<12>(p, s, sx, sy, nsamples, st, flags);
        case 16: return launch_samples_b<16>(p, s, sx, sy, nsamples, st, flags);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace qext
