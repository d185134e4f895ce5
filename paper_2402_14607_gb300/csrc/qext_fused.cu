// Fused ingest + extraction (qext_extract_samples) for q = 4 and q = 16:
// raw b-bit ADC samples in, m-bit block outputs out, the packed streams never
// leave shared memory.
//
// Warp-specialised CTA of 256 threads.  Warps 4..7 (producers) load the raw
// samples of a tile of 128 blocks with 16-byte loads, pack them into stream
// words (sample s at stream bits [s*b, (s+1)*b)) and store them into one of
// two shared-memory tile buffers.  Warps 0..3 (consumers) compute one block
// per thread from the other buffer (Ext_IP, Definition 3.2) and assemble
// the outputs of their 32 consecutive blocks per warp.  The buffers change
// hands through mbarriers: full[b] (128 producer arrivals) and empty[b] (128
// consumer arrivals); every wait is bounded and records QEXT_E_TIMEOUT.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_block.cuh"
#include "qext_internal.h"

using namespace qxd;

namespace {

constexpr uint32_t kConsumers = 128;  // one block per consumer thread
constexpr uint32_t kProducers = 128;
constexpr uint32_t kTile = kConsumers;

struct FusedArgs {
    StreamArgs s;
    const uint16_t *sx;
    const uint16_t *sy;
    uint64_t nsamples;
    uint64_t ntiles;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int Q, int B>
__global__ void __launch_bounds__(kConsumers + kProducers) extract_fused_kernel(const FusedArgs fa) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ __align__(8) uint64_t empty[2];
    const StreamArgs &s = fa.s;
    const uint32_t tid = threadIdx.x;
    const uint32_t tw = kTile * s.wpb;  // words per tile per source
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], kProducers);
            mbar_init(&empty[i], kConsumers);
        }
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t k = 0;
    if (tid >= kConsumers) {
        // producers: pack tile k into buffer k & 1 once the consumers freed it
        const uint32_t ptid = tid - kConsumers;
        for (uint64_t tile = blockIdx.x; tile < fa.ntiles; tile += gridDim.x, ++k) {
            const uint32_t b = k & 1u, use = k >> 1;
            if (use > 0 && !mbar_wait_bounded(&empty[b], (use - 1) & 1u)) {
                record_status(s.status, QEXT_E_TIMEOUT);
                return;
            }
            uint32_t *xs = smem + 2 * b * tw, *ys = xs + tw;
            const uint64_t nb = s.nblocks - tile * kTile < kTile ? s.nblocks - tile * kTile : kTile;
            pack_tile<B>(fa.sx, fa.sy, fa.nsamples, tile * tw, uint32_t(nb * s.wpb), xs, ys, ptid, kProducers);
            mbar_arrive(&full[b]);
        }
    } else {
        // consumers: one block per thread, 32 consecutive blocks per warp
        for (uint64_t tile = blockIdx.x; tile < fa.ntiles; tile += gridDim.x, ++k) {
            const uint32_t b = k & 1u, use = k >> 1;
            if (!mbar_wait_bounded(&full[b], use & 1u)) {
                record_status(s.status, QEXT_E_TIMEOUT);
                return;
            }
            const uint32_t *xs = smem + 2 * b * tw, *ys = xs + tw;
            const uint64_t blk = tile * kTile + tid;
            uint64_t v = 0;
            if (blk < s.nblocks)
                v = block_small_q<Q>(xs + tid * s.wpb, ys + tid * s.wpb, s.wpb, s.wpb % 4 == 0, tid, s) &
                    mask_m(s.m);
            mbar_arrive(&empty[b]);
            store_warp(v, tile * kTile + (tid & ~31u), s.nblocks, s.m, s.out);
        }
    }
}

template <int Q, int B>
int launch_fused(const StreamArgs &s, const uint16_t *sx, const uint16_t *sy, uint64_t nsamples,
                 cudaStream_t st) {
    static qext::DeviceSlots grid_caps;
    const size_t smem = size_t(2) * 2 * kTile * s.wpb * 4;
    if (smem > 200 * 1024) return QEXT_E_UNSUPPORTED;
    const int dev = qext::current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int grid_cap = grid_caps.get(dev, [&] {
        int occ = 0;
        const int sms = qext::sm_count(dev);
        if (sms <= 0 ||
            cudaFuncSetAttribute(extract_fused_kernel<Q, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, extract_fused_kernel<Q, B>,
                                                          int(kConsumers + kProducers), smem) != cudaSuccess)
            return 0;
        return sms * (occ > 0 ? occ : 1);
    });
    if (grid_cap <= 0) return QEXT_E_CUDA;
    FusedArgs fa;
    fa.s = s;
    fa.sx = sx;
    fa.sy = sy;
    fa.nsamples = nsamples;
    fa.ntiles = (s.nblocks + kTile - 1) / kTile;
    const int grid = int(fa.ntiles < uint64_t(grid_cap) ? fa.ntiles : uint64_t(grid_cap));
    extract_fused_kernel<Q, B><<<grid, kConsumers + kProducers, smem, st>>>(fa);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

template <int Q>
int launch_fused_q(uint32_t b, const StreamArgs &s, const uint16_t *sx, const uint16_t *sy, uint64_t nsamples,
                   cudaStream_t st) {
    switch (b) {
        case 8: return launch_fused<Q, 8>(s, sx, sy, nsamples, st);
        case 12: return launch_fused<Q, 12>(s, sx, sy, nsamples, st);
        case 16: return launch_fused<Q, 16>(s, sx, sy, nsamples, st);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace

namespace qext {

int launch_fused_samples(uint32_t q, uint32_t b, const StreamArgs &s, const uint16_t *sx, const uint16_t *sy,
                         uint64_t nsamples, qext_cuda_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (q) {
        case 4: return launch_fused_q<4>(b, s, sx, sy, nsamples, st);
        case 16: return launch_fused_q<16>(b, s, sx, sy, nsamples, st);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace qext
