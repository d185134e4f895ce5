// Min-entropy monitoring of raw samples: the extractor's guarantees rest on
// the sources' min-entropy H_min(X) = -log2 max_x P(X = x) (Sec. 2; the rate
// delta of Algorithms 1 and 2), so a stream whose sources drift (the ADC's
// noise level, an offset) is watched through the histogram of its b-bit
// sample values and the plug-in estimate -log2(max count / total).
//
// Kernel: persistent CTAs; for b <= 13 each CTA counts into shared-memory
// histograms (32-bit bins, shared atomics; 2^13 / 2^b copies, up to one per
// warp) over a grid-stride walk of 16-byte chunks (8 samples), then adds the
// non-zero sums of its copies to the 64-bit global counts;
// wider samples count straight into global memory.  Bits above b are ignored,
// as in the ingest.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qext_device.cuh"
#include "qext_internal.h"
#include "qext_nvtx.h"

namespace {

constexpr int kMonThreads = 512;
constexpr uint32_t kMaxSmemBits = 13;  // 2^13 32-bit bins = 32 KB

template <bool kShared>
__global__ void __launch_bounds__(kMonThreads)
    histogram_kernel(const uint16_t *__restrict__ samples, uint64_t nsamples, uint32_t b,
                     unsigned long long *__restrict__ counts, int vec) {
    extern __shared__ uint32_t bins[];
    qxd::pdl_prologue();
    const uint32_t nbins = 1u << b, mask = nbins - 1u;
    // several copies of the bins (warp w counts into copy w % copies) spread
    // the shared atomics of the few hot values a noise distribution has
    const uint32_t copies = kShared ? min(kMonThreads / 32u, (1u << kMaxSmemBits) >> b) : 1u;
    uint32_t *const mine = bins + ((threadIdx.x >> 5) % copies) * nbins;
    if constexpr (kShared) {
        for (uint32_t v = threadIdx.x; v < copies * nbins; v += blockDim.x) bins[v] = 0;
        __syncthreads();
    }
    auto add = [&](uint32_t v) {
        if constexpr (kShared)
            atomicAdd(&mine[v & mask], 1u);
        else
            atomicAdd(&counts[v & mask], 1ull);
    };
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t done = 0;
    if (vec) {
        const uint64_t nchunks = nsamples / 8;
        const uint4 *c = reinterpret_cast<const uint4 *>(samples);
        for (uint64_t i = tid; i < nchunks; i += stride) {
            const uint4 q = __ldg(c + i);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                add(w[j] & 0xFFFFu);
                add(w[j] >> 16);
            }
        }
        done = nchunks * 8;
    }
    for (uint64_t s = done + tid; s < nsamples; s += stride) add(samples[s]);
    if constexpr (kShared) {
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < nbins; v += blockDim.x) {
            uint32_t total = 0;
            for (uint32_t c = 0; c < copies; ++c) total += bins[c * nbins + v];
            if (total) atomicAdd(&counts[v], (unsigned long long)total);
        }
    }
}

}  // namespace

extern "C" {

int qext_sample_histogram(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint64_t *counts,
                          qext_cuda_stream stream) {
    if (b < 1 || b > 16) return QEXT_E_INVAL;
    if (nsamples == 0) return QEXT_OK;
    if (!samples || !counts || reinterpret_cast<uintptr_t>(samples) % 2 || reinterpret_cast<uintptr_t>(counts) % 8)
        return QEXT_E_INVAL;
    const qext::NvtxRange range("qext min-entropy histogram");
    static qext::DeviceSlots grid_caps[2];
    const int dev = qext::current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const bool shared = b <= kMaxSmemBits;
    const size_t smem = shared ? size_t(4) << kMaxSmemBits : 0;  // all copies of the bins
    const int cap = grid_caps[shared].get(dev, [&] {
        int occ = 0;
        const int sms = qext::sm_count(dev);
        const cudaError_t e =
            shared ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, histogram_kernel<true>, kMonThreads,
                                                                   size_t(4) << kMaxSmemBits)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, histogram_kernel<false>, kMonThreads, 0);
        return sms <= 0 || e != cudaSuccess ? 0 : sms * (occ > 0 ? occ : 1);
    });
    if (cap <= 0) return QEXT_E_CUDA;
    const int vec = reinterpret_cast<uintptr_t>(samples) % 16 == 0;
    const uint64_t want = (nsamples / 8 + kMonThreads - 1) / kMonThreads;
    const int grid = int(want < 1 ? 1 : want < uint64_t(cap) ? want : uint64_t(cap));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto *c = reinterpret_cast<unsigned long long *>(counts);
    if (shared) return qext::launch_pdl(histogram_kernel<true>, grid, kMonThreads, smem, st, samples, nsamples, b, c, vec);
    return qext::launch_pdl(histogram_kernel<false>, grid, kMonThreads, 0, st, samples, nsamples, b, c, vec);
}

double qext_min_entropy_estimate(uint32_t b, const uint64_t *counts_host) {
    if (b < 1 || b > 16 || !counts_host) return -1.0;
    uint64_t total = 0, top = 0;
    for (uint64_t v = 0; v < (uint64_t(1) << b); ++v) {
        total += counts_host[v];
        if (counts_host[v] > top) top = counts_host[v];
    }
    return total ? -std::log2(double(top) / double(total)) : -1.0;
}

}  // extern "C"
