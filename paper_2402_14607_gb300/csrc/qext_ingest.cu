// Ingest: raw b-bit ADC samples (low bits of uint16 containers) to a packed
// LSB-first bit stream (Sec. 3: X = X_1 ... X_N in ({0,1}^b)^N), and the
// device status word shared by the library's kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_device.cuh"
#include "qext_internal.h"

// Sticky device status (QEXT_OK or a negative QEXT_E_* code) written by
// kernels that give up a bounded wait; read and cleared by the host.  Kernels
// of the other translation units receive its device address (device_status_ptr).
static __device__ int qext_device_status_word = 0;

namespace {

// One thread packs one period of the pattern: S = 32/gcd(b,32) samples fill
// exactly L = b/gcd(b,32) words.  Samples past nsamples read as 0, and words
// past nwords are not written.
__global__ void __launch_bounds__(256) pack_kernel(const uint16_t *__restrict__ s, uint64_t nsamples, uint32_t b,
                                                   uint32_t S, uint32_t L, uint32_t *__restrict__ out,
                                                   uint64_t nwords, uint64_t nperiods) {
    qxd::pdl_prologue();
    const uint32_t mask = b >= 16 ? 0xFFFFu : ((1u << b) - 1u);
    for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nperiods;
         c += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t s0 = c * S, w0 = c * L;
        uint64_t buf = 0;
        uint32_t nb = 0, wi = 0;
        for (uint32_t j = 0; j < S; ++j) {
            const uint32_t v = (s0 + j < nsamples) ? (uint32_t(__ldg(s + s0 + j)) & mask) : 0u;
            buf |= uint64_t(v) << nb;
            nb += b;
            if (nb >= 32) {
                if (w0 + wi < nwords) out[w0 + wi] = uint32_t(buf);
                ++wi;
                buf >>= 32;
                nb -= 32;
            }
        }
    }
}

// b = 12: one thread per period of 8 samples (one 16-byte load) -> 3 words.
// b = 8: 16 samples (two 16-byte loads) -> 4 words (one 16-byte store).
// b = 16: 8 samples -> 4 words (a masked copy).
// Requires a 16-byte aligned sample pointer; a period that runs past
// nsamples is read sample by sample (missing samples are 0).
template <int B>
__global__ void __launch_bounds__(256) pack_kernel_vec(const uint16_t *__restrict__ s, uint64_t nsamples,
                                                       uint32_t *__restrict__ out, uint64_t nwords,
                                                       uint64_t nperiods) {
    qxd::pdl_prologue();
    constexpr uint32_t S = B == 8 ? 16 : 8;                 // samples per thread
    constexpr uint32_t L = B == 12 ? 3 : 4;                  // words per thread
    constexpr uint32_t MASK2 = B == 16 ? 0xFFFFFFFFu : B == 12 ? 0x0FFF0FFFu : 0x00FF00FFu;
    for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nperiods;
         c += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t s0 = c * S;
        uint32_t p[S / 2];  // sample pairs, low sample in the low half
        if (s0 + S <= nsamples) {
#pragma unroll
            for (uint32_t v = 0; v < S / 8; ++v) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(s + s0) + v);
                p[4 * v] = q.x;
                p[4 * v + 1] = q.y;
                p[4 * v + 2] = q.z;
                p[4 * v + 3] = q.w;
            }
        } else {
#pragma unroll
            for (uint32_t j = 0; j < S / 2; ++j) {
                const uint32_t lo = s0 + 2 * j < nsamples ? __ldg(s + s0 + 2 * j) : 0u;
                const uint32_t hi = s0 + 2 * j + 1 < nsamples ? __ldg(s + s0 + 2 * j + 1) : 0u;
                p[j] = lo | (hi << 16);
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < S / 2; ++j) p[j] &= MASK2;
        uint32_t w[L];
        if constexpr (B == 12) {
            const uint32_t a0 = p[0] & 0xFFFu, a1 = p[0] >> 16, a2 = p[1] & 0xFFFu, a3 = p[1] >> 16;
            const uint32_t a4 = p[2] & 0xFFFu, a5 = p[2] >> 16, a6 = p[3] & 0xFFFu, a7 = p[3] >> 16;
            w[0] = a0 | (a1 << 12) | (a2 << 24);
            w[1] = (a2 >> 8) | (a3 << 4) | (a4 << 16) | (a5 << 28);
            w[2] = (a5 >> 4) | (a6 << 8) | (a7 << 20);
        } else if constexpr (B == 8) {
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) w[j] = __byte_perm(p[2 * j], p[2 * j + 1], 0x6420);
        } else {
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) w[j] = p[j];
        }
        const uint64_t w0 = c * L;
        if constexpr (L == 4) {
            if (w0 + 4 <= nwords) {
                *reinterpret_cast<uint4 *>(out + w0) = make_uint4(w[0], w[1], w[2], w[3]);
                continue;
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < L; ++j)
            if (w0 + j < nwords) out[w0 + j] = w[j];
    }
}

uint32_t gcd32(uint32_t a, uint32_t b) {
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace

namespace qext {

int launch_pack(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint32_t *out, qext_cuda_stream stream) {
    const uint32_t g = gcd32(b, 32);
    const uint32_t S = 32 / g, L = b / g;
    const uint64_t nwords = (nsamples * b + 31) / 32;
    const uint64_t nperiods = (nsamples + S - 1) / S;
    const int dev = current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int sms = sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    const int grid_cap = sms * 8;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool a16 = reinterpret_cast<uintptr_t>(samples) % 16 == 0;
    const bool o16 = reinterpret_cast<uintptr_t>(out) % 16 == 0;
    auto grid_for = [&](uint64_t periods) {
        const uint64_t ctas = (periods + 255) / 256;
        return int(ctas < uint64_t(grid_cap) ? ctas : uint64_t(grid_cap));
    };
    if (a16 && b == 12) {
        const uint64_t np = (nsamples + 7) / 8;
        return launch_pdl(pack_kernel_vec<12>, grid_for(np), 256, 0, st, samples, nsamples, out, nwords, np);
    } else if (a16 && o16 && b == 8) {
        const uint64_t np = (nsamples + 15) / 16;
        return launch_pdl(pack_kernel_vec<8>, grid_for(np), 256, 0, st, samples, nsamples, out, nwords, np);
    } else if (a16 && o16 && b == 16) {
        const uint64_t np = (nsamples + 7) / 8;
        return launch_pdl(pack_kernel_vec<16>, grid_for(np), 256, 0, st, samples, nsamples, out, nwords, np);
    } else {
        return launch_pdl(pack_kernel, grid_for(nperiods), 256, 0, st, samples, nsamples, b, S, L, out, nwords,
                          nperiods);
    }
}

int sm_count(int dev) {
    static DeviceSlots sms;
    return sms.get(dev, [dev] {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess ? v : 0;
    });
}

int *device_status_ptr() {
    static std::atomic<int *> ptrs[kMaxDevices];  // zero-initialised; races store the same address
    const int dev = current_device();
    if (dev < 0) return nullptr;
    int *p = ptrs[dev].load(std::memory_order_relaxed);
    if (!p) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, qext_device_status_word) != cudaSuccess) return nullptr;
        p = static_cast<int *>(a);
        ptrs[dev].store(p, std::memory_order_relaxed);
    }
    return p;
}

int read_device_status(int *status) {
    int v = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&v, qext_device_status_word, sizeof v) != cudaSuccess) return QEXT_E_CUDA;
    if (cudaMemcpyToSymbol(qext_device_status_word, &zero, sizeof zero) != cudaSuccess) return QEXT_E_CUDA;
    *status = v;
    return QEXT_OK;
}

}  // namespace qext
