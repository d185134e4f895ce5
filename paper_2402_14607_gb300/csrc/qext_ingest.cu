// Ingest: raw b-bit ADC samples (low bits of uint16 containers) to a packed
// LSB-first bit stream (Sec. 3: X = X_1 ... X_N in ({0,1}^b)^N), and the
// device status word shared by the library's kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_internal.h"

// Sticky device status (QEXT_OK or a negative QEXT_E_* code) written by
// kernels that give up a bounded wait; read and cleared by the host.
__device__ int qext_device_status_word = 0;

namespace {

// One thread packs one period of the pattern: S = 32/gcd(b,32) samples fill
// exactly L = b/gcd(b,32) words.  Samples past nsamples read as 0, and words
// past nwords are not written.
__global__ void __launch_bounds__(256) pack_kernel(const uint16_t *__restrict__ s, uint64_t nsamples, uint32_t b,
                                                   uint32_t S, uint32_t L, uint32_t *__restrict__ out,
                                                   uint64_t nwords, uint64_t nperiods) {
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
    static int grid_cap = 0;
    if (!grid_cap) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return QEXT_E_CUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QEXT_E_CUDA;
        grid_cap = sms * 8;
    }
    const uint64_t ctas = (nperiods + 255) / 256;
    const int grid = int(ctas < uint64_t(grid_cap) ? ctas : uint64_t(grid_cap));
    pack_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(samples, nsamples, b, S, L, out, nwords,
                                                                          nperiods);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
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
