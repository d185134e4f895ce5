// Internal declarations shared by the translation units of libqext.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <utility>

#include "../../include/qext.h"

// An immutable extraction plan (Definition 2.3's (t, m, k, eps) resolved to a
// block factorisation n = q * n_p and a field polynomial).
struct qext_plan {
    uint32_t n;          // block bits per source
    uint32_t n_p;        // field elements per block
    uint32_t q;          // field degree
    uint32_t m;          // output bits per block
    double k;            // min-entropy per block (bits)
    double eps;          // per-block error target
    double log2_eps;     // Theorem 3.1's per-block error, log2
    uint32_t ntaps;      // number of entries of taps[] used
    uint32_t taps[4];    // exponents of P(x) - x^q, descending, ending with 0
    int gpu_supported;   // every GPU entry point has a kernel for this plan
    int gpu_q80;         // q = 80: qext_extract / qext_extract_samples (b = 16) only
};

// Device-resident state of a stream (qext_stream.cu).
struct qext_stream {
    const qext_plan *plan;
    uint32_t n, m, wpb;
    uint64_t blocks_done;   // blocks output so far
    uint64_t tail_bits;     // t < n
    uint32_t pending_bits;  // p < 32
    int cur;                // which tail buffer holds the tail
    uint32_t *tail[2][2];   // [buffer][source], wpb + 1 words each (device)
    uint32_t *pending;      // 1 word (device)
    int device;
    uint32_t *stage[2];     // packed copies of raw-sample pushes on the general path (device, grown on demand)
    uint64_t stage_words;   // capacity of each, words
};

namespace qxd {
struct StreamArgs;
}

namespace qext {

constexpr int kMaxDevices = 64;

// The current device, or -1 (error, or beyond kMaxDevices).
inline int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

// A launch fact of one device (SM count, occupancy, "attribute set"),
// computed on first use and kept for the process.  0 means not yet known;
// host threads that race on a slot compute and store the same value, so
// relaxed atomics suffice.  Static instances are zero-initialised.
struct DeviceSlots {
    std::atomic<int> v[kMaxDevices];
    // the slot's value, computing it with f() (> 0 on success) on first use
    template <typename F>
    int get(int dev, F f) {
        int x = v[dev].load(std::memory_order_relaxed);
        if (x > 0) return x;
        x = f();
        if (x > 0) v[dev].store(x, std::memory_order_relaxed);
        return x;
    }
};

// Launches kernel<<<grid, block, smem, stream>>>(args...) with programmatic
// stream serialization: the next kernel of the stream may be scheduled while
// this one drains.  Only for kernels that begin with qxd::pdl_prologue(),
// which makes every such kernel wait for its predecessor's completion before
// it touches global memory.
template <typename... KArgs, typename... Args>
int launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t stream, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(block));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...) == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

// Multiprocessor count of device dev (cached), or 0 on error.
int sm_count(int dev);

// Field degrees with a GPU kernel.
bool gpu_q_supported(uint32_t q);
// The field polynomial of degree q (minimum weight, lexicographically first;
// taps descending, ending with 0), q <= max_field_degree().
bool field_poly(uint32_t q, uint32_t taps[4], uint32_t *ntaps);
// Theorem 3.1's per-block error, log2, for an n-bit block of min-entropy k.
double log2_eps_block(uint32_t n, double k, uint32_t q);
uint32_t max_field_degree();

// Ingest and extraction launchers (defined in the .cu files).
int launch_extract(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                   qext_cuda_stream stream, uint32_t flags);
int launch_extract_samples(const qext_plan *p, uint32_t b, const uint16_t *sx, const uint16_t *sy,
                           uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream,
                           uint32_t flags);
int launch_fused_samples(uint32_t q, uint32_t b, const qxd::StreamArgs &s, const uint16_t *sx, const uint16_t *sy,
                         uint64_t nsamples, qext_cuda_stream stream);
// Per-warp raw-sample kernel (q = 4, 16 with n_p = 64); QEXT_E_UNSUPPORTED for
// other shapes.
int launch_raw_samples(uint32_t q, uint32_t b, const qxd::StreamArgs &s, const uint16_t *sx, const uint16_t *sy,
                       uint64_t nsamples, qext_cuda_stream stream, uint32_t flags);
// Per-warp kernel for packed words, q = 16 with n_p = 64 (s.x, s.y 16-byte
// aligned); QEXT_E_UNSUPPORTED for other block lengths.  flags: 0 or
// QEXT_F_TEST_TIMEOUT.
int launch_extract_packed16(const qxd::StreamArgs &s, qext_cuda_stream stream, uint32_t flags);
// q = 80 blocks (any n_p), packed words.
int launch_extract_q80(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                       qext_cuda_stream stream,
                       uint32_t flags = 0);
int launch_pack(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint32_t *out, qext_cuda_stream stream);
int read_device_status(int *status);
// Device address of the status word of the current device (null if the
// lookup failed); kernels record QEXT_E_* codes there.
int *device_status_ptr();

// Batched launch from caller-provided device tables / pinned host staging
// (qext_batch.cu); used by the serving loop.
size_t batch_table_bytes();
int batch_launch_tables(const qext_batch_item *items, uint32_t nitems, void *d_table, void *h_stage,
                        qext_cuda_stream stream);

}  // namespace qext
