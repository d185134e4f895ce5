// Host-to-host extraction: a stream pair resident in HOST memory is cut into
// chunks of whole blocks, each copied to one of two device buffers, extracted
// (qext_extract, or qext_extract_samples for raw ADC samples) and copied
// back, with the copies in, the kernels and the copies out on three CUDA
// streams so that chunk i+1 travels while chunk i is computed.
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "qext_internal.h"
#include "qext_nvtx.h"

struct qext_pipeline {
    const qext_plan *plan;
    uint32_t b;            // 0: packed words; else bits per sample (uint16 containers)
    uint64_t chunk_blocks;
    uint64_t in_bytes;     // per source per chunk buffer
    uint64_t out_words;    // per chunk
    void *in[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [buffer][source]
    uint32_t *out[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, computed[2] = {nullptr, nullptr}, drained[2] = {nullptr, nullptr};
};

namespace {

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

void release(qext_pipeline *p) {
    for (int i = 0; i < 2; ++i) {
        cudaFree(p->in[i][0]);
        cudaFree(p->in[i][1]);
        cudaFree(p->out[i]);
        if (p->copied[i]) cudaEventDestroy(p->copied[i]);
        if (p->computed[i]) cudaEventDestroy(p->computed[i]);
        if (p->drained[i]) cudaEventDestroy(p->drained[i]);
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_comp) cudaStreamDestroy(p->s_comp);
    if (p->s_out) cudaStreamDestroy(p->s_out);
}

}  // namespace

extern "C" {

int qext_pipeline_create(const qext_plan *p, uint32_t b, uint64_t chunk_blocks, qext_pipeline **out) {
    if (!p || !out || chunk_blocks == 0 || (b != 0 && b != 8 && b != 12 && b != 16)) return QEXT_E_INVAL;
    *out = nullptr;
    if (!p->gpu_supported) return QEXT_E_UNSUPPORTED;
    if (b && p->q != 4 && p->q != 16 && p->q != 64) return QEXT_E_UNSUPPORTED;
    // chunks hold whole samples and whole output words
    uint64_t period = 32 / gcd64(p->m, 32);
    if (b) {
        const uint64_t ps = b / gcd64(p->n, b);
        period = period / gcd64(period, ps) * ps;
    }
    chunk_blocks = (chunk_blocks + period - 1) / period * period;
    qext_pipeline *pp = new (std::nothrow) qext_pipeline();
    if (!pp) return QEXT_E_INVAL;
    pp->plan = p;
    pp->b = b;
    pp->chunk_blocks = chunk_blocks;
    const uint64_t bits = chunk_blocks * p->n;
    pp->in_bytes = b ? bits / b * 2 : bits / 8;
    pp->out_words = chunk_blocks * p->m / 32;
    bool ok = cudaStreamCreateWithFlags(&pp->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pp->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pp->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i)
        ok = cudaMalloc(&pp->in[i][0], pp->in_bytes) == cudaSuccess &&
             cudaMalloc(&pp->in[i][1], pp->in_bytes) == cudaSuccess &&
             cudaMalloc(&pp->out[i], pp->out_words * 4) == cudaSuccess &&
             cudaEventCreateWithFlags(&pp->copied[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pp->computed[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pp->drained[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        release(pp);
        delete pp;
        return QEXT_E_CUDA;
    }
    *out = pp;
    return QEXT_OK;
}

int qext_pipeline_destroy(qext_pipeline *pp) {
    if (!pp) return QEXT_OK;
    release(pp);
    delete pp;
    return QEXT_OK;
}

int qext_pipeline_info(const qext_pipeline *pp, uint64_t *chunk_blocks) {
    if (!pp) return QEXT_E_INVAL;
    if (chunk_blocks) *chunk_blocks = pp->chunk_blocks;
    return QEXT_OK;
}

int qext_pipeline_run(qext_pipeline *pp, const void *x_host, const void *y_host, uint64_t count, uint64_t nblocks,
                      uint32_t *out_host) {
    if (!pp || !x_host || !y_host || !out_host) return QEXT_E_INVAL;
    const qext_plan *p = pp->plan;
    const uint64_t have_bits = pp->b ? count * pp->b : count;
    if (nblocks > have_bits / p->n) return QEXT_E_INVAL;
    if (nblocks == 0) return QEXT_OK;
    const qext::NvtxRange range("qext pipeline run");
    const uint8_t *hx = static_cast<const uint8_t *>(x_host), *hy = static_cast<const uint8_t *>(y_host);
    const uint64_t nchunks = (nblocks + pp->chunk_blocks - 1) / pp->chunk_blocks;
    for (uint64_t c = 0; c < nchunks; ++c) {
        const int k = int(c & 1u);
        const uint64_t b0 = c * pp->chunk_blocks;
        const uint64_t nb = nblocks - b0 < pp->chunk_blocks ? nblocks - b0 : pp->chunk_blocks;
        const uint64_t bit0 = b0 * p->n, nbits = nb * p->n;
        uint64_t off, bytes, nsamples = 0;
        if (pp->b) {
            const uint64_t s0 = bit0 / pp->b;  // whole samples: chunks are sample-aligned
            nsamples = (nbits + pp->b - 1) / pp->b;
            if (s0 + nsamples > count) nsamples = count - s0;
            off = s0 * 2;
            bytes = nsamples * 2;
        } else {
            off = bit0 / 8;
            bytes = nbits / 8;
        }
        // buffer k is free once chunk c-2's kernel has read it
        if (c >= 2 && cudaStreamWaitEvent(pp->s_in, pp->computed[k], 0) != cudaSuccess) return QEXT_E_CUDA;
        {
            const qext::NvtxRange copy_in("qext copy host->device");
            if (cudaMemcpyAsync(pp->in[k][0], hx + off, bytes, cudaMemcpyHostToDevice, pp->s_in) != cudaSuccess ||
                cudaMemcpyAsync(pp->in[k][1], hy + off, bytes, cudaMemcpyHostToDevice, pp->s_in) != cudaSuccess ||
                cudaEventRecord(pp->copied[k], pp->s_in) != cudaSuccess)
                return QEXT_E_CUDA;
        }
        // the output buffer k is free once chunk c-2's output was copied out
        if (cudaStreamWaitEvent(pp->s_comp, pp->copied[k], 0) != cudaSuccess) return QEXT_E_CUDA;
        if (c >= 2 && cudaStreamWaitEvent(pp->s_comp, pp->drained[k], 0) != cudaSuccess) return QEXT_E_CUDA;
        int rc;
        if (pp->b)
            rc = qext_extract_samples(p, pp->b, static_cast<const uint16_t *>(pp->in[k][0]),
                                      static_cast<const uint16_t *>(pp->in[k][1]), nsamples, nb, pp->out[k],
                                      reinterpret_cast<qext_cuda_stream>(pp->s_comp));
        else
            rc = qext_extract(p, static_cast<const uint32_t *>(pp->in[k][0]), static_cast<const uint32_t *>(pp->in[k][1]),
                              nb, pp->out[k], reinterpret_cast<qext_cuda_stream>(pp->s_comp));
        if (rc != QEXT_OK) return rc;
        if (cudaEventRecord(pp->computed[k], pp->s_comp) != cudaSuccess) return QEXT_E_CUDA;
        const uint64_t ow = (nb * p->m + 31) / 32;
        const qext::NvtxRange copy_out("qext copy device->host");
        if (cudaStreamWaitEvent(pp->s_out, pp->computed[k], 0) != cudaSuccess ||
            cudaMemcpyAsync(out_host + b0 * p->m / 32, pp->out[k], ow * 4, cudaMemcpyDeviceToHost, pp->s_out) !=
                cudaSuccess ||
            cudaEventRecord(pp->drained[k], pp->s_out) != cudaSuccess)
            return QEXT_E_CUDA;
    }
    return cudaStreamSynchronize(pp->s_out) == cudaSuccess && cudaStreamSynchronize(pp->s_comp) == cudaSuccess
               ? QEXT_OK
               : QEXT_E_CUDA;
}

}  // extern "C"
