// Stream-state manager: Algorithm 1 over a stream delivered in chunks of any
// bit length.  Blocks are consumed strictly in time order and x/y blocks pair
// by index (the loop of Algorithm 1 with its cursor advanced by one block per
// step); the output is the concatenation Z^(1) Z^(2) ... of m-bit values.
//
// Device-resident state per stream: the unconsumed tail of each source (fewer
// than n bits, in one of two ping-pong buffers, bits past the tail length are
// zero) and the pending output word (fewer than 32 bits not yet emitted).  The
// host keeps the counters (blocks done, tail bits, pending bits), which follow
// from the chunk lengths alone, so a push never waits for the device.
//
// A push of L bits forms the virtual stream V = tail ++ chunk (t + L bits),
// extracts its floor(V/n) whole blocks and keeps the rest as the new tail.
// Fast path (no tail, no pending bits): the chunk is extracted in place by the
// tiled kernel.  General path: a kernel reads block words from V at any bit
// offset and ORs each m-bit value into the zeroed output at bit offset
// pending + j*m, after the pending bits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>

#include "qext_block.cuh"
#include "qext_wide.cuh"
#include "qext_internal.h"
#include "qext_nvtx.h"

using namespace qxd;

namespace {

constexpr int kStreamThreads = 32;
constexpr uint32_t kMaxGeneralWpb = 256;  // general path: blocks up to 8192 bits

// 32 bits of a word array at bit offset `bit` (words past nwords read as 0)
__device__ __forceinline__ uint32_t bits32(const uint32_t *w, uint64_t nwords, uint64_t bit) {
    const uint64_t i = bit >> 5;
    const uint32_t sh = uint32_t(bit & 31u);
    const uint32_t lo = i < nwords ? w[i] : 0u;
    const uint32_t hi = i + 1 < nwords ? w[i + 1] : 0u;
    return sh ? __funnelshift_r(lo, hi, sh) : lo;
}

// 32 bits of V = tail (t bits, zero above) ++ chunk, at virtual bit v
__device__ __forceinline__ uint32_t vbits32(const uint32_t *tail, uint64_t t, const uint32_t *chunk,
                                            uint64_t chunk_words, uint64_t v) {
    if (v >= t) return bits32(chunk, chunk_words, v - t);
    const uint32_t from_tail = bits32(tail, (t + 31) / 32, v);  // zero above t
    const uint64_t have = t - v;                                 // tail bits in this word
    if (have >= 32) return from_tail;
    return from_tail | (bits32(chunk, chunk_words, 0) << have);
}

struct GeneralArgs {
    StreamArgs s;           // s.x, s.y: chunk words; s.out: output; s.nblocks: blocks in V
    const uint32_t *tx, *ty;
    uint64_t t;             // tail bits
    uint64_t chunk_words;
    uint32_t out_bit0;      // pending bits before the first new value
};

template <int Q>
__global__ void __launch_bounds__(kStreamThreads) stream_general_kernel(const GeneralArgs g) {
    extern __shared__ uint32_t sm[];
    const StreamArgs &s = g.s;
    uint32_t *xs = sm + threadIdx.x * 2 * s.wpb, *ys = xs + s.wpb;
    for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < s.nblocks;
         j += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t v0 = j * uint64_t(s.wpb) * 32;
        for (uint32_t w = 0; w < s.wpb; ++w) {
            xs[w] = vbits32(g.tx, g.t, s.x, g.chunk_words, v0 + 32ull * w);
            ys[w] = vbits32(g.ty, g.t, s.y, g.chunk_words, v0 + 32ull * w);
        }
        uint64_t v;
        if constexpr (Q == 64) {
            uint64_t A = 0, B = 0, C = 0;
            half_products64(xs, ys, s.wpb, 0, 0, 0, 1, A, B, C, s);
            v = combine_q64(A, B, C, s);
        } else {
            v = block_small_q<Q>(xs, ys, s.wpb, 0, 0, s);
        }
        v &= mask_m(s.m);
        // OR the value into the zeroed output at bit g.out_bit0 + j*m
        const uint64_t ob = g.out_bit0 + j * s.m;
        const uint32_t sh = uint32_t(ob & 31u);
        const uint64_t wi = ob >> 5;
        atomicOr(s.out + wi, uint32_t(v << sh));
        if (sh + s.m > 32) atomicOr(s.out + wi + 1, uint32_t((v >> (32 - sh)) & 0xFFFFFFFFu));
        if (sh + s.m > 64) atomicOr(s.out + wi + 2, uint32_t(v >> (64 - sh)));
    }
}

// New tail: virtual bits [from, from + nbits) into dst (ceil(nbits/32) words,
// bits past nbits zeroed) -- both sources.
__global__ void tail_copy_kernel(const uint32_t *tx, const uint32_t *ty, uint64_t t, const uint32_t *cx,
                                 const uint32_t *cy, uint64_t chunk_words, uint64_t from, uint64_t nbits,
                                 uint32_t *dx, uint32_t *dy, uint32_t dst_words) {
    for (uint32_t i = threadIdx.x; i < dst_words; i += blockDim.x) {
        uint32_t a = 0, b = 0;
        const uint64_t bit = 32ull * i;
        if (bit < nbits) {
            a = vbits32(tx, t, cx, chunk_words, from + bit);
            b = vbits32(ty, t, cy, chunk_words, from + bit);
            const uint64_t keep = nbits - bit;
            if (keep < 32) {
                const uint32_t mk = (1u << keep) - 1u;
                a &= mk;
                b &= mk;
            }
        }
        dx[i] = a;
        dy[i] = b;
    }
}

// 32 stream bits starting at bit `bit` of the b-bit samples smp[0 .. ns)
// (sample j at bits [j*b, (j+1)*b), LSB first; bits past ns*b read as 0)
__device__ __forceinline__ uint32_t sample_bits32(const uint16_t *smp, uint64_t ns, uint32_t b, uint64_t bit) {
    const uint32_t mask = b >= 16 ? 0xFFFFu : (1u << b) - 1u;
    uint32_t w = 0;
    for (uint64_t j = bit / b; j < ns && j * b < bit + 32; ++j) {
        const uint32_t v = smp[j] & mask;
        const int64_t sh = int64_t(j * b) - int64_t(bit);  // position of the sample's bit 0 in w
        w |= sh >= 0 ? v << sh : v >> -sh;
    }
    return w;
}

// New tail from a raw-sample push with no carried tail: stream bits
// [from, from + nbits) of the samples into dx, dy (dst_words words, zero
// above nbits).
__global__ void tail_from_samples_kernel(const uint16_t *sx, const uint16_t *sy, uint64_t ns, uint32_t b,
                                         uint64_t from, uint64_t nbits, uint32_t *dx, uint32_t *dy,
                                         uint32_t dst_words) {
    for (uint32_t i = threadIdx.x; i < dst_words; i += blockDim.x) {
        uint32_t a = 0, c = 0;
        const uint64_t bit = 32ull * i;
        if (bit < nbits) {
            a = sample_bits32(sx, ns, b, from + bit);
            c = sample_bits32(sy, ns, b, from + bit);
            const uint64_t keep = nbits - bit;
            if (keep < 32) {
                const uint32_t mk = (1u << keep) - 1u;
                a &= mk;
                c &= mk;
            }
        }
        dx[i] = a;
        dy[i] = c;
    }
}

// pending <- out[word] & low `bits` bits (bits in 1..31)
__global__ void save_pending_kernel(const uint32_t *out, uint64_t word, uint32_t bits, uint32_t *pending) {
    if (threadIdx.x == 0) *pending = out[word] & ((1u << bits) - 1u);
}

template <int Q>
int launch_general(const GeneralArgs &g, cudaStream_t st) {
    const size_t smem = size_t(kStreamThreads) * 2 * g.s.wpb * 4;
    static qext::DeviceSlots attr_set;
    const int dev = qext::current_device();
    if (dev < 0 || attr_set.get(dev, [] {
            return cudaFuncSetAttribute(stream_general_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kStreamThreads * 2 * kMaxGeneralWpb * 4) == cudaSuccess ? 1 : 0;
        }) <= 0)
        return QEXT_E_CUDA;
    uint64_t ctas = (g.s.nblocks + kStreamThreads - 1) / kStreamThreads;
    if (ctas > 4096) ctas = 4096;
    stream_general_kernel<Q><<<int(ctas), kStreamThreads, smem, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

int launch_general_q(uint32_t q, const GeneralArgs &g, cudaStream_t st) {
    switch (q) {
        case 1: return launch_general<1>(g, st);
        case 2: return launch_general<2>(g, st);
        case 4: return launch_general<4>(g, st);
        case 8: return launch_general<8>(g, st);
        case 16: return launch_general<16>(g, st);
        case 32: return launch_general<32>(g, st);
        case 64: return launch_general<64>(g, st);
        default: return QEXT_E_UNSUPPORTED;
    }
}

bool aligned4(const void *p) { return reinterpret_cast<uintptr_t>(p) % 4 == 0; }

constexpr uint32_t kSaveMagic = 0x51455853u;  // "SXEQ"
constexpr uint32_t kSaveVersion = 1;

struct SaveHeader {
    uint32_t magic, version;
    uint32_t n, m, q, n_p;
    uint64_t blocks_done, tail_bits;
    uint32_t pending_bits, pending_word;
};

}  // namespace

extern "C" {

int qext_stream_create(const qext_plan *p, qext_stream **out) {
    if (!p || !out) return QEXT_E_INVAL;
    *out = nullptr;
    if (!p->gpu_supported) return QEXT_E_UNSUPPORTED;
    qext_stream *s = new (std::nothrow) qext_stream();
    if (!s) return QEXT_E_INVAL;
    s->plan = p;
    s->n = p->n;
    s->m = p->m;
    s->wpb = p->n / 32;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return QEXT_E_CUDA;
    }
    const size_t tail_words = s->wpb + 1;
    uint32_t *mem = nullptr;
    if (cudaMalloc(&mem, (4 * tail_words + 1) * sizeof(uint32_t)) != cudaSuccess) {
        delete s;
        return QEXT_E_CUDA;
    }
    if (cudaMemset(mem, 0, (4 * tail_words + 1) * sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(mem);
        delete s;
        return QEXT_E_CUDA;
    }
    for (int b = 0; b < 2; ++b)
        for (int src = 0; src < 2; ++src) s->tail[b][src] = mem + (2 * b + src) * tail_words;
    s->pending = mem + 4 * tail_words;
    *out = s;
    return QEXT_OK;
}

int qext_stream_destroy(qext_stream *s) {
    if (!s) return QEXT_OK;
    cudaFree(s->tail[0][0]);
    cudaFree(s->stage[0]);
    delete s;
    return QEXT_OK;
}

int qext_stream_info(const qext_stream *s, uint64_t *blocks_done, uint64_t *tail_bits, uint32_t *pending_bits) {
    if (!s) return QEXT_E_INVAL;
    if (blocks_done) *blocks_done = s->blocks_done;
    if (tail_bits) *tail_bits = s->tail_bits;
    if (pending_bits) *pending_bits = s->pending_bits;
    return QEXT_OK;
}

int qext_stream_push(qext_stream *s, const uint32_t *x, const uint32_t *y, uint64_t nbits, uint32_t *out,
                     uint64_t out_capacity_words, uint64_t *out_words, qext_cuda_stream stream) {
    if (!s || !out_words) return QEXT_E_INVAL;
    *out_words = 0;
    if (nbits == 0) return QEXT_OK;
    if (!x || !y || !aligned4(x) || !aligned4(y)) return QEXT_E_INVAL;
    const qext::NvtxRange range("qext stream push");
    const uint64_t t = s->tail_bits, p = s->pending_bits, n = s->n, m = s->m;
    if (nbits > UINT64_MAX - t) return QEXT_E_INVAL;
    const uint64_t V = t + nbits;
    const uint64_t B = V / n;
    const uint64_t total_out = p + B * m;
    const uint64_t need = (total_out + 31) / 32;
    if (need && (!out || !aligned4(out))) return QEXT_E_INVAL;
    if (out_capacity_words < need) return QEXT_E_NOSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t chunk_words = (nbits + 31) / 32;
    int rc = QEXT_OK;
    if (B > 0) {
        if (t == 0 && p == 0) {
            rc = qext::launch_extract(s->plan, x, y, B, out, stream, 0);  // in place, tiled kernel
        } else {
            if (s->wpb > kMaxGeneralWpb) return QEXT_E_UNSUPPORTED;
            if (cudaMemsetAsync(out, 0, need * sizeof(uint32_t), st) != cudaSuccess) return QEXT_E_CUDA;
            if (p && cudaMemcpyAsync(out, s->pending, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return QEXT_E_CUDA;
            GeneralArgs g;
            std::memset(&g, 0, sizeof g);
            g.s.x = x;
            g.s.y = y;
            g.s.out = out;
            g.s.nblocks = B;
            g.s.wpb = s->wpb;
            g.s.m = s->m;
            g.s.ntaps = s->plan->ntaps;
            for (int i = 0; i < 4; ++i) {
                g.s.taps[i] = s->plan->taps[i];
            }
            g.s.set_multipliers();
            g.s.status = qext::device_status_ptr();
            g.tx = s->tail[s->cur][0];
            g.ty = s->tail[s->cur][1];
            g.t = t;
            g.chunk_words = chunk_words;
            g.out_bit0 = uint32_t(p);
            rc = launch_general_q(s->plan->q, g, st);
        }
        if (rc != QEXT_OK) return rc;
    }
    // new pending word: the partial last output word (no output: keep it)
    const uint32_t r = uint32_t(total_out & 31u);
    if (B > 0 && r) {
        save_pending_kernel<<<1, 32, 0, st>>>(out, total_out >> 5, r, s->pending);
        if (cudaGetLastError() != cudaSuccess) return QEXT_E_CUDA;
    }
    // new tail: virtual bits [B*n, V) into the other buffer
    const uint64_t nt = V - B * n;
    const int nxt = s->cur ^ 1;
    const uint32_t dst_words = s->wpb + 1;
    if (nt > 0 || t > 0) {
        tail_copy_kernel<<<1, 256, 0, st>>>(s->tail[s->cur][0], s->tail[s->cur][1], t, x, y, chunk_words, B * n, nt,
                                            s->tail[nxt][0], s->tail[nxt][1], dst_words);
        if (cudaGetLastError() != cudaSuccess) return QEXT_E_CUDA;
        s->cur = nxt;
    }
    s->tail_bits = nt;
    s->pending_bits = r;
    s->blocks_done += B;
    *out_words = total_out >> 5;
    return QEXT_OK;
}

int qext_stream_push_samples(qext_stream *s, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                             uint64_t nsamples, uint32_t *out, uint64_t out_capacity_words, uint64_t *out_words,
                             qext_cuda_stream stream) {
    if (!s || !out_words) return QEXT_E_INVAL;
    *out_words = 0;
    if (b < 1 || b > 16) return QEXT_E_INVAL;
    if (nsamples == 0) return QEXT_OK;
    if (!x_samples || !y_samples || reinterpret_cast<uintptr_t>(x_samples) % 2 ||
        reinterpret_cast<uintptr_t>(y_samples) % 2)
        return QEXT_E_INVAL;
    if (nsamples > (UINT64_MAX - s->tail_bits) / 16) return QEXT_E_INVAL;
    const qext::NvtxRange range("qext stream push (raw samples)");
    const uint64_t t = s->tail_bits, p = s->pending_bits, n = s->n, m = s->m;
    const uint64_t nbits = nsamples * b;
    const uint64_t B = (t + nbits) / n;
    const uint64_t total_out = p + B * m;
    const uint64_t need = (total_out + 31) / 32;
    if (need && (!out || !aligned4(out))) return QEXT_E_INVAL;
    if (out_capacity_words < need) return QEXT_E_NOSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t q = s->plan->q;
    const bool fused = t == 0 && p == 0 && B > 0 && (b == 8 || b == 12 || b == 16) && (q == 4 || q == 16 || q == 64) &&
                       reinterpret_cast<uintptr_t>(x_samples) % 16 == 0 && reinterpret_cast<uintptr_t>(y_samples) % 16 == 0;
    if (!fused) {
        // general path: pack into the stream's staging buffers, then push the bits
        const uint64_t words = (nbits + 31) / 32;
        if (words > s->stage_words) {
            uint32_t *mem = nullptr;
            if (cudaStreamSynchronize(st) != cudaSuccess) return QEXT_E_CUDA;  // old buffers may be in use
            if (cudaMalloc(&mem, 2 * words * sizeof(uint32_t)) != cudaSuccess) return QEXT_E_CUDA;
            cudaFree(s->stage[0]);
            s->stage[0] = mem;
            s->stage[1] = mem + words;
            s->stage_words = words;
        }
        int rc = qext::launch_pack(b, x_samples, nsamples, s->stage[0], stream);
        if (rc == QEXT_OK) rc = qext::launch_pack(b, y_samples, nsamples, s->stage[1], stream);
        if (rc != QEXT_OK) return rc;
        return qext_stream_push(s, s->stage[0], s->stage[1], nbits, out, out_capacity_words, out_words, stream);
    }
    // fused path: no carried state, whole blocks straight from the samples
    int rc = qext::launch_extract_samples(s->plan, b, x_samples, y_samples, nsamples, B, out, stream, 0);
    if (rc != QEXT_OK) return rc;
    const uint32_t r = uint32_t(total_out & 31u);
    if (r) {
        save_pending_kernel<<<1, 32, 0, st>>>(out, total_out >> 5, r, s->pending);
        if (cudaGetLastError() != cudaSuccess) return QEXT_E_CUDA;
    }
    const uint64_t nt = nbits - B * n;
    if (nt > 0) {
        const int nxt = s->cur ^ 1;
        tail_from_samples_kernel<<<1, 256, 0, st>>>(x_samples, y_samples, nsamples, b, B * n, nt, s->tail[nxt][0],
                                                    s->tail[nxt][1], s->wpb + 1);
        if (cudaGetLastError() != cudaSuccess) return QEXT_E_CUDA;
        s->cur = nxt;
    }
    s->tail_bits = nt;
    s->pending_bits = r;
    s->blocks_done += B;
    *out_words = total_out >> 5;
    return QEXT_OK;
}

int qext_stream_flush(qext_stream *s, uint32_t *out, uint64_t out_capacity_words, uint32_t *out_bits,
                      qext_cuda_stream stream) {
    if (!s || !out_bits) return QEXT_E_INVAL;
    *out_bits = 0;
    if (s->pending_bits) {
        if (!out || !aligned4(out)) return QEXT_E_INVAL;
        if (out_capacity_words < 1) return QEXT_E_NOSPACE;
        if (cudaMemcpyAsync(out, s->pending, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
            return QEXT_E_CUDA;
        *out_bits = s->pending_bits;
    }
    // Algorithm 1 outputs whole blocks only: an incomplete block is dropped
    s->pending_bits = 0;
    s->tail_bits = 0;
    return QEXT_OK;
}

size_t qext_stream_state_size(const qext_stream *s) {
    if (!s) return 0;
    return sizeof(SaveHeader) + 2 * size_t(s->wpb + 1) * sizeof(uint32_t);
}

int qext_stream_save(const qext_stream *s, void *host_buf, size_t capacity, size_t *size, qext_cuda_stream stream) {
    if (!s || !host_buf || !size) return QEXT_E_INVAL;
    const size_t need = qext_stream_state_size(s);
    *size = need;
    if (capacity < need) return QEXT_E_NOSPACE;
    SaveHeader h;
    std::memset(&h, 0, sizeof h);
    h.magic = kSaveMagic;
    h.version = kSaveVersion;
    h.n = s->n;
    h.m = s->m;
    h.q = s->plan->q;
    h.n_p = s->plan->n_p;
    h.blocks_done = s->blocks_done;
    h.tail_bits = s->tail_bits;
    h.pending_bits = s->pending_bits;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *dst = static_cast<uint8_t *>(host_buf);
    const size_t tw = size_t(s->wpb + 1) * sizeof(uint32_t);
    if (cudaMemcpyAsync(&h.pending_word, s->pending, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(dst + sizeof h, s->tail[s->cur][0], tw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(dst + sizeof h + tw, s->tail[s->cur][1], tw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QEXT_E_CUDA;
    if (!s->pending_bits) h.pending_word = 0;
    std::memcpy(dst, &h, sizeof h);
    return QEXT_OK;
}

int qext_stream_restore(const qext_plan *p, const void *host_buf, size_t size, qext_stream **out,
                        qext_cuda_stream stream) {
    if (!p || !host_buf || !out) return QEXT_E_INVAL;
    *out = nullptr;
    if (size < sizeof(SaveHeader)) return QEXT_E_INVAL;
    SaveHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (h.magic != kSaveMagic || h.version != kSaveVersion) return QEXT_E_INVAL;
    if (h.n != p->n || h.m != p->m || h.q != p->q || h.n_p != p->n_p) return QEXT_E_STATE;
    if (h.tail_bits >= h.n || h.pending_bits >= 32) return QEXT_E_INVAL;
    qext_stream *s = nullptr;
    int rc = qext_stream_create(p, &s);
    if (rc != QEXT_OK) return rc;
    if (size < qext_stream_state_size(s)) {
        qext_stream_destroy(s);
        return QEXT_E_INVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint8_t *src = static_cast<const uint8_t *>(host_buf);
    const size_t tw = size_t(s->wpb + 1) * sizeof(uint32_t);
    if (cudaMemcpyAsync(s->pending, &h.pending_word, sizeof(uint32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->tail[0][0], src + sizeof h, tw, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->tail[0][1], src + sizeof h + tw, tw, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        qext_stream_destroy(s);
        return QEXT_E_CUDA;
    }
    s->cur = 0;
    s->blocks_done = h.blocks_done;
    s->tail_bits = h.tail_bits;
    s->pending_bits = h.pending_bits;
    *out = s;
    return QEXT_OK;
}

}  // extern "C"
