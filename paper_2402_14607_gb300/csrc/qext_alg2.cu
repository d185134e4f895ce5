// Algorithm 2 (Ext_bs^neq, Sec. 3.3): block sizes that grow with the block
// index, so that an unbounded stream can be extracted (Theorem 3.3).
//
// Parameters q_1 and Delta; n = ceil(24 / (2 delta - 1)) elements per block.
// Block l (0-based) lives in GF(2^{q_l}), q_l = q_1 + l Delta b, with that
// degree's field polynomial; it takes the next q_l n bits of each stream (the
// paper's cursor advances by q_l n / b samples) and outputs Z^(l) =
// Ext_IP^{n, q_l} (q_l bits), concatenated in block order.
//
// GPU form.  q_1 and Delta b are multiples of 16, so every q_l, every window
// start (n * sum q_j) and every output offset (sum q_j) is a multiple of 16:
// the streams and the output are arrays of 16-bit units and an element of
// block l is k_l = q_l / 16 consecutive units.  One CTA per block: per group of
// 32 elements, thread (source, u) slices unit u of the 32 elements
// (slice<16>, elements i and i + 16 in word i: element e in slot e), then
// the k_l^2 unit products S_u^x (x) S_v^y are spread over the threads, each a
// 16 x 16 sliced Gram product whose 31 diagonal parities (POPC chain) are
// XORed into the block's unreduced sum at bit 16 (u + v).  Thread 0 reduces
// the (2 q_l - 1)-bit sum mod P bit by bit and writes the block's k_l units.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "qext_block.cuh"
#include "qext_wide.cuh"
#include "qext_internal.h"
#include "qext_nvtx.h"

using namespace qxd;

struct Alg2Block {
    uint32_t q;        // q_l
    uint32_t k;        // q_l / 16
    uint32_t ntaps;
    uint32_t taps[4];  // of P_{q_l} below x^{q_l}, descending, ending with 0
    uint64_t in_unit;  // first 16-bit unit of the window: n * sum_{j<l} q_j / 16
    uint64_t out_unit; // first output unit: sum_{j<l} q_j / 16
};

struct qext_alg2_plan {
    double delta;
    uint32_t b, q1, Delta, n_p, max_blocks;
    std::vector<Alg2Block> blocks;
    Alg2Block *d_blocks = nullptr;
    int device = 0;
};

namespace {

constexpr int kAlg2Threads = 256;
constexpr uint32_t kMaxUnits = 16;  // q_l <= 256

__global__ void __launch_bounds__(kAlg2Threads)
    alg2_kernel(const Alg2Block *__restrict__ table, uint32_t n_p, const uint16_t *__restrict__ x,
                const uint16_t *__restrict__ y, uint16_t *__restrict__ out) {
    __shared__ uint32_t S[2][kMaxUnits][16];  // sliced units of the current group
    __shared__ uint32_t z[kMaxUnits + 1];     // unreduced sum, 2 q_l - 1 bits
    const Alg2Block blk = table[blockIdx.x];
    const uint32_t k = blk.k, tid = threadIdx.x;
    if (tid <= kMaxUnits) z[tid] = 0;
    const uint32_t ngroups = (n_p + 31) / 32;
    for (uint32_t g = 0; g < ngroups; ++g) {
        __syncthreads();  // the previous group's products are done with S
        if (tid < 2 * k) {
            const uint32_t src = tid / k, u = tid % k;
            const uint16_t *s = (src ? y : x) + blk.in_unit + u;
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t ea = 32 * g + uint32_t(i), eb = ea + 16;
                const uint32_t a = ea < n_p ? s[uint64_t(ea) * k] : 0u;
                const uint32_t c = eb < n_p ? s[uint64_t(eb) * k] : 0u;
                w[i] = a | (c << 16);
            }
            slice<16>(w);
#pragma unroll
            for (int i = 0; i < 16; ++i) S[src][u][i] = w[i];
        }
        __syncthreads();
        for (uint32_t p = tid; p < k * k; p += blockDim.x) {
            const uint32_t u = p / k, v = p % k;
            uint32_t X[16], Y[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                X[i] = S[0][u][i];
                Y[i] = S[1][v][i];
            }
            const uint32_t c = diagonal_chain<16>(X, Y) >> 1;  // diagonal d at bit d
            const uint32_t off = u + v;                                   // in 16-bit units
            if (off & 1u) {
                atomicXor(&z[off >> 1], c << 16);
                atomicXor(&z[(off >> 1) + 1], c >> 16);
            } else {
                atomicXor(&z[off >> 1], c);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // reduce mod P = x^q + sum taps: clear bits 2q-2 .. q from the top
        const uint32_t q = blk.q;
        for (uint32_t d = 2 * q - 2; d >= q; --d) {
            if (!((z[d >> 5] >> (d & 31)) & 1u)) continue;
            z[d >> 5] ^= 1u << (d & 31);
            for (uint32_t t = 0; t < blk.ntaps; ++t) {
                const uint32_t e = d - q + blk.taps[t];
                z[e >> 5] ^= 1u << (e & 31);
            }
        }
    }
    __syncthreads();
    if (tid < k) out[blk.out_unit + tid] = uint16_t(z[tid >> 1] >> (16 * (tid & 1u)));
}

void release(qext_alg2_plan *p) {
    if (p->d_blocks) cudaFree(p->d_blocks);
    p->d_blocks = nullptr;
}

}  // namespace

extern "C" {

int qext_alg2_plan_create(double delta, uint32_t b, uint32_t q1, uint32_t Delta, uint32_t max_blocks,
                          qext_alg2_plan **out) {
    if (!out) return QEXT_E_INVAL;
    *out = nullptr;
    if (!(delta <= 1.0) || b == 0 || b > 16 || q1 == 0 || max_blocks == 0) return QEXT_E_INVAL;
    if (!(delta > 0.5)) return QEXT_E_ENTROPY;
    const uint64_t dq = uint64_t(Delta) * b;
    if (q1 % 16 || dq % 16) return QEXT_E_UNSUPPORTED;  // the GPU works in 16-bit units
    if (q1 + dq * (max_blocks - 1) > qext::max_field_degree()) return QEXT_E_UNSUPPORTED;
    const double nn = std::ceil(24.0 / (2.0 * delta - 1.0));  // Algorithm 2's n
    if (!(nn >= 1.0) || nn > 1e6) return QEXT_E_INVAL;
    qext_alg2_plan *p = new (std::nothrow) qext_alg2_plan();
    if (!p) return QEXT_E_INVAL;
    p->delta = delta;
    p->b = b;
    p->q1 = q1;
    p->Delta = Delta;
    p->n_p = uint32_t(nn);
    p->max_blocks = max_blocks;
    p->blocks.resize(max_blocks);
    uint64_t bits = 0, obits = 0;
    for (uint32_t l = 0; l < max_blocks; ++l) {
        Alg2Block &blk = p->blocks[l];
        blk.q = uint32_t(q1 + dq * l);
        blk.k = blk.q / 16;
        for (int i = 0; i < 4; ++i) blk.taps[i] = 0;
        if (!qext::field_poly(blk.q, blk.taps, &blk.ntaps)) {
            delete p;
            return QEXT_E_PARAM;
        }
        blk.in_unit = bits / 16;
        blk.out_unit = obits / 16;
        bits += uint64_t(blk.q) * p->n_p;
        obits += blk.q;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaMalloc(&p->d_blocks, sizeof(Alg2Block) * max_blocks) != cudaSuccess ||
        cudaMemcpy(p->d_blocks, p->blocks.data(), sizeof(Alg2Block) * max_blocks, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        release(p);
        delete p;
        return QEXT_E_CUDA;
    }
    *out = p;
    return QEXT_OK;
}

int qext_alg2_plan_info(const qext_alg2_plan *p, uint32_t *n_p, uint32_t *max_blocks, double *log2_error_bound) {
    if (!p) return QEXT_E_INVAL;
    if (n_p) *n_p = p->n_p;
    if (max_blocks) *max_blocks = p->max_blocks;
    if (log2_error_bound) {
        // Theorem 3.3: sqrt(3) sum_l 2^(-1/4 - (delta/4 - 1/8) q_l n + 2 q_l), summed in the
        // log domain from the largest term
        double top = -INFINITY;
        std::vector<double> l2(p->max_blocks);
        for (uint32_t l = 0; l < p->max_blocks; ++l) {
            const uint32_t q = p->blocks[l].q;
            l2[l] = qext::log2_eps_block(q * p->n_p, p->delta * q * p->n_p, q);
            if (l2[l] > top) top = l2[l];
        }
        double s = 0.0;
        for (double v : l2) s += std::exp2(v - top);
        *log2_error_bound = top + std::log2(s);
    }
    return QEXT_OK;
}

int qext_alg2_block_info(const qext_alg2_plan *p, uint32_t l, uint32_t *q_l, uint64_t *in_bit, uint64_t *out_bit,
                         uint64_t poly_taps[4]) {
    if (!p || l > p->max_blocks) return QEXT_E_INVAL;
    // l == max_blocks: the end of the last block (window start and output offset only)
    uint64_t ib = 0, ob = 0;
    if (l < p->max_blocks) {
        ib = p->blocks[l].in_unit * 16;
        ob = p->blocks[l].out_unit * 16;
    } else {
        const Alg2Block &last = p->blocks[l - 1];
        ib = last.in_unit * 16 + uint64_t(last.q) * p->n_p;
        ob = last.out_unit * 16 + last.q;
    }
    if (q_l) *q_l = l < p->max_blocks ? p->blocks[l].q : 0;
    if (in_bit) *in_bit = ib;
    if (out_bit) *out_bit = ob;
    if (poly_taps) {
        for (int i = 0; i < 4; ++i) poly_taps[i] = 0;
        if (l < p->max_blocks) {
            int o = 0;
            for (uint32_t i = 0; i < p->blocks[l].ntaps; ++i)
                if (p->blocks[l].taps[i]) poly_taps[o++] = p->blocks[l].taps[i];
        }
    }
    return QEXT_OK;
}

int qext_alg2_extract(const qext_alg2_plan *p, const uint16_t *x, const uint16_t *y, uint32_t nblocks, uint16_t *out,
                      qext_cuda_stream stream) {
    if (!p || nblocks > p->max_blocks) return QEXT_E_INVAL;
    if (nblocks == 0) return QEXT_OK;
    const qext::NvtxRange range("qext algorithm 2 extract");
    if (!x || !y || !out || reinterpret_cast<uintptr_t>(x) % 2 || reinterpret_cast<uintptr_t>(y) % 2 ||
        reinterpret_cast<uintptr_t>(out) % 2)
        return QEXT_E_INVAL;
    alg2_kernel<<<nblocks, kAlg2Threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p->d_blocks, p->n_p, x, y, out);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

int qext_alg2_destroy(qext_alg2_plan *p) {
    if (!p) return QEXT_OK;
    release(p);
    delete p;
    return QEXT_OK;
}

}  // extern "C"
