// Device primitives of the extraction kernels (sm_103a): register bit-matrix
// transposes, the sliced GF(2) Gram-diagonal accumulation of Ext_IP
// (Definition 3.2), parities by POPC, reduction mod P, output assembly, and
// the TMA bulk-copy / mbarrier helpers with bounded waits.
//
// Formulation.  For one block, Z = sum_i x_i * y_i in GF(2^q).  Reduction
// mod P is F_2-linear, so the unreduced sum of carry-less products
//     z_k = XOR_{i} XOR_{j+l=k} x_{i,j} & y_{i,l}      (k < 2q-1)
// is accumulated first and reduced once per block.  Thirty-two elements are
// "sliced": a register transpose turns q packed words (32/q elements each)
// into q words S[j] whose bit s is bit j of element s.  Then
//     acc[j+l] ^= SX[j] & SY[l]     (one LOP3 per 32 bit-products)
// and z_k = parity(acc[k]) once all elements are in.  The slot order inside
// the words is the same for x and y and the parity sums over slots, so the
// order of elements (and of whole words) inside a block never matters.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qext_internal.h"

namespace qxd {

// Everything a kernel needs to know about one stream pair.
struct StreamArgs {
    const uint32_t *x;      // packed words (or samples, for the fused ingest)
    const uint32_t *y;
    uint32_t *out;
    uint64_t nblocks;
    uint32_t wpb;           // words per block per source (n / 32)
    uint32_t m;             // output bits per block
    uint32_t ntaps;         // taps of P below x^q (0 for q = 1), descending, last 0
    uint32_t taps[4];
    uint32_t tap_mul[4];    // 2^taps[t] for t < ntaps, else 0 (run-time multipliers: shifts by taps as IMADs)
    int *status;            // device status word (qext_device_status), or null
    // Run-time multipliers of the byte-field parity assembly (Acc16K2): kept
    // out of the compiler's sight so that the steps stay IMADs on the FMA pipe
    // instead of shifts on the ALU pipe, which the products saturate.
    uint32_t byte_mul;      // 256
    uint32_t byte_pos[4];   // 2^(8i)
    uint32_t nib_mul[8];    // 2^(4i)
    __host__ __device__ void set_multipliers() {
        for (int t = 0; t < 4; ++t) tap_mul[t] = t < int(ntaps) ? 1u << (taps[t] & 31u) : 0u;
        byte_mul = 256u;
        for (int i = 0; i < 4; ++i) byte_pos[i] = 1u << (8 * i);
        for (int i = 0; i < 8; ++i) nib_mul[i] = 1u << (4 * i);
    }
};

// Programmatic dependent launch (sm_90+).  A kernel launched with the
// programmatic-serialization attribute lets the next kernel of its stream be
// scheduled as soon as every CTA has passed pdl_prologue(), and that next
// kernel's own pdl_prologue() returns only once this grid has completed and
// its memory is visible.  So nothing before the prologue may touch global
// memory; the overlap is the next launch's set-up and CTA start-up, hidden
// behind this grid's tail.  Without the attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Register bit-matrix primitives.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ constexpr uint32_t low_mask() {
    return G == 1 ? 0x55555555u : G == 2 ? 0x33333333u : G == 4 ? 0x0F0F0F0Fu : G == 8 ? 0x00FF00FFu : 0x0000FFFFu;
}

// Single LOP3 instructions (truth tables over a = 0xF0, b = 0xCC, c = 0xAA).
// (a & c) | (b & ~c): bitwise select of a where c is set, else b
__device__ __forceinline__ uint32_t lop_select(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// c ^ (a & b): one GF(2) multiply-accumulate per bit
__device__ __forceinline__ uint32_t lop_and_xor(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// a ^ b ^ c
__device__ __forceinline__ uint32_t lop_xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// One exchange stage of a recursive bit transpose between words a and b:
// in every 2G-bit lane, a keeps its low G bits and receives b's low G bits
// on top; b receives a's high G bits below its own high G bits.  (Shifts
// written as run-time multiplies measured slower in every kernel.)
template <int G>
__device__ __forceinline__ void exchange(uint32_t &a, uint32_t &b) {
    if constexpr (G == 16) {
        const uint32_t na = __byte_perm(a, b, 0x5410), nb = __byte_perm(a, b, 0x7632);
        a = na;
        b = nb;
    } else if constexpr (G == 8) {
        const uint32_t na = __byte_perm(a, b, 0x6240), nb = __byte_perm(a, b, 0x7351);
        a = na;
        b = nb;
    } else {
        constexpr uint32_t M = low_mask<G>();
        const uint32_t up = b << G, dn = a >> G;
        const uint32_t na = lop_select(a, up, M);
        const uint32_t nb = lop_select(dn, b, M);
        a = na;
        b = nb;
    }
}

// Transpose stages G = N/2 .. 1 over N words.  With N = Q <= 32 and Q-bit
// elements packed 32/Q per word, word j afterwards holds bit j of every
// element; with N = 32 it is the full 32x32 bit transpose.
template <int N, int G>
__device__ __forceinline__ void slice_stages(uint32_t (&w)[N]) {
    if constexpr (G >= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & G) == 0) exchange<G>(w[i], w[i + G]);
        slice_stages<N, G / 2>(w);
    }
}

template <int N>
__device__ __forceinline__ void slice(uint32_t (&w)[N]) {
    if constexpr (N > 1) slice_stages<N, N / 2>(w);
}

// acc[j + l] ^= X[j] & Y[l] for j < NX, l < NY (offsets into the arrays).
template <int NX, int NY, int NA>
__device__ __forceinline__ void gram_diagonals(const uint32_t *X, const uint32_t *Y, uint32_t (&acc)[NA]) {
    static_assert(NA >= NX + NY - 1, "accumulator too short");
#pragma unroll
    for (int j = 0; j < NX; ++j)
#pragma unroll
        for (int l = 0; l < NY; ++l) acc[j + l] = lop_and_xor(X[j], Y[l], acc[j + l]);
}

// Parities of K <= 32 words, one POPC each:
//     r = (r >> 1) + (popc(acc[k]) << 31)        for k = 0 .. K-1
// puts parity(acc[k]) in bit 32 - K + k (no carries: r >> 1 has bit 31
// clear and popc << 31 keeps only the popcount's low bit).
template <int K>
__device__ __forceinline__ uint32_t parity_bits32_top(const uint32_t *acc) {
    static_assert(K >= 1 && K <= 32, "1..32 words");
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) r = (r >> 1) + (uint32_t(__popc(acc[k])) << 31);
    return r;
}

// bit k of the result = parity(acc[k]) for k < K (K <= 32).
template <int K>
__device__ __forceinline__ uint32_t parity_bits32(const uint32_t *acc) {
    const uint32_t r = parity_bits32_top<K>(acc);
    if constexpr (K == 32) {
        return r;
    } else {
        return r >> (32 - K);
    }
}

template <int K>
__device__ __forceinline__ uint64_t parity_bits64(const uint32_t *acc) {
    if constexpr (K <= 32) {
        return parity_bits32<K>(acc);
    } else {
        return uint64_t(parity_bits32<32>(acc)) | (uint64_t(parity_bits32<K - 32>(acc + 32)) << 32);
    }
}

// ---------------------------------------------------------------------------
// Reduction mod P = x^q + sum_t x^taps[t] (taps end with 0).  Two folds of the
// part at and above x^q suffice when the top tap c satisfies 2c - 2 < q
// (checked at plan time).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ uint64_t reduce_mod_p(uint64_t z, const StreamArgs &s) {
    if constexpr (Q == 1) {
        return z & 1u;
    } else if constexpr (Q <= 16) {
        // 2q-1 <= 31 bits: 32-bit arithmetic, shifts by taps as IMADs
        // unused taps carry multiplier 0, so no predicates are needed
        uint32_t w = uint32_t(z);
        constexpr uint32_t LOW = (1u << Q) - 1u;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const uint32_t hi = w >> Q;
            w = lop_xor3(w & LOW, hi * s.tap_mul[0], hi * s.tap_mul[1]);
            w = lop_xor3(w, hi * s.tap_mul[2], hi * s.tap_mul[3]);
        }
        return w;
    } else {
        constexpr uint64_t LOW = Q == 64 ? ~uint64_t(0) : (uint64_t(1) << (Q % 64)) - 1;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const uint64_t hi = z >> Q;
            z &= LOW;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < int(s.ntaps)) z ^= hi << s.taps[t];
        }
        return z;
    }
}

// 127-bit (lo, hi) reduced mod a degree-64 P.
__device__ __forceinline__ uint64_t reduce_mod_p64(uint64_t lo, uint64_t hi, const StreamArgs &s) {
    uint64_t carry = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(s.ntaps)) {
            const uint32_t sh = s.taps[t];
            lo ^= hi << sh;
            if (sh) carry ^= hi >> (64 - sh);
        }
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(s.ntaps)) lo ^= carry << s.taps[t];
    return lo;
}

// ---------------------------------------------------------------------------
// Output: 32 consecutive blocks base .. base+31 (base a multiple of 32, one
// per lane, value v already truncated to m bits, 0 past nblocks) own exactly
// m output words starting at word (base/32)*m.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_warp(uint64_t v, uint64_t base, uint64_t nblocks, uint32_t m,
                                           uint32_t *__restrict__ out) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t word0 = (base >> 5) * m;
    const uint64_t total = (nblocks * m + 31) >> 5;
    if (m == 64) {
        const uint64_t w = word0 + 2 * lane;
        if (w < total) out[w] = uint32_t(v);
        if (w + 1 < total) out[w + 1] = uint32_t(v >> 32);
        return;
    }
    if ((32u % m) == 0) {
        const uint32_t k = 32u / m;  // values per word
        uint32_t word = uint32_t(v) << (m * (lane % k));
        for (uint32_t off = 1; off < k; off <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, int(off));
        const uint64_t w = word0 + lane / k;
        if (lane % k == 0 && w < total) out[w] = word;
        return;
    }
    const uint32_t reach = 31u / m + 2u;  // most lanes that can meet one word
    for (uint32_t r = 0; r * 32u < m; ++r) {
        const uint32_t w = lane + 32u * r;
        const uint32_t first = (32u * w) / m;
        uint32_t word = 0;
        for (uint32_t t = 0; t < reach; ++t) {
            const uint32_t i = first + t;
            const uint64_t vi = __shfl_sync(0xffffffffu, v, int(i < 32u ? i : 31u));
            const int sft = int(i * m) - int(32u * w);
            if (w < m && i < 32u && sft < 32) {
                if (sft >= 0)
                    word |= uint32_t(vi << sft);
                else if (sft > -64)
                    word |= uint32_t(vi >> (-sft));
            }
        }
        if (w < m && word0 + w < total) out[word0 + w] = word;
    }
}

__device__ __forceinline__ uint64_t mask_m(uint32_t m) {
    return m >= 64 ? ~uint64_t(0) : ((uint64_t(1) << m) - 1);
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (sm_90+ async proxy, used on sm_103a).
// ---------------------------------------------------------------------------
constexpr uint32_t kMaxPolls = 4u << 20;  // bounded mbarrier wait (polls)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on bar (16-byte
// aligned addresses, size a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory writes before later
// async-proxy (bulk copy) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of bar to complete; gives up after max_polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t max_polls = kMaxPolls) {
    for (uint32_t i = 0; i < max_polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Sticky: the first error recorded stays until the host reads it.
__device__ __forceinline__ void record_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace qxd
