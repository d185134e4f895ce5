// Per-block extraction kernels for Ext_IP^{n_p,q} (Definition 3.2) inside
// Algorithm 1's block loop, for GB300 (sm_103a).
//
// Formulation.  For one block, Z = sum_i x_i * y_i in GF(2^q).  Reduction
// mod P is F_2-linear, so the unreduced sum of carry-less products
//     z_k = XOR_{i} XOR_{j+l=k} x_{i,j} & y_{i,l}      (k < 2q-1)
// is accumulated first and reduced once per block.  Thirty-two elements are
// "sliced": a register transpose turns q packed words (32/q elements each)
// into q words S[j] whose bit s is bit j of element s.  Then
//     acc[j+l] ^= SX[j] & SY[l]     (one LOP3 per 32 bit-products)
// and z_k = parity(acc[k]) after all elements are in.  The slot order inside
// the words is the same for x and y, and the parity sums over slots, so the
// element order inside a group never matters.
//
// Everything is exact GF(2): AND, XOR, shifts and byte permutes only.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_internal.h"

namespace {

// 2^G and 2^(32-G) for G = 1, 2, 4 (index log2 G).  Passed at run time so the
// shifts of the transpose stages issue as IMAD / IMAD.HI on the FMA pipe
// instead of SHF on the ALU pipe, which the AND/XOR work already saturates.
struct ShiftMuls {
    uint32_t lo[3];  // 2^G
    uint32_t hi[3];  // 2^(32-G): umulhi(a, 2^(32-G)) = a >> G
};

struct ExtractArgs {
    const uint32_t *x;
    const uint32_t *y;
    uint32_t *out;
    uint64_t nblocks;
    uint32_t wpb;      // words per block per source (n / 32)
    uint32_t m;        // output bits per block
    uint32_t ntaps;    // taps of P below x^q (0 for q = 1)
    uint32_t taps[4];  // descending, last is 0 (the constant term)
    int vec16;         // x, y 16-byte aligned and wpb % 4 == 0
    int vec8;          // x, y 8-byte aligned and wpb % 2 == 0
    ShiftMuls mu;
};

// ---------------------------------------------------------------------------
// Register bit-matrix primitives.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ constexpr uint32_t low_mask() {
    return G == 1 ? 0x55555555u : G == 2 ? 0x33333333u : G == 4 ? 0x0F0F0F0Fu : G == 8 ? 0x00FF00FFu : 0x0000FFFFu;
}

// One exchange stage of a recursive bit transpose between words a and b:
// in every 2G-bit lane, a keeps its low G bits and receives b's low G bits
// on top; b receives a's high G bits below its own high G bits.
template <int G>
__device__ __forceinline__ constexpr int log2_of() {
    return G == 1 ? 0 : G == 2 ? 1 : 2;
}

template <int G>
__device__ __forceinline__ void exchange(uint32_t &a, uint32_t &b, const ShiftMuls &mu) {
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
        const uint32_t up = b * mu.lo[log2_of<G>()];             // b << G   (IMAD)
        const uint32_t dn = __umulhi(a, mu.hi[log2_of<G>()]);    // a >> G   (IMAD.HI)
        const uint32_t na = (a & M) | (up & ~M);
        const uint32_t nb = (dn & M) | (b & ~M);
        a = na;
        b = nb;
    }
}

// Transpose stages G = Q/2 .. 1 over Q words: afterwards w[j] holds bit j of
// every element (Q-bit elements packed 32/Q per word).
template <int Q, int G>
__device__ __forceinline__ void slice_stages(uint32_t (&w)[Q], const ShiftMuls &mu) {
    if constexpr (G >= 1) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((i & G) == 0) exchange<G>(w[i], w[i + G], mu);
        slice_stages<Q, G / 2>(w, mu);
    }
}

template <int Q>
__device__ __forceinline__ void slice(uint32_t (&w)[Q], const ShiftMuls &mu) {
    slice_stages<Q, Q / 2>(w, mu);
}

// acc[j + l] ^= X[j] & Y[l] for all j, l < Q (schoolbook Gram diagonals).
template <int Q>
__device__ __forceinline__ void gram_diagonals(const uint32_t (&X)[Q], const uint32_t (&Y)[Q], uint32_t (&acc)[2 * Q - 1]) {
#pragma unroll
    for (int j = 0; j < Q; ++j)
#pragma unroll
        for (int l = 0; l < Q; ++l) acc[j + l] ^= X[j] & Y[l];
}

// Parities of 32 words at once: after folding stages G = 16 .. 1 (each an
// exchange followed by XOR of the pair), bit p of the result is the parity
// of a[p].
template <int G>
__device__ __forceinline__ void parity_fold(uint32_t (&a)[32], const ShiftMuls &mu) {
    if constexpr (G >= 1) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            uint32_t u = a[i], v = a[i + G];
            exchange<G>(u, v, mu);
            a[i] = u ^ v;
        }
        parity_fold<G / 2>(a, mu);
    }
}

template <int K>
__device__ __forceinline__ uint32_t parity_bits32(const uint32_t *acc, const ShiftMuls &mu) {
    uint32_t a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = i < K ? acc[i] : 0u;
    parity_fold<16>(a, mu);
    return a[0];
}

// ---------------------------------------------------------------------------
// Loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ldg4(const uint32_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// Q consecutive words of a block starting at word g0 (zero past wpb).
template <int Q>
__device__ __forceinline__ void load_group(const uint32_t *blk, uint32_t g0, uint32_t wpb, int vec16, uint32_t (&w)[Q]) {
    if (g0 + Q <= wpb) {
        if constexpr (Q % 4 == 0) {
            if (vec16) {
#pragma unroll
                for (int i = 0; i < Q; i += 4) {
                    const uint4 v = ldg4(blk + g0 + i);
                    w[i] = v.x;
                    w[i + 1] = v.y;
                    w[i + 2] = v.z;
                    w[i + 3] = v.w;
                }
                return;
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) w[i] = __ldg(blk + g0 + i);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) w[i] = (g0 + i < wpb) ? __ldg(blk + g0 + i) : 0u;
    }
}

// ---------------------------------------------------------------------------
// Reduction mod P = x^q + sum_t x^taps[t] (taps include 0).  Two folds of the
// part at and above x^q suffice when the top tap c satisfies 2c - 2 < q
// (checked at plan time).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ uint64_t reduce_small(uint64_t z, const ExtractArgs &a) {
    if constexpr (Q == 1) {
        return z & 1u;
    } else {
        constexpr uint64_t LOW = (uint64_t(1) << Q) - 1;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const uint64_t hi = z >> Q;
            z &= LOW;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < int(a.ntaps)) z ^= hi << a.taps[t];
        }
        return z;
    }
}

// 127-bit (lo, hi) reduced mod a degree-64 P.
__device__ __forceinline__ uint64_t reduce_64(uint64_t lo, uint64_t hi, const ExtractArgs &a) {
    uint64_t carry = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(a.ntaps)) {
            const uint32_t s = a.taps[t];
            lo ^= hi << s;
            if (s) carry ^= hi >> (64 - s);
        }
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(a.ntaps)) lo ^= carry << a.taps[t];
    return lo;
}

// ---------------------------------------------------------------------------
// One block: reduced Z (q bits; q <= 64).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ uint64_t block_value(const uint32_t *xb, const uint32_t *yb, const ExtractArgs &a) {
    uint32_t acc[2 * Q - 1];
#pragma unroll
    for (int i = 0; i < 2 * Q - 1; ++i) acc[i] = 0;
    for (uint32_t g0 = 0; g0 < a.wpb; g0 += Q) {
        uint32_t X[Q], Y[Q];
        load_group<Q>(xb, g0, a.wpb, a.vec16, X);
        load_group<Q>(yb, g0, a.wpb, a.vec16, Y);
        slice<Q>(X, a.mu);
        slice<Q>(Y, a.mu);
        gram_diagonals<Q>(X, Y, acc);
    }
    uint64_t z;
    if constexpr (2 * Q - 1 <= 32) {
        z = parity_bits32<2 * Q - 1>(acc, a.mu);
    } else {
        z = uint64_t(parity_bits32<32>(acc, a.mu)) | (uint64_t(parity_bits32<2 * Q - 1 - 32>(acc + 32, a.mu)) << 32);
    }
    return reduce_small<Q>(z, a);
}

// q = 64: elements are word pairs (low word = bits 0..31, high = 32..63).
// One Karatsuba level over the halves:  z = A + x^64 B + x^32 (C - A - B),
// A = sum lo*lo, B = sum hi*hi, C = sum (lo^hi)*(hi^lo); each a 32x32
// sliced Gram product over groups of 32 elements.  Transposition is linear,
// so C's operands are sliced from the XOR of the raw words.
template <int PART>
__device__ __forceinline__ void load_half64(const uint32_t *blk, uint32_t g0, uint32_t wpb, int vec8,
                                            uint32_t (&w)[32]) {
    // a group of 32 elements is the 64 words starting at g0; wpb is even
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const uint32_t i = g0 + 2 * e;
        uint32_t lo = 0, hi = 0;
        if (i < wpb) {
            if (vec8) {
                const uint2 v = __ldg(reinterpret_cast<const uint2 *>(blk + i));
                lo = v.x;
                hi = v.y;
            } else {
                lo = __ldg(blk + i);
                hi = __ldg(blk + i + 1);
            }
        }
        w[e] = PART == 0 ? lo : PART == 1 ? hi : (lo ^ hi);
    }
}

template <int PART>
__device__ __forceinline__ uint64_t half_product64(const uint32_t *xb, const uint32_t *yb, const ExtractArgs &a) {
    uint32_t acc[63];
#pragma unroll
    for (int i = 0; i < 63; ++i) acc[i] = 0;
    for (uint32_t g0 = 0; g0 < a.wpb; g0 += 64) {
        uint32_t X[32], Y[32];
        load_half64<PART>(xb, g0, a.wpb, a.vec8, X);
        load_half64<PART>(yb, g0, a.wpb, a.vec8, Y);
        slice<32>(X, a.mu);
        slice<32>(Y, a.mu);
        gram_diagonals<32>(X, Y, acc);
    }
    return uint64_t(parity_bits32<32>(acc, a.mu)) | (uint64_t(parity_bits32<31>(acc + 32, a.mu)) << 32);
}

template <>
__device__ __forceinline__ uint64_t block_value<64>(const uint32_t *xb, const uint32_t *yb, const ExtractArgs &a) {
    const uint64_t A = half_product64<0>(xb, yb, a);
    const uint64_t B = half_product64<1>(xb, yb, a);
    const uint64_t C = half_product64<2>(xb, yb, a);
    const uint64_t M = C ^ A ^ B;  // middle term, degree <= 62
    const uint64_t lo = A ^ (M << 32);
    const uint64_t hi = B ^ (M >> 32);
    return reduce_64(lo, hi, a);
}

// ---------------------------------------------------------------------------
// Output: 32 consecutive blocks (one per lane, starting at a multiple of 32)
// own exactly m output words.  Lane w assembles word w (and w + 32) from the
// m-bit values of the lanes whose bit ranges meet it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_warp(uint64_t v, uint64_t base, const ExtractArgs &a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t m = a.m;
    const uint64_t word0 = (base >> 5) * m;
    const uint64_t total = (a.nblocks * m + 31) >> 5;
    const uint32_t reach = 31u / m + 2u;  // most lanes that can meet one word
    for (uint32_t r = 0; r * 32u < m; ++r) {
        const uint32_t w = lane + 32u * r;
        const uint32_t first = (32u * w) / m;
        uint32_t word = 0;
        for (uint32_t t = 0; t < reach; ++t) {
            const uint32_t i = first + t;
            const uint64_t vi = __shfl_sync(0xffffffffu, v, int(i < 32u ? i : 31u));
            const int s = int(i * m) - int(32u * w);
            if (w < m && i < 32u && s < 32) {
                if (s >= 0)
                    word |= uint32_t(vi << s);
                else if (s > -64)
                    word |= uint32_t(vi >> (-s));
            }
        }
        if (w < m && word0 + w < total) a.out[word0 + w] = word;
    }
}

template <int Q>
__global__ void __launch_bounds__(128) extract_kernel(const ExtractArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t mmask = a.m >= 64 ? ~uint64_t(0) : ((uint64_t(1) << a.m) - 1);
    for (uint64_t base = warp * 32; base < a.nblocks; base += nwarps * 32) {
        const uint64_t blk = base + lane;
        uint64_t v = 0;
        if (blk < a.nblocks) v = block_value<Q>(a.x + blk * a.wpb, a.y + blk * a.wpb, a) & mmask;
        store_warp(v, base, a);
    }
}

template <int Q>
int launch_q(const ExtractArgs &a, cudaStream_t s) {
    static int grid_cap = 0;
    if (!grid_cap) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return QEXT_E_CUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QEXT_E_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, extract_kernel<Q>, 128, 0) != cudaSuccess)
            return QEXT_E_CUDA;
        grid_cap = sms * (per_sm > 0 ? per_sm : 1);
    }
    const uint64_t warps = (a.nblocks + 31) / 32;
    const uint64_t ctas = (warps + 3) / 4;
    const int grid = int(ctas < uint64_t(grid_cap) ? ctas : uint64_t(grid_cap));
    extract_kernel<Q><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? QEXT_OK : QEXT_E_CUDA;
}

}  // namespace

namespace qext {

int launch_extract(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                   qext_cuda_stream stream) {
    ExtractArgs a;
    a.x = x;
    a.y = y;
    a.out = out;
    a.nblocks = nblocks;
    a.wpb = p->n / 32;
    a.m = p->m;
    a.ntaps = p->ntaps;
    for (int i = 0; i < 4; ++i) a.taps[i] = p->taps[i];
    const uintptr_t al = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y);
    a.vec16 = (al % 16 == 0) && (a.wpb % 4 == 0);
    a.vec8 = (al % 8 == 0) && (a.wpb % 2 == 0);
    for (int i = 0; i < 3; ++i) {
        a.mu.lo[i] = 1u << (1 << i);
        a.mu.hi[i] = 1u << (32 - (1 << i));
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (p->q) {
        case 1: return launch_q<1>(a, s);
        case 2: return launch_q<2>(a, s);
        case 4: return launch_q<4>(a, s);
        case 8: return launch_q<8>(a, s);
        case 16: return launch_q<16>(a, s);
        case 32: return launch_q<32>(a, s);
        case 64: return launch_q<64>(a, s);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace qext
