// Extraction at the paper's own field size, q = 80 (Sec. 4.2: n_p = 71,
// 5680-bit blocks of 16-bit samples), for any n_p: Ext_IP^{n_p,80}
// (Definition 3.2) per block of Algorithm 1, one block per thread.
//
// Layout.  Block l is stream bits [l*n, (l+1)*n), n = 80 n_p, element i its
// bits [80i, 80i+80).  Both l*n and 80i are multiples of 16, so every element
// starts on a 16-bit boundary: its parts x0 (bits 0..31), x1 (32..63) and
// x2 (64..79) are read from one or two stream words with one PRMT.  The
// loads of a warp's 32 blocks are coalesced through a shared staging array
// (load_part32).
//
// Product.  Three-way Karatsuba over the parts (six products instead of
// nine):  x*y = P00 + t^32 (P01 - P00 - P11) + t^64 (P02 - P00 - P22 + P11)
//             + t^96 (P12 - P11 - P22) + t^128 P22,
// with Pab = (xa + xb)(ya + yb), Paa = xa ya.  Each is accumulated over the
// block's elements as sliced Gram-diagonal parities, 32 elements per group:
// the 32-bit parts by a 32 x 32 transpose (element e in slot e) and
// gram32_parities (two more Karatsuba levels, parities in byte fields), x2 by
// slice<16> with elements k and k+16 in word k (which
// also puts element e in slot e, so x0 + x2 is a slot-wise XOR of slices).
// Parities are linear, so groups and Karatsuba parts combine after the
// POPCs; the 159-bit sum is reduced mod P once per block.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_block.cuh"
#include "qext_wide.cuh"
#include "qext_internal.h"

using namespace qxd;

namespace {

constexpr int kThreads80 = 64;

struct Q80Args {
    StreamArgs s;
    uint32_t n_p;
    uint32_t zero;  // always 0 (see after())
};

// Left alone, the compilers overlap the products of a group (loads and
// slicing of the next product hoisted into the previous one: several hundred
// registers).  Each load therefore takes its blocks' base through a run-time
// zero (`zero` = 0, a kernel argument) added to the previous result: base +
// (value & zero) cannot be formed before that value exists.
__device__ __forceinline__ uint64_t after(uint64_t base, uint64_t done, uint32_t zero) {
    return base + (uint32_t(done) & zero);
}

// Operand loads through a per-warp staging array.  Thread t of a warp owns
// block base + t, whose elements lie 710 bytes (n / 8) apart from the next
// block's: one element per thread would touch 32 lines per load.  Instead
// lane j loads element 32g + j of each of the warp's 32 blocks in turn (the
// 32 lanes read 320 consecutive bytes: three lines per load), the values go
// through shared memory (row b = block b, rows padded to an odd number of
// words so that both the row writes and the column reads are conflict-free)
// and each thread reads back its own block's row.  Blocks past nblocks
// repeat the last block (their outputs are not stored); elements past n_p
// read as 0.  A block's bit 0 and every element start on a 16-bit boundary,
// so a part is one PRMT of the two words it touches.
constexpr uint32_t kStageRow32 = 33;  // words per staged row of 32-bit parts
constexpr uint32_t kStageRow16 = 17;  // words per staged row of x2 pairs
constexpr uint32_t kStageWords = 32 * kStageRow32;

// 32-bit part A (0: bits 0..31, 1: bits 32..63) of elements 32g + e, e < 32,
// of the thread's block: R[e] (element e in word e).
template <int A>
__device__ __forceinline__ void load_part32(const uint32_t *__restrict__ w, uint64_t base, uint64_t nblocks,
                                            uint64_t n, uint32_t g, uint32_t n_p, uint32_t *stage,
                                            uint32_t (&R)[32]) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t elem = 32 * g + lane;
    const bool in = elem < n_p;
    const uint64_t off = 80ull * (in ? elem : 0u) + 32 * A;
#pragma unroll 16
    for (uint32_t b = 0; b < 32; ++b) {
        const uint64_t blk = base + b < nblocks ? base + b : nblocks - 1;
        const uint64_t bit = blk * n + off;
        const uint32_t *p = w + (bit >> 5);
        const uint32_t v = __byte_perm(__ldg(p), __ldg(p + 1), (bit & 16u) ? 0x5432u : 0x3210u);
        stage[b * kStageRow32 + lane] = in ? v : 0u;
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 32; ++e) R[e] = stage[lane * kStageRow32 + e];
    __syncwarp();  // the next load reuses the stage
}

// x2 parts (bits 64..79) of elements 32g + k and 32g + k + 16 in word k of
// R (low and high half), k < 16, of the thread's block.
__device__ __forceinline__ void load_part16(const uint32_t *__restrict__ w, uint64_t base, uint64_t nblocks,
                                            uint64_t n, uint32_t g, uint32_t n_p, uint32_t *stage,
                                            uint32_t (&R)[16]) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t elem = 32 * g + lane;
    const bool in = elem < n_p;
    const uint64_t off = 80ull * (in ? elem : 0u) + 64;
#pragma unroll 16
    for (uint32_t b = 0; b < 32; ++b) {
        const uint64_t blk = base + b < nblocks ? base + b : nblocks - 1;
        const uint64_t bit = blk * n + off;
        const uint32_t word = __ldg(w + (bit >> 5));
        const uint32_t v = in ? ((bit & 16u) ? word >> 16 : word & 0xFFFFu) : 0u;
        const uint32_t hi = __shfl_down_sync(0xffffffffu, v, 16);  // element 32g + lane + 16
        if (lane < 16) stage[b * kStageRow16 + lane] = v | (hi << 16);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) R[k] = stage[lane * kStageRow16 + k];
    __syncwarp();
}

// z (159 bits: z0 = bits 0..63, z1 = 64..127, z2 = 128..158) mod P, P = x^80 +
// sum of taps (descending, last 0): two folds (2c - 2 < 80 checked at plan time).
__device__ __forceinline__ void reduce_mod_p80(uint64_t z0, uint64_t z1, uint64_t z2, const StreamArgs &s,
                                               uint64_t &r0, uint32_t &r1) {
    // fold 1: H = z >> 80 (79 bits)
    uint64_t h0 = (z1 >> 16) | (z2 << 48), h1 = z2 >> 16;
    uint64_t l0 = z0, l1 = z1 & 0xFFFFull;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(s.ntaps)) {
            const uint32_t c = s.taps[t];
            l0 ^= h0 << c;
            l1 ^= c ? (h1 << c) | (h0 >> (64 - c)) : h1;
        }
    // fold 2: bits 80 .. 80 + c of the result
    const uint64_t g = l1 >> 16;
    l1 &= 0xFFFFull;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < int(s.ntaps)) {
            const uint32_t c = s.taps[t];
            l0 ^= g << c;
            l1 ^= c ? g >> (64 - c) : 0u;
        }
    r0 = l0;
    r1 = uint32_t(l1);
}

// Bits [off, off + 32) of a value held as three words (v[2] holds its top bits).
__device__ __forceinline__ uint32_t bits32(const uint32_t (&v)[3], uint32_t off) {
    const uint32_t i = off >> 5, sh = off & 31u;
    const uint32_t a = i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : 0u;
    const uint32_t b = i == 0 ? v[1] : i == 1 ? v[2] : 0u;
    return sh ? __funnelshift_r(a, b, sh) : a;
}

// Output of 32 consecutive blocks base .. base+31 (one per lane, 32 < m <= 96
// bits, value v truncated to m bits and 0 past nblocks): the warp owns exactly
// m output words starting at word (base / 32) * m; with m > 32 a word holds
// bits of at most two blocks.
__device__ __forceinline__ void store_warp_wide(const uint32_t (&v)[3], uint64_t base, uint64_t nblocks, uint32_t m,
                                                uint32_t *__restrict__ out) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t word0 = (base >> 5) * m;
    const uint64_t total = (nblocks * m + 31) >> 5;
    for (uint32_t r = 0; r * 32u < m; ++r) {
        const uint32_t w = lane + 32u * r;            // the warp's output word w: bits [32w, 32w + 32)
        const uint32_t first = w < m ? (32u * w) / m : 0u;
        const uint32_t off = 32u * w - first * m;      // bit offset inside block `first`
        uint32_t a[3], b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            a[i] = __shfl_sync(0xffffffffu, v[i], int(first));
            b[i] = __shfl_sync(0xffffffffu, v[i], int(first + 1 < 32u ? first + 1 : 31u));
        }
        if (w < m) {
            uint32_t word = bits32(a, off);
            if (off + 32u > m) {
                const uint32_t keep = m - off;  // bits still from block `first` (1 .. 31)
                word = (word & ((1u << keep) - 1u)) | (first + 1 < 32u ? b[0] << keep : 0u);
            }
            if (word0 + w < total) out[word0 + w] = word;
        }
    }
}

// Truncation of an 80-bit value (three words) to its low m bits.
__device__ __forceinline__ void truncate80(uint32_t (&v)[3], uint32_t m) {
    if (m < 64) {
        v[2] = 0;
        v[1] = m <= 32 ? 0u : v[1] & uint32_t(mask_m(m - 32));
        if (m < 32) v[0] &= uint32_t(mask_m(m));
    } else if (m < 80) {
        v[2] &= uint32_t(mask_m(m - 64));
    }
}

__global__ void __launch_bounds__(kThreads80, 6) extract_q80_kernel(const Q80Args a) {
    // per thread: 80 sliced words of each source, interleaved across threads
    // (word k of thread t at k * kThreads80 + t: conflict-free)
    __shared__ uint32_t slices[2 * 80 * kThreads80];
    __shared__ uint32_t stages[kThreads80 / 32][kStageWords];
    uint32_t *const sl = slices + threadIdx.x;
    uint32_t *const stage = stages[threadIdx.x >> 5];
    pdl_prologue();
    const StreamArgs &s = a.s;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t n = 80ull * a.n_p;
    const uint32_t ngroups = (a.n_p + 31) / 32;
    for (uint64_t base = warp * 32; base < s.nblocks; base += nwarps * 32) {
        const uint64_t blk = base + lane;
        uint64_t p00 = 0, p11 = 0, p01 = 0, p02 = 0, p12 = 0;
        uint32_t p22 = 0;
        for (uint32_t g = 0; g < ngroups; ++g) {
            // slice each part of both sources once into this thread's
            // column of the shared array (word k at sl[k * nthreads]):
            // S0 = slices 0..31, S1 = 32..63, S2 = 64..79 (x), +80 (y)
            uint64_t dep = p02;  // after the previous group
#pragma unroll 1
            for (uint32_t src = 0; src < 2; ++src) {
                const uint32_t *ws = src ? s.y : s.x;
                uint32_t *const col = sl + src * 80 * kThreads80;
                {
                    uint32_t R[32];
                    load_part32<0>(ws, after(base, dep, a.zero), s.nblocks, n, g, a.n_p, stage, R);
                    slice<32>(R);
#pragma unroll
                    for (int k = 0; k < 32; ++k) col[k * kThreads80] = R[k];
                    dep = R[31];
                }
                {
                    uint32_t R[32];
                    load_part32<1>(ws, after(base, dep, a.zero), s.nblocks, n, g, a.n_p, stage, R);
                    slice<32>(R);
#pragma unroll
                    for (int k = 0; k < 32; ++k) col[(32 + k) * kThreads80] = R[k];
                    dep = R[31];
                }
                {
                    uint32_t R[16];
                    load_part16(ws, after(base, dep, a.zero), s.nblocks, n, g, a.n_p, stage, R);
                    slice<16>(R);
#pragma unroll
                    for (int k = 0; k < 16; ++k) col[(64 + k) * kThreads80] = R[k];
                    dep = R[15];
                }
            }
            const uint32_t *const cx = sl, *const cy = sl + 80 * kThreads80;
            {
                uint32_t X2[16], Y2[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    X2[k] = cx[(64 + k) * kThreads80];
                    Y2[k] = cy[(64 + k) * kThreads80];
                }
                p22 ^= diagonal_chain<16>(X2, Y2) >> 1;
            }
            // the five 32 x 32 products; operands are XORs of slices (slicing
            // is linear):  pr 0: S1 (P11), 1: S1 + S2 (P12), 2: S0 + S1 (P01),
            // 3: S0 (P00), 4: S0 + S2 (P02), S2 covering slices 0..15
#pragma unroll 1
            for (uint32_t pr = 0; pr < 5; ++pr) {
                uint32_t X[32], Y[32];
                const uint32_t first = pr <= 2 ? 32u : 0u;  // S1 or S0
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    X[k] = cx[(first + k) * kThreads80];
                    Y[k] = cy[(first + k) * kThreads80];
                }
                if (pr == 2) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        X[k] ^= cx[k * kThreads80];
                        Y[k] ^= cy[k * kThreads80];
                    }
                } else if (pr == 1 || pr == 4) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        X[k] ^= cx[(64 + k) * kThreads80];
                        Y[k] ^= cy[(64 + k) * kThreads80];
                    }
                }
                const uint64_t r = gram32_parities(X, Y, s);
                p11 ^= pr == 0 ? r : 0;
                p12 ^= pr == 1 ? r : 0;
                p01 ^= pr == 2 ? r : 0;
                p00 ^= pr == 3 ? r : 0;
                p02 ^= pr == 4 ? r : 0;
            }
        }
        // recombine the six products (63-bit parities; P22 31-bit)
        const uint64_t t1 = p01 ^ p00 ^ p11, t2 = p02 ^ p00 ^ p11 ^ p22, t3 = p12 ^ p11 ^ p22;
        const uint64_t z0 = p00 ^ (t1 << 32), z1 = (t1 >> 32) ^ t2 ^ (t3 << 32), z2 = (t3 >> 32) ^ p22;
        uint64_t r0;
        uint32_t r1;
        reduce_mod_p80(z0, z1, z2, s, r0, r1);
        uint32_t v[3] = {uint32_t(r0), uint32_t(r0 >> 32), r1};
        truncate80(v, s.m);
        if (blk >= s.nblocks) v[0] = v[1] = v[2] = 0;
        if (s.m <= 64)
            store_warp(uint64_t(v[0]) | (uint64_t(v[1]) << 32), base, s.nblocks, s.m, s.out);
        else
            store_warp_wide(v, base, s.nblocks, s.m, s.out);
    }
}

// ---------------------------------------------------------------------------
// Blocks in lanes (the default for n_p up to the shared-memory limit).  A CTA
// takes tiles of 32 consecutive blocks; bit b of every sliced word belongs to
// block b of the tile, so one AND-XOR serves 32 blocks and the Gram sums
// need no parities: word k of the accumulated product is coefficient k of
// the 32 blocks' unreduced sums.  An element is split into five 16-bit
// column groups G_0..G_4 (x = sum_c G_c u^c, u = t^16) and multiplied by
// the generalised Karatsuba formula over them (Weimerskirch and Paar,
// "Generalizations of the Karatsuba Algorithm for Efficient
// Implementations", 2006):
//     x y = sum_c P_cc u^2c + sum_{c<d} (P_cd + P_cc + P_dd) u^(c+d),
//     P_cd = (G_c(x) + G_d(x)) (G_c(y) + G_d(y)),
// fifteen 16 x 16 sliced products, each by two Karatsuba levels (8-word,
// then 4-word halves: the accumulators of Acc16K2).  The products are linear in their accumulators, so every thread
// keeps one product's accumulators across all elements of the tile and the
// recombination (fifteen products into the 159-bit sum) runs once per tile.
//
// Per tile: the 32 blocks of both sources arrive by one bulk copy each (or
// plain loads for a ragged last tile or unaligned sources); elements are
// processed in chunks of kChunk80: 5 x 2 x kChunk80 threads slice one column
// group of one element of one source each (32 halfword rows -> 16 words),
// then 15 x kChunk80 threads multiply, thread (slot e, product u) taking
// element e of the chunk.  The next tile's copy is issued once the last
// chunk is sliced.  At the end of the tile the accumulators are summed over
// the slots, recombined into the 159 coefficient words, transposed back to
// one value per block and reduced mod P by warp 0.
// ---------------------------------------------------------------------------
constexpr int kThreadsLanes = 128;
constexpr uint32_t kChunk80 = 8;          // elements per chunk
constexpr uint32_t kProducts80 = 15;      // P_cd, c <= d < 5
constexpr uint32_t kVecStride = 20;       // words between column-group vectors (distinct bank groups)
constexpr uint32_t kSliceStride = 5 * kVecStride;  // words per (element, source)
constexpr uint32_t kRedWords = (kThreadsLanes / 32) * kProducts80 * 31;  // per-warp partial products
constexpr uint32_t kWorkWords =           // slices, or (aliased) the tile's recombination buffers
    (2 * kChunk80 * kSliceStride > kRedWords + 160 + 160) ? 2 * kChunk80 * kSliceStride : kRedWords + 160 + 160;

// Products 0..4 are P_cc, 5..14 the pairs c < d in lexicographic order.
__host__ __device__ constexpr uint32_t product_lo(uint32_t u) {
    return u < 5 ? u : u < 9 ? 0 : u < 12 ? 1 : u < 14 ? 2 : 3;
}
__host__ __device__ constexpr uint32_t product_hi(uint32_t u) {
    return u < 5 ? u : u < 9 ? u - 4 : u < 12 ? u - 7 : u < 14 ? u - 9 : 4;
}

// Products placed at u^m in x y (m = 0 .. 8): P_cd with c < d, c + d = m, and
// P_cc with 0 <= m - c <= 4 (at u^2c, and at u^(c+e) for every e != c).
__constant__ uint8_t kAtOffset[9][7] = {{0},          {0, 1, 5},          {0, 1, 2, 6},    {0, 1, 2, 3, 7, 9},
                                        {0, 1, 2, 3, 4, 8, 10}, {1, 2, 3, 4, 11, 12}, {2, 3, 4, 13}, {3, 4, 14},
                                        {4}};
__constant__ uint8_t kAtOffsetLen[9] = {1, 3, 4, 6, 7, 6, 4, 3, 1};

// 32 x 32 bit transpose across a warp: lane e holds row e on entry, column
// e on return (bit b of lane e's result = bit e of lane b's row), by five
// exchange stages between lanes G apart.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t w, uint32_t lane) {
    constexpr uint32_t kLow[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t G = 16u >> i, M = kLow[i];
        const uint32_t v = __shfl_xor_sync(0xffffffffu, w, int(G));
        w = (lane & G) ? lop_select(v >> G, w, M) : lop_select(w, v << G, M);
    }
    return w;
}

struct LanesArgs {
    StreamArgs s;
    uint32_t n_p;
    int bulk;             // sources 16-byte aligned: whole tiles arrive by bulk copy
    uint64_t src_words;   // readable words of each source, ceil(nblocks n / 32)
    uint32_t max_polls;   // bound of every mbarrier wait
    int no_copy;          // test of failure detection: barrier armed, no copy issued
};

// NP > 0: n_p fixed at compile time (the row strides of the slicing become
// immediate offsets); NP = 0: any n_p.
template <uint32_t NP>
__global__ void __launch_bounds__(kThreadsLanes, 4) extract_q80_lanes_kernel(const LanesArgs a) {
    extern __shared__ __align__(16) uint32_t smem80[];
    __shared__ __align__(8) uint64_t bar;
    const StreamArgs &s = a.s;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t n_p = NP ? NP : a.n_p, n = 80 * n_p, hw_row = 5 * n_p;  // hw_row: halfwords per block row
    // y tile 16 bytes past the x tile (the slicing reads spread over the banks)
    const uint32_t y_off = n + 4;
    uint32_t *const tin = smem80;               // x tile, then y tile
    uint32_t *const work = smem80 + y_off + n;  // slices / recombination
    const uint64_t ntiles = (s.nblocks + 31) / 32;
    auto full_tile = [&](uint64_t t) { return a.bulk && 32 * (t + 1) <= s.nblocks; };
    auto issue = [&](uint64_t t) {
        mbar_expect_tx(&bar, 8u * n);
        if (a.no_copy) return;  // the completion never comes: the wait must give up
        tma_load_1d(tin, s.x + t * n, 4u * n, &bar);
        tma_load_1d(tin + y_off, s.y + t * n, 4u * n, &bar);
    };
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_prologue();
    uint64_t t = blockIdx.x;
    if (tid == 0 && t < ntiles && full_tile(t)) issue(t);
    const uint32_t u = tid & 15u, slot = tid >> 4;
    const uint32_t ca = product_lo(u < kProducts80 ? u : 0), cb = product_hi(u < kProducts80 ? u : 0);
    const uint32_t pmask = ca == cb ? 0u : ~0u;
    for (uint32_t phase = 0; t < ntiles; t += gridDim.x) {
        if (full_tile(t)) {
            const bool ok = mbar_wait_bounded(&bar, phase & 1u, a.max_polls);
            ++phase;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    record_status(s.status, QEXT_E_TIMEOUT);
                    if (!a.no_copy) mbar_wait_bounded(&bar, (phase - 1) & 1u, a.max_polls);  // let the copies land
                }
                return;
            }
        } else {
            // ragged last tile or unaligned sources: plain loads, zeros past the streams
            for (uint32_t i = tid; i < n; i += kThreadsLanes) {
                const uint64_t w = t * n + i;
                tin[i] = w < a.src_words ? s.x[w] : 0u;
                tin[y_off + i] = w < a.src_words ? s.y[w] : 0u;
            }
            __syncthreads();
        }
        Acc16K2 acc;  // this thread's product, over every element of the tile
        for (uint32_t c0 = 0; c0 < n_p; c0 += kChunk80) {
            // slicing: job (element e, source src, column group g)
            if (tid < 10 * kChunk80) {
                const uint32_t e = tid / 10, src = (tid / 5) & 1u, g = tid % 5;
                if (c0 + e < n_p) {
                    const uint16_t *const rows =
                        reinterpret_cast<const uint16_t *>(tin + src * y_off) + 5 * (c0 + e) + g;
                    uint32_t W[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        W[k] = __byte_perm(rows[k * hw_row], rows[(k + 16) * hw_row], 0x5410);
                    slice<16>(W);  // word j: bit j of the group, row b in bit b
                    uint32_t *const dst = work + (2 * e + src) * kSliceStride + kVecStride * g;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        *reinterpret_cast<uint4 *>(dst + 4 * k) = make_uint4(W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3]);
                }
            }
            __syncthreads();
            if (c0 + kChunk80 >= n_p && tid == 0 && t + gridDim.x < ntiles && full_tile(t + gridDim.x))
                issue(t + gridDim.x);  // every row of this tile is sliced: the tile buffer is free
            if (u < kProducts80 && c0 + slot < n_p) {
                const uint32_t *const ex = work + 2 * slot * kSliceStride, *const ey = ex + kSliceStride;
                uint32_t X[16], Y[16];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 xa = lds4(ex + kVecStride * ca + 4 * k), xb = lds4(ex + kVecStride * cb + 4 * k);
                    const uint4 ya = lds4(ey + kVecStride * ca + 4 * k), yb = lds4(ey + kVecStride * cb + 4 * k);
                    X[4 * k] = lop_and_xor(xb.x, pmask, xa.x);
                    X[4 * k + 1] = lop_and_xor(xb.y, pmask, xa.y);
                    X[4 * k + 2] = lop_and_xor(xb.z, pmask, xa.z);
                    X[4 * k + 3] = lop_and_xor(xb.w, pmask, xa.w);
                    Y[4 * k] = lop_and_xor(yb.x, pmask, ya.x);
                    Y[4 * k + 1] = lop_and_xor(yb.y, pmask, ya.y);
                    Y[4 * k + 2] = lop_and_xor(yb.z, pmask, ya.z);
                    Y[4 * k + 3] = lop_and_xor(yb.w, pmask, ya.w);
                }
                acc.add(X, Y);  // two Karatsuba levels (8 + 8, then 4 + 4), word accumulators
            }
            __syncthreads();
        }
        // the product's 31 coefficient words: R = D (1 + t^8) + t^8 C with
        // D = F (1 + t^4) + t^4 G and C = E (1 + t^4) + t^4 M (Acc16K2's parts),
        // summed over the slots (two per warp by a shuffle, then over the warps)
        uint32_t *const red = work, *const zw = work + kRedWords, *const ow = zw + 160;
        {
            uint32_t D[23], C[15], R[31];
#pragma unroll
            for (int k = 0; k < 23; ++k)
                D[k] = (k < 19 ? acc.F[k] : 0u) ^ (k >= 4 ? acc.F[k - 4] ^ (k - 4 < 15 ? acc.G[k - 4] : 0u) : 0u);
#pragma unroll
            for (int k = 0; k < 15; ++k)
                C[k] = (k < 11 ? acc.E[k] : 0u) ^ (k >= 4 ? acc.E[k - 4] ^ (k - 4 < 7 ? acc.M[k - 4] : 0u) : 0u);
#pragma unroll
            for (int k = 0; k < 31; ++k) {
                uint32_t r = k < 23 ? D[k] : 0u;
                if (k >= 8) r ^= D[k - 8] ^ (k - 8 < 15 ? C[k - 8] : 0u);
                R[k] = r ^ __shfl_xor_sync(0xffffffffu, r, 16);
            }
            if (lane < kProducts80) {
#pragma unroll
                for (int k = 0; k < 31; ++k) red[(warp * kProducts80 + lane) * 31 + k] = R[k];
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < kProducts80 * 31; i += kThreadsLanes) {
            uint32_t r = red[i];
#pragma unroll
            for (uint32_t w = 1; w < kThreadsLanes / 32; ++w) r ^= red[w * kProducts80 * 31 + i];
            red[i] = r;
        }
        __syncthreads();
        // z_k: the products placed at u^m for the (at most two) m with
        // 16m <= k < 16m + 31
        for (uint32_t k = tid; k < 160; k += kThreadsLanes) {
            uint32_t z = 0;
#pragma unroll
            for (uint32_t mm = 0; mm < 2; ++mm) {
                const uint32_t m = (k >> 4) - mm, idx = k - 16 * m;  // m = -1 wraps past 8
                if (m <= 8 && idx < 31) {
                    const uint32_t len = kAtOffsetLen[m];
                    for (uint32_t j = 0; j < len; ++j) z ^= red[kAtOffset[m][j] * 31 + idx];
                }
            }
            zw[k] = z;
        }
        __syncthreads();
        // back to one value per block: words 32g .. 32g + 31 of z transposed
        // by warp g (warp 0 also takes g = 4)
        for (uint32_t g = warp; g < 5; g += kThreadsLanes / 32) ow[32 * g + lane] = warp_transpose32(zw[32 * g + lane], lane);
        __syncthreads();
        if (warp == 0) {
            const uint64_t z0 = ow[lane] | (uint64_t(ow[32 + lane]) << 32);
            const uint64_t z1 = ow[64 + lane] | (uint64_t(ow[96 + lane]) << 32);
            const uint64_t z2 = ow[128 + lane];
            uint64_t r0;
            uint32_t r1;
            reduce_mod_p80(z0, z1, z2, s, r0, r1);
            uint32_t v[3] = {uint32_t(r0), uint32_t(r0 >> 32), r1};
            truncate80(v, s.m);
            const uint64_t base = 32 * t;
            if (base + lane >= s.nblocks) v[0] = v[1] = v[2] = 0;
            if (s.m <= 64)
                store_warp(uint64_t(v[0]) | (uint64_t(v[1]) << 32), base, s.nblocks, s.m, s.out);
            else
                store_warp_wide(v, base, s.nblocks, s.m, s.out);
        }
        // the next tile's first slicing overwrites the buffers warp 0 reads:
        // the barrier after its copy (or its loads) orders them
    }
}

}  // namespace

namespace qext {

int launch_extract_q80(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                       qext_cuda_stream stream, uint32_t flags) {
    if (p->q != 80) return QEXT_E_UNSUPPORTED;
    if (flags & ~uint32_t(QEXT_F_TEST_TIMEOUT)) return QEXT_E_INVAL;
    if (nblocks == 0) return QEXT_OK;
    static DeviceSlots grid_caps, smem_optin, attr_set[2];
    const int dev = current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int sms = sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    StreamArgs s;
    s.x = x;
    s.y = y;
    s.out = out;
    s.nblocks = nblocks;
    s.wpb = 0;  // blocks need not be whole words
    s.m = p->m;
    s.ntaps = p->ntaps;
    for (int i = 0; i < 4; ++i) s.taps[i] = p->taps[i];
    s.set_multipliers();
    s.status = device_status_ptr();

    // blocks in lanes while two tiles of 32 blocks and the work buffers fit
    const int optin = smem_optin.get(dev, [dev] {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess ? v : 0;
    });
    if (optin <= 0) return QEXT_E_CUDA;
    const uint64_t n = 80ull * p->n_p;
    const uint64_t lanes_smem = (2 * n + 4 + kWorkWords) * 4;
    if (lanes_smem + 1024 <= uint64_t(optin)) {
        // the paper's n_p = 71 with compile-time row strides, any other n_p at run time
        const bool fixed = p->n_p == 71;
        void (*const kernel)(const LanesArgs) = fixed ? extract_q80_lanes_kernel<71> : extract_q80_lanes_kernel<0>;
        if (attr_set[fixed].get(dev, [optin, kernel] {
                return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024) ==
                               cudaSuccess ? 1 : 0;
            }) <= 0)
            return QEXT_E_CUDA;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreadsLanes, size_t(lanes_smem)) !=
            cudaSuccess)
            return QEXT_E_CUDA;
        LanesArgs a;
        a.s = s;
        a.n_p = p->n_p;
        a.bulk = (reinterpret_cast<uintptr_t>(x) % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0) ? 1 : 0;
        a.src_words = (nblocks * n + 31) / 32;
        a.no_copy = (flags & QEXT_F_TEST_TIMEOUT) ? 1 : 0;
        a.max_polls = a.no_copy ? 256u : kMaxPolls;
        // the test needs every tile on the bulk-copy path
        if (a.no_copy && (!a.bulk || nblocks % 32)) return QEXT_E_INVAL;
        const uint64_t ntiles = (nblocks + 31) / 32, cap = uint64_t(sms) * uint64_t(occ > 0 ? occ : 1);
        const int grid = int(ntiles < cap ? ntiles : cap);
        return launch_pdl(kernel, grid, kThreadsLanes, size_t(lanes_smem), st, a);
    }

    if (flags) return QEXT_E_INVAL;  // one block per thread: no bulk copies to time out
    const int grid_cap = grid_caps.get(dev, [sms] {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, extract_q80_kernel, kThreads80, 0) != cudaSuccess)
            return 0;
        return sms * (occ > 0 ? occ : 1);
    });
    if (grid_cap <= 0) return QEXT_E_CUDA;
    Q80Args a;
    a.s = s;
    a.n_p = p->n_p;
    a.zero = 0;
    const uint64_t ctas = (nblocks + kThreads80 - 1) / kThreads80;
    const int grid = int(ctas < uint64_t(grid_cap) ? ctas : uint64_t(grid_cap));
    return launch_pdl(extract_q80_kernel, grid, kThreads80, 0, st, a);
}

}  // namespace qext
