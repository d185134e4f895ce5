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
        // truncate to m bits
        uint32_t v[3] = {uint32_t(r0), uint32_t(r0 >> 32), r1};
        if (s.m < 64) {
            v[2] = 0;
            v[1] = s.m <= 32 ? 0u : v[1] & uint32_t(mask_m(s.m - 32));
            if (s.m < 32) v[0] &= uint32_t(mask_m(s.m));
        } else if (s.m < 80) {
            v[2] &= uint32_t(mask_m(s.m - 64));
        }
        if (blk >= s.nblocks) v[0] = v[1] = v[2] = 0;
        if (s.m <= 64)
            store_warp(uint64_t(v[0]) | (uint64_t(v[1]) << 32), base, s.nblocks, s.m, s.out);
        else
            store_warp_wide(v, base, s.nblocks, s.m, s.out);
    }
}

}  // namespace

namespace qext {

int launch_extract_q80(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                       qext_cuda_stream stream) {
    if (p->q != 80) return QEXT_E_UNSUPPORTED;
    if (nblocks == 0) return QEXT_OK;
    static DeviceSlots grid_caps;
    const int dev = current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int grid_cap = grid_caps.get(dev, [dev] {
        int occ = 0;
        const int sms = sm_count(dev);
        if (sms <= 0 || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, extract_q80_kernel, kThreads80, 0) !=
                            cudaSuccess)
            return 0;
        return sms * (occ > 0 ? occ : 1);
    });
    if (grid_cap <= 0) return QEXT_E_CUDA;
    Q80Args a;
    a.s.x = x;
    a.s.y = y;
    a.s.out = out;
    a.s.nblocks = nblocks;
    a.s.wpb = 0;  // blocks need not be whole words
    a.s.m = p->m;
    a.s.ntaps = p->ntaps;
    for (int i = 0; i < 4; ++i) {
        a.s.taps[i] = p->taps[i];
    }
    a.s.set_multipliers();
    a.s.status = device_status_ptr();
    a.n_p = p->n_p;
    a.zero = 0;
    const uint64_t ctas = (nblocks + kThreads80 - 1) / kThreads80;
    const int grid = int(ctas < uint64_t(grid_cap) ? ctas : uint64_t(grid_cap));
    return launch_pdl(extract_q80_kernel, grid, kThreads80, 0, reinterpret_cast<cudaStream_t>(stream), a);
}

}  // namespace qext
