// Device helpers of the wide fields: q = 64 (elements are word pairs) and
// the 32 x 32 / 16 x 16 sliced Gram products by Karatsuba levels and diagonal
// parities that q = 64, q = 80 and Algorithm 2 share.
#pragma once

#include "qext_block.cuh"

namespace qxd {

// ---------------------------------------------------------------------------
// q = 64 (elements are word pairs: low word = bits 0..31, high = 32..63).
// One Karatsuba level over the halves: z = A + x^64 B + x^32 (C - A - B) with
// A = sum lo*lo, B = sum hi*hi, C = sum (lo^hi)*(lo^hi), each a sliced 32x32
// Gram product over groups of 32 elements (itself split once more, see
// gram32_parities).  Transposition is linear, so C's
// operands are sliced from the XOR of the raw halves.  The thread handles the
// groups g_first, g_first + g_step, ... of its block.
// ---------------------------------------------------------------------------
// Parity chain of the 2H-1 Gram diagonals of X[0..H) x Y[0..H), one diagonal
// at a time (one live accumulator): bit 32 - (2H-1) + d of the result is
// parity(XOR_{j+l=d} X[j] & Y[l]) (see parity_bits32_top).
template <int H>
__device__ __forceinline__ uint32_t diagonal_chain(const uint32_t *X, const uint32_t *Y) {
    static_assert(2 * H - 1 <= 32, "one word of parities");
    uint32_t c = 0;
#pragma unroll
    for (int d = 0; d < 2 * H - 1; ++d) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = d < H ? 0 : d - H + 1; j <= (d < H ? d : H - 1); ++j) acc = lop_and_xor(X[j], Y[d - j], acc);
        c = (c >> 1) + (uint32_t(__popc(acc)) << 31);
    }
    return c;
}

// Parities of the diagonals D0 .. D1-1 of sum_b t^(S b) (X_b x Y_b), where
// X_b = X[O0 + OSTEP b .. + 8) and likewise Y_b: diagonal d takes the pairs
// j + l = d - S b of block b.  One live accumulator per diagonal; bit d - D0
// of the result is the parity of diagonal d.  The parities are assembled in
// byte fields (popcounts of four consecutive diagonals packed by IMADs,
// w = w + popc * 2^(8f), every field <= 32; the four low bits gathered by
// ((w & 0x01010101) * 0x01020408) >> 24 and placed by an IMAD), which keeps
// the assembly on the FMA pipe, off the ALU pipe the products fill.
template <int NB, int O0, int OSTEP, int S, int D0, int D1>
__device__ __forceinline__ uint32_t block_parities(const uint32_t *X, const uint32_t *Y, const StreamArgs &s) {
    static_assert(D1 - D0 >= 1 && D1 - D0 <= 32, "one word of parities");
    uint32_t r = 0, w = 0;
#pragma unroll
    for (int d = D0; d < D1; ++d) {
        uint32_t acc = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int k = d - S * b, o = O0 + OSTEP * b;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (k - j >= 0 && k - j < 8) acc = lop_and_xor(X[o + j], Y[o + k - j], acc);
        }
        const int f = (d - D0) & 3;
        const uint32_t pc = uint32_t(__popc(acc));
        w = f == 0 ? pc : pc * s.byte_pos[f] + w;
        if (f == 3 || d == D1 - 1) {
            const uint32_t nib = ((w & 0x01010101u) * 0x01020408u) >> 24;
            r = nib * s.nib_mul[(d - D0) >> 2] + r;
        }
    }
    return r;
}

// Parities of the 31 diagonals of a sliced 16 x 16 Gram product by one
// Karatsuba level (8 + 8): with D = A + t^8 B (the halves' products, 23
// diagonals, one shared chain per diagonal) and C = (X_L + X_H)(Y_L + Y_H)
// (15), the product is D (1 + t^8) + t^8 C.  Bit d of the result = parity of
// diagonal d.  X and Y are overwritten (their low halves become the sums).
__device__ __forceinline__ uint32_t gram16_parities(uint32_t *X, uint32_t *Y, const StreamArgs &s) {
    const uint32_t d = block_parities<2, 0, 8, 8, 0, 23>(X, Y, s);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        X[j] ^= X[8 + j];
        Y[j] ^= Y[8 + j];
    }
    const uint32_t c = block_parities<1, 0, 0, 0, 0, 15>(X, Y, s);
    return d ^ (d << 8) ^ (c << 8);
}

// Parities of the 63 diagonals of a sliced 32 x 32 Gram product by two
// Karatsuba levels over the slice index (32 -> 16 + 16 -> 8 + 8), nine 8 x 8
// products.  With halves L, H and sum S at each level,
//     u v = A + t^h (A + B + C) + t^2h B = D (1 + t^h) + t^h C,  D = A + t^h B,
// so products whose results are added at a fixed shift share one chain:
//     R = E (1 + t^8)(1 + t^16) + t^8 F (1 + t^16) + t^16 DC (1 + t^8) + t^24 SC
// with E = A_LL + t^8 A_HH + t^16 B_LL + t^24 B_HH (the four diagonal 8 x 8
// blocks), F = A_SS + t^16 B_SS, DC = C_LL + t^8 C_HH, SC = C_SS (A, B, C
// the 16 x 16 products of the outer level): 107 diagonal parities instead
// of 135.  X and Y are overwritten.  Bit d of the result = parity of
// diagonal d.
__device__ __forceinline__ uint64_t gram32_parities(uint32_t (&X)[32], uint32_t (&Y)[32], const StreamArgs &s) {
    const uint64_t E = uint64_t(block_parities<4, 0, 8, 8, 0, 32>(X, Y, s)) |
                       (uint64_t(block_parities<4, 0, 8, 8, 32, 39>(X, Y, s)) << 32);
    // inner sums of A's and B's halves (words 8.. and 24..)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        X[8 + j] ^= X[j];
        Y[8 + j] ^= Y[j];
        X[24 + j] ^= X[16 + j];
        Y[24 + j] ^= Y[16 + j];
    }
    const uint64_t F = uint64_t(block_parities<1, 8, 0, 0, 0, 15>(X, Y, s)) |
                       (uint64_t(block_parities<1, 24, 0, 0, 0, 15>(X, Y, s)) << 16);
    // outer sum (words 0..15) and its inner half sum (words 24..31)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        X[j] ^= X[16 + j];
        Y[j] ^= Y[16 + j];
        X[24 + j] ^= X[8 + j];
        Y[24 + j] ^= Y[8 + j];
        X[8 + j] = X[24 + j] ^ X[j];
        Y[8 + j] = Y[24 + j] ^ Y[j];
    }
    const uint64_t DC = block_parities<2, 0, 8, 8, 0, 23>(X, Y, s);
    const uint64_t SC = block_parities<1, 24, 0, 0, 0, 15>(X, Y, s);
    return E ^ ((E ^ F) << 8) ^ ((E ^ DC) << 16) ^ ((E ^ F ^ DC ^ SC) << 24);
}

// The part's word of an element: PART 0 = lo, 1 = hi, 2 = lo ^ hi; PART -1
// picks at run time, lo or hi by the PRMT selector sel (0x3210 / 0x7654) plus
// hi & mask (mask = ~0 for lo ^ hi): one code path for several parts keeps
// the kernels within the instruction cache.
template <int PART>
__device__ __forceinline__ uint32_t pick64(uint32_t lo, uint32_t hi, uint32_t sel, uint32_t mask) {
    if constexpr (PART < 0) return lop_and_xor(hi, mask, __byte_perm(lo, hi, sel));
    return PART == 0 ? lo : PART == 1 ? hi : (lo ^ hi);
}

template <int PART>
__device__ __forceinline__ uint64_t half_product64(const uint32_t *xs, const uint32_t *ys, uint32_t wpb, int vec,
                                                   uint32_t rot, uint32_t g_first, uint32_t g_step,
                                                   const StreamArgs &s, uint32_t sel = 0x3210u, uint32_t mask = 0) {
    uint64_t z = 0;  // parities are linear: XOR of the groups' parities
    for (uint32_t g0 = 64 * g_first; g0 < wpb; g0 += 64 * g_step) {
        uint32_t X[32], Y[32];
        if (vec) {
            // 16 chunks of 2 elements each, rotated within the group
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const uint32_t w = g0 + 4 * ((uint32_t(c) + rot) & 15u);
                uint4 vx = make_uint4(0, 0, 0, 0), vy = vx;
                if (w < wpb) {
                    vx = lds4(xs + w);
                    vy = lds4(ys + w);
                }
                X[2 * c] = pick64<PART>(vx.x, vx.y, sel, mask);
                X[2 * c + 1] = pick64<PART>(vx.z, vx.w, sel, mask);
                Y[2 * c] = pick64<PART>(vy.x, vy.y, sel, mask);
                Y[2 * c + 1] = pick64<PART>(vy.z, vy.w, sel, mask);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const uint32_t w = g0 + 2 * e;
                const bool in = w < wpb;
                X[e] = in ? pick64<PART>(xs[w], xs[w + 1], sel, mask) : 0u;
                Y[e] = in ? pick64<PART>(ys[w], ys[w + 1], sel, mask) : 0u;
            }
        }
        slice<32>(X);
        slice<32>(Y);
        z ^= gram32_parities(X, Y, s);
    }
    return z;
}

// A, B and C of one thread's groups with a single copy of half_product64
// (a run-time loop over the parts).
__device__ __forceinline__ void half_products64(const uint32_t *xs, const uint32_t *ys, uint32_t wpb, int vec,
                                                uint32_t rot, uint32_t g_first, uint32_t g_step, uint64_t &A,
                                                uint64_t &B, uint64_t &C, const StreamArgs &s) {
#pragma unroll 1
    for (uint32_t part = 0; part < 3; ++part) {
        const uint64_t r = half_product64<-1>(xs, ys, wpb, vec, rot, g_first, g_step, s,
                                              part == 1 ? 0x7654u : 0x3210u, part == 2 ? ~0u : 0u);
        A = part == 0 ? r : A;
        B = part == 1 ? r : B;
        C = part == 2 ? r : C;
    }
}

// A, B and C of one thread's groups, each group sliced once.  Slicing is
// linear, so the slices of lo ^ hi are the XOR of the slices of lo and hi:
// the group's 32 elements (lo and hi words, 64 words per source) are loaded
// once, lo and hi sliced in registers, and the four slice sets written back
// over the group's own 64 words of x and y in shared memory (the raw words are
// no longer needed; chunks in the same lane-rotated order as the loads), then
// read back for A = lo x lo, B = hi x hi and C = (lo ^ hi) x (lo ^ hi).  Two
// transposes fewer per group than half_products64 and no part selection.
// Only whole groups are staged this way: a last group that ends past the
// block (its tail words belong to the next block) goes through
// half_product64.  xs, ys are shared memory; a bulk copy into them later needs
// a proxy fence after this (the caller's).
__device__ __forceinline__ void half_products64_inplace(uint32_t *xs, uint32_t *ys, uint32_t wpb, uint32_t rot,
                                                        uint32_t g_first, uint32_t g_step, uint64_t &A, uint64_t &B,
                                                        uint64_t &C, const StreamArgs &s) {
    A = B = C = 0;
    for (uint32_t g0 = 64 * g_first; g0 < wpb; g0 += 64 * g_step) {
        if (g0 + 64 > wpb) {
            const uint32_t g = g0 / 64, one = wpb;  // a step past the block: this group only
            A ^= half_product64<0>(xs, ys, wpb, 1, rot, g, one, s);
            B ^= half_product64<1>(xs, ys, wpb, 1, rot, g, one, s);
            C ^= half_product64<2>(xs, ys, wpb, 1, rot, g, one, s);
            continue;
        }
#pragma unroll 1
        for (uint32_t src = 0; src < 2; ++src) {
            uint32_t *const w = (src ? ys : xs) + g0;
            uint32_t L[32], H[32];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const uint4 v = lds4(w + 4 * ((uint32_t(c) + rot) & 15u));
                L[2 * c] = v.x;
                H[2 * c] = v.y;
                L[2 * c + 1] = v.z;
                H[2 * c + 1] = v.w;
            }
            slice<32>(L);
            slice<32>(H);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                *reinterpret_cast<uint4 *>(w + 4 * ((uint32_t(k) + rot) & 15u)) =
                    make_uint4(L[4 * k], L[4 * k + 1], L[4 * k + 2], L[4 * k + 3]);
                *reinterpret_cast<uint4 *>(w + 4 * ((uint32_t(k) + 8u + rot) & 15u)) =
                    make_uint4(H[4 * k], H[4 * k + 1], H[4 * k + 2], H[4 * k + 3]);
            }
        }
        const uint32_t *const wx = xs + g0, *const wy = ys + g0;
#pragma unroll 1
        for (uint32_t part = 0; part < 3; ++part) {
            uint32_t X[32], Y[32];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                // lo slices in chunks k + rot, hi slices in chunks k + 8 + rot (mod 16)
                const uint32_t cl = 4 * ((uint32_t(k) + rot) & 15u), ch = 4 * ((uint32_t(k) + 8u + rot) & 15u);
                const uint32_t c0 = part == 1 ? ch : cl;
                uint4 vx = lds4(wx + c0), vy = lds4(wy + c0);
                if (part == 2) {
                    const uint4 hx = lds4(wx + ch), hy = lds4(wy + ch);
                    vx = make_uint4(vx.x ^ hx.x, vx.y ^ hx.y, vx.z ^ hx.z, vx.w ^ hx.w);
                    vy = make_uint4(vy.x ^ hy.x, vy.y ^ hy.y, vy.z ^ hy.z, vy.w ^ hy.w);
                }
                X[4 * k] = vx.x;
                X[4 * k + 1] = vx.y;
                X[4 * k + 2] = vx.z;
                X[4 * k + 3] = vx.w;
                Y[4 * k] = vy.x;
                Y[4 * k + 1] = vy.y;
                Y[4 * k + 2] = vy.z;
                Y[4 * k + 3] = vy.w;
            }
            const uint64_t r = gram32_parities(X, Y, s);
            A ^= part == 0 ? r : 0;
            B ^= part == 1 ? r : 0;
            C ^= part == 2 ? r : 0;
        }
    }
}

__device__ __forceinline__ uint64_t combine_q64(uint64_t A, uint64_t B, uint64_t C, const StreamArgs &s) {
    const uint64_t M = C ^ A ^ B;  // middle term, degree <= 62
    return reduce_mod_p64(A ^ (M << 32), B ^ (M >> 32), s);
}

}  // namespace qxd
