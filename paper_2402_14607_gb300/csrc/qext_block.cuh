// Per-block compute of Ext_IP (Definition 3.2) from a block's words, shared
// by the extraction kernels, plus the raw-sample packing of the fused ingest.
// See qext_device.cuh for the sliced GF(2) formulation.
#pragma once

#include "qext_device.cuh"

namespace qxd {

__device__ __forceinline__ uint4 lds4(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }

// ---------------------------------------------------------------------------
// Accumulator of one block's sliced Gram diagonals, q <= 32.
// ---------------------------------------------------------------------------
// One Karatsuba level over the element bits (q = 16 in kernels whose register
// budget is tight), with low half L (bits 0..7), high half H (8..15) and sum
// S = L + H of each element:
//     x y = A + t^8 (A + B + C) + t^16 B,   A = LxLy, B = HxHy, C = SxSy,
//         = D + t^8 D + t^8 C,             D = A + t^8 B.
// So A and B accumulate into one array D (A at offset 0, B at offset 8; 23
// diagonals) and C into its own (15): 38 accumulators and parities.
template <int Q>
struct Acc {
    static constexpr bool kKaratsuba = Q == 16;
    static constexpr int NA = kKaratsuba ? 38 : 2 * Q - 1;
    uint32_t a[NA];
    __device__ __forceinline__ Acc() {
#pragma unroll
        for (int i = 0; i < NA; ++i) a[i] = 0;
    }
    // Sliced group of 32 elements: X[j], Y[j] = bit j of the 32 elements.
    __device__ __forceinline__ void add(uint32_t (&X)[Q], uint32_t (&Y)[Q]) {
        if constexpr (kKaratsuba) {
            uint32_t *D = a, *C = a + 23;
            uint32_t XS[8], YS[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                XS[j] = X[j] ^ X[j + 8];
                YS[j] = Y[j] ^ Y[j + 8];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int l = 0; l < 8; ++l) {
                    D[j + l] = lop_and_xor(X[j], Y[l], D[j + l]);
                    D[j + l + 8] = lop_and_xor(X[j + 8], Y[l + 8], D[j + l + 8]);
                    C[j + l] = lop_and_xor(XS[j], YS[l], C[j + l]);
                }
        } else {
            gram_diagonals<Q, Q>(X, Y, a);
        }
    }
    // z (2q-1 bits) = parities of the Gram diagonals
    __device__ __forceinline__ uint64_t unreduced(const StreamArgs &) {
        if constexpr (kKaratsuba) {
            // z = D + t^8 D + t^8 C on the parities (parity is linear): rD
            // holds D's 23 parity bits in bits 9..31, rC C's 15 in bits 17..31
            const uint32_t rD = parity_bits32_top<23>(a), rC = parity_bits32_top<15>(a + 23);
            return lop_xor3(rD >> 9, rD >> 1, rC >> 9);
        } else {
            return parity_bits64<2 * Q - 1>(a);
        }
    }
};

// ---------------------------------------------------------------------------
// q = 16 with two Karatsuba levels and byte-field parity sums (the default
// wherever 128 registers per thread are available).
// ---------------------------------------------------------------------------
// The second level splits every 8 x 8 product U V (U = U0 + t^4 U1) into
//     U V = E + t^4 E + t^4 M,   E = U0 V0 + t^4 U1 V1,   M = (U0 + U1)(V0 + V1),
// three 4 x 4 products.  With the first level's D = A + t^8 B this gives
//     D = F + t^4 F + t^4 G,     F = E_A + t^8 E_B (19),  G = M_A + t^8 M_B (15),
//     C = E_C + t^4 E_C + t^4 M_C,                        E_C (11), M_C (7),
//     x y = D + t^8 D + t^8 C,
// 9 x 16 = 144 AND-XORs and 40 operand sums per group of 32 elements
// (instead of 192 and 16) into 52 accumulators.  Their parities are linear
// combinations, taken in byte fields: the popcounts of four consecutive
// accumulators are packed into one word by IMADs (w = w * 256 + popc, every
// field <= 32), so t^4 and t^8 are shifts by one and two whole words and sums
// of three fields stay below 256; the fields' low bits are masked between
// combination steps, and the four parity bits of a word gather into a nibble
// by one multiply: ((w & 0x01010101) * 0x01020408) >> 24.  The field steps
// run on the FMA pipe, next to the products and transposes that fill the
// ALU pipe.
struct Acc16K2 {
    uint32_t F[19], G[15], E[11], M[7];
    __device__ __forceinline__ Acc16K2() {
#pragma unroll
        for (int i = 0; i < 19; ++i) F[i] = 0;
#pragma unroll
        for (int i = 0; i < 15; ++i) G[i] = 0;
#pragma unroll
        for (int i = 0; i < 11; ++i) E[i] = 0;
#pragma unroll
        for (int i = 0; i < 7; ++i) M[i] = 0;
    }
    // acc[j + l] ^= u[j] & v[l], 4 x 4
    __device__ __forceinline__ static void mul4(const uint32_t *u, const uint32_t *v, uint32_t *acc) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int l = 0; l < 4; ++l) acc[j + l] = lop_and_xor(u[j], v[l], acc[j + l]);
    }
    // one 8 x 8 product: E-part into e (11 diagonals), M-part into m (7)
    __device__ __forceinline__ static void mul8(const uint32_t *U, const uint32_t *V, uint32_t *e, uint32_t *m) {
        uint32_t us[4], vs[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            us[j] = U[j] ^ U[j + 4];
            vs[j] = V[j] ^ V[j + 4];
        }
        mul4(U, V, e);
        mul4(U + 4, V + 4, e + 4);
        mul4(us, vs, m);
    }
    // Sliced group of 32 elements: X[j], Y[j] = bit j of the 32 elements.
    __device__ __forceinline__ void add(uint32_t (&X)[16], uint32_t (&Y)[16]) {
        uint32_t XS[8], YS[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            XS[j] = X[j] ^ X[j + 8];
            YS[j] = Y[j] ^ Y[j + 8];
        }
        mul8(X, Y, F, G);              // A = L L
        mul8(X + 8, Y + 8, F + 8, G + 8);  // B = H H, at t^8
        mul8(XS, YS, E, M);            // C = S S
    }
    // popcounts of acc[0 .. N) as byte fields of ceil(N / 4) words
    template <int N, int W>
    __device__ __forceinline__ static void fields(const uint32_t *acc, uint32_t (&w)[W], const StreamArgs &s) {
        static_assert(W == (N + 3) / 4, "one word per four fields");
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int top = (4 * i + 3 < N ? 4 * i + 3 : N - 1);
            uint32_t v = __popc(acc[top]);
#pragma unroll
            for (int f = top - 1; f >= 4 * i; --f) v = v * s.byte_mul + uint32_t(__popc(acc[f]));
            w[i] = v;
        }
    }
    // z (31 bits), unreduced
    __device__ __forceinline__ uint64_t unreduced(const StreamArgs &s) const {
        constexpr uint32_t ONE = 0x01010101u;
        uint32_t WF[5], WG[4], WE[3], WM[2];
        fields<19, 5>(F, WF, s);
        fields<15, 4>(G, WG, s);
        fields<11, 3>(E, WE, s);
        fields<7, 2>(M, WM, s);
        uint32_t WD[6], WC[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) {  // D = F + t^4 F + t^4 G
            uint32_t v = i < 5 ? WF[i] : 0u;
            if (i >= 1) v += WF[i - 1] + (i - 1 < 4 ? WG[i - 1] : 0u);
            WD[i] = v & ONE;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // C = E + t^4 E + t^4 M
            uint32_t v = i < 3 ? WE[i] : 0u;
            if (i >= 1) v += WE[i - 1] + (i - 1 < 2 ? WM[i - 1] : 0u);
            WC[i] = v & ONE;
        }
        uint32_t z = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {  // z = D + t^8 D + t^8 C
            uint32_t v = i < 6 ? WD[i] : 0u;
            if (i >= 2) v += WD[i - 2] + (i - 2 < 4 ? WC[i - 2] : 0u);
            const uint32_t nib = ((v & ONE) * 0x01020408u) >> 24;
            z = nib * s.nib_mul[i] + z;
        }
        return z;
    }
};

template <int Q>
struct BlockAccT {
    using type = Acc<Q>;
};
template <>
struct BlockAccT<16> {
    using type = Acc16K2;
};
// The accumulator of one block at field degree Q.
template <int Q>
using BlockAcc = typename BlockAccT<Q>::type;

// One block, q <= 32, from a block's words xs / ys (shared or global memory).
// With vec, the block's 16-byte chunks are read starting at chunk rot.
template <int Q>
__device__ __forceinline__ uint64_t block_small_q(const uint32_t *xs, const uint32_t *ys, uint32_t wpb, int vec,
                                                  uint32_t rot, const StreamArgs &s) {
    BlockAcc<Q> acc;
    if constexpr (Q >= 4) {
        if (vec && wpb == 2 * Q) {
            // n_p = 64: two groups of 32 elements, 2Q/4 chunks, fully unrolled
            constexpr uint32_t NCH = Q / 2;
            const uint32_t r0 = rot & (NCH - 1);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint32_t X[Q], Y[Q];
#pragma unroll
                for (int c = 0; c < Q / 4; ++c) {
                    const uint32_t ch = (uint32_t(g * (Q / 4) + c) + r0) & (NCH - 1);
                    const uint4 vx = lds4(xs + 4 * ch), vy = lds4(ys + 4 * ch);
                    X[4 * c] = vx.x;
                    X[4 * c + 1] = vx.y;
                    X[4 * c + 2] = vx.z;
                    X[4 * c + 3] = vx.w;
                    Y[4 * c] = vy.x;
                    Y[4 * c + 1] = vy.y;
                    Y[4 * c + 2] = vy.z;
                    Y[4 * c + 3] = vy.w;
                }
                slice<Q>(X);
                slice<Q>(Y);
                acc.add(X, Y);
            }
            return reduce_mod_p<Q>(acc.unreduced(s), s);
        }
    }
    if (vec) {
        const uint32_t nch = wpb >> 2;
        const uint32_t r0 = rot % nch;
        if constexpr (Q >= 4) {
            constexpr int CPG = Q / 4;  // chunks per group
            for (uint32_t g = 0; g < nch; g += CPG) {
                uint32_t X[Q], Y[Q];
#pragma unroll
                for (int c = 0; c < CPG; ++c) {
                    uint4 vx = make_uint4(0, 0, 0, 0), vy = vx;
                    if (g + c < nch) {
                        uint32_t ch = g + c + r0;
                        ch = ch >= nch ? ch - nch : ch;
                        vx = lds4(xs + 4 * ch);
                        vy = lds4(ys + 4 * ch);
                    }
                    X[4 * c] = vx.x;
                    X[4 * c + 1] = vx.y;
                    X[4 * c + 2] = vx.z;
                    X[4 * c + 3] = vx.w;
                    Y[4 * c] = vy.x;
                    Y[4 * c + 1] = vy.y;
                    Y[4 * c + 2] = vy.z;
                    Y[4 * c + 3] = vy.w;
                }
                slice<Q>(X);
                slice<Q>(Y);
                acc.add(X, Y);
            }
        } else {
            for (uint32_t c = 0; c < nch; ++c) {
                uint32_t ch = c + r0;
                ch = ch >= nch ? ch - nch : ch;
                const uint4 vx = lds4(xs + 4 * ch), vy = lds4(ys + 4 * ch);
                const uint32_t wx[4] = {vx.x, vx.y, vx.z, vx.w}, wy[4] = {vy.x, vy.y, vy.z, vy.w};
#pragma unroll
                for (int g = 0; g < 4 / Q; ++g) {
                    uint32_t X[Q], Y[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        X[i] = wx[g * Q + i];
                        Y[i] = wy[g * Q + i];
                    }
                    slice<Q>(X);
                    slice<Q>(Y);
                    acc.add(X, Y);
                }
            }
        }
    } else {
        for (uint32_t g0 = 0; g0 < wpb; g0 += Q) {
            uint32_t X[Q], Y[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                X[i] = g0 + i < wpb ? xs[g0 + i] : 0u;
                Y[i] = g0 + i < wpb ? ys[g0 + i] : 0u;
            }
            slice<Q>(X);
            slice<Q>(Y);
            acc.add(X, Y);
        }
    }
    return reduce_mod_p<Q>(acc.unreduced(s), s);
}

// ---------------------------------------------------------------------------
// Fused ingest: pack the raw b-bit samples behind stream words [w0, w0 + nw)
// straight into shared memory (sample s at stream bits [s*b, (s+1)*b), LSB
// first; samples past nsamples read as 0).  One period per thread and step:
//   b = 12: 8 samples (16 bytes) -> 3 words; b = 8: 4 samples -> 1 word;
//   b = 16: 2 samples -> 1 word.
// ---------------------------------------------------------------------------
// 8 raw samples (16 bytes) at smp[s0 .. s0+8); samples at or past `avail`
// read as 0.
__device__ __forceinline__ uint4 load_period8(const uint16_t *__restrict__ smp, uint32_t s0, uint32_t avail) {
    if (s0 + 8 <= avail) return __ldg(reinterpret_cast<const uint4 *>(smp + s0));
    uint32_t q[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t lo = s0 + 2 * j < avail ? __ldg(smp + s0 + 2 * j) : 0u;
        const uint32_t hi = s0 + 2 * j + 1 < avail ? __ldg(smp + s0 + 2 * j + 1) : 0u;
        q[j] = lo | (hi << 16);
    }
    return make_uint4(q[0], q[1], q[2], q[3]);
}

// The words a period of 8 samples yields: b = 12 -> 3 words, b = 8 -> 2 words
// (two periods of 4), b = 16 -> 4 words.
template <int B>
struct PeriodOf {
    static constexpr int kWords = B == 12 ? 3 : B == 8 ? 2 : 4;
};

// 12-bit sample pair q = s | t << 16 -> bits 0..23 of s | t << 12: bits
// 0..11 from q, bits 12..23 from q >> 4.  The bits of s and t above 12 fall
// outside bits 0..23 (t's land in byte 3), which the byte permutes below
// never take.
__device__ __forceinline__ uint32_t pack_pair12(uint32_t q) {
    return lop_select(q, __umulhi(q, 1u << 28), 0x00000FFFu);
}

template <int B>
__device__ __forceinline__ void pack_period8(const uint4 v, uint32_t (&w)[PeriodOf<B>::kWords]) {
    if constexpr (B == 12) {
        // word j = bytes of the packed pairs P_j, P_j+1 (bytes 0..2 of each)
        const uint32_t P[4] = {pack_pair12(v.x), pack_pair12(v.y), pack_pair12(v.z), pack_pair12(v.w)};
        w[0] = __byte_perm(P[0], P[1], 0x4210);
        w[1] = __byte_perm(P[1], P[2], 0x5421);
        w[2] = __byte_perm(P[2], P[3], 0x6542);
    } else if constexpr (B == 8) {
        w[0] = __byte_perm(v.x, v.y, 0x6420);  // low bytes of four samples
        w[1] = __byte_perm(v.z, v.w, 0x6420);
    } else {
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    }
}

// Fused ingest: pack the raw b-bit samples behind stream words [w0, w0 + nw)
// of both sources straight into shared memory (sample s at stream bits
// [s*b, (s+1)*b), LSB first; samples past nsamples read as 0).  Work comes in
// periods of 8 samples; each thread loads kBatch periods of x and of y before
// packing any, so that many 16-byte loads are in flight.  Indices are local to
// the tile (32-bit); only the first and last period can straddle the tile.
template <int B>
__device__ __forceinline__ void pack_tile(const uint16_t *__restrict__ sx, const uint16_t *__restrict__ sy,
                                          uint64_t nsamples, uint64_t w0, uint32_t nw, uint32_t *__restrict__ dx,
                                          uint32_t *__restrict__ dy, uint32_t tid, uint32_t nthreads) {
    constexpr uint32_t WP = PeriodOf<B>::kWords;  // words per period of 8 samples
    constexpr int kBatch = 4;
    const uint64_t p0 = w0 / WP;
    const uint32_t phi = uint32_t(w0 - p0 * WP);  // tile words that precede w0 in period p0
    const uint32_t nper = (phi + nw + WP - 1) / WP;
    const uint64_t s_base = 8 * p0;
    const uint64_t left = nsamples > s_base ? nsamples - s_base : 0;
    const uint32_t avail = left > 0xFFFFFFF0ull ? 0xFFFFFFF0u : uint32_t(left);
    const uint16_t *bx = sx + s_base, *by = sy + s_base;
    for (uint32_t jb = tid; jb < nper; jb += kBatch * nthreads) {
        uint4 vx[kBatch], vy[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const uint32_t j = jb + k * nthreads;
            vx[k] = vy[k] = make_uint4(0, 0, 0, 0);
            if (j < nper) {
                vx[k] = load_period8(bx, 8 * j, avail);
                vy[k] = load_period8(by, 8 * j, avail);
            }
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const uint32_t j = jb + k * nthreads;
            if (j < nper) {
                uint32_t wx[WP], wy[WP];
                pack_period8<B>(vx[k], wx);
                pack_period8<B>(vy[k], wy);
                const uint32_t lw = WP * j - phi;  // tile word of the period's first word (wraps if < 0)
                if (j > 0 && j + 1 < nper) {
#pragma unroll
                    for (uint32_t i = 0; i < WP; ++i) {
                        dx[lw + i] = wx[i];
                        dy[lw + i] = wy[i];
                    }
                } else {
#pragma unroll
                    for (uint32_t i = 0; i < WP; ++i)
                        if (lw + i < nw) {
                            dx[lw + i] = wx[i];
                            dy[lw + i] = wy[i];
                        }
                }
            }
        }
    }
}

// Fused ingest from a raw-sample tile already in shared memory: the periods
// of 8 samples covering stream words [w0, w0 + nw) of each source (raw_x[j],
// raw_y[j] = period p0 + j) are packed IN PLACE, the packed words landing over
// the front of the same buffers (tile word i at raw_x[0..], raw_y[0..]).
// Rounds of kPer periods per thread: every thread loads its round's periods,
// the CTA synchronises, then stores.  A round's stores reach at most byte
// (WP*4) * (periods so far), which never passes the raw bytes already loaded
// (WP*4 <= 16 bytes per period), so no period is overwritten before it is read.
template <int B>
__device__ __forceinline__ void pack_tile_in_place(uint4 *raw_x, uint4 *raw_y, uint32_t phi, uint32_t nw,
                                                   uint32_t tid, uint32_t nthreads) {
    constexpr uint32_t WP = PeriodOf<B>::kWords;
    constexpr int kPer = 2;
    const uint32_t nper = (phi + nw + WP - 1) / WP;
    uint32_t *dx = reinterpret_cast<uint32_t *>(raw_x), *dy = reinterpret_cast<uint32_t *>(raw_y);
    for (uint32_t base = 0; base < nper; base += kPer * nthreads) {
        uint4 vx[kPer], vy[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const uint32_t j = base + tid + r * nthreads;
            if (j < nper) {
                vx[r] = raw_x[j];
                vy[r] = raw_y[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const uint32_t j = base + tid + r * nthreads;
            if (j < nper) {
                uint32_t wx[WP], wy[WP];
                pack_period8<B>(vx[r], wx);
                pack_period8<B>(vy[r], wy);
                const uint32_t lw = WP * j - phi;
#pragma unroll
                for (uint32_t i = 0; i < WP; ++i)
                    if (lw + i < nw) {
                        dx[lw + i] = wx[i];
                        dy[lw + i] = wy[i];
                    }
            }
        }
    }
    fence_proxy_async_smem();  // the buffer is refilled by a bulk copy after this tile
    __syncthreads();
}

}  // namespace qxd
