// Extraction straight from raw b-bit ADC samples (qext_extract_samples) for
// q = 4 and q = 16 with n_p = 64: Ext_IP (Definition 3.2) per block of
// Algorithm 1, one block per thread, with per-warp copy pipelines.
//
// Every warp runs its own pipeline over sub-tiles of R rows of 32 consecutive
// blocks (one block per lane and row; R = 4 for q = 4 so that copies stay
// large, else 1).  Lane 0 copies the sub-tile's raw samples, as whole
// periods of 8 samples (16 bytes), into the warp's shared-memory buffer with
// two 1-D TMA bulk copies that complete on the warp's mbarrier.  Each lane
// then reads its own block's periods from shared memory and packs them into
// stream words in registers (sample s at stream bits [s*b, (s+1)*b), LSB
// first): no packed copy in shared memory and no CTA-wide barrier.  With one
// buffer per warp, the next sub-tile's copy is issued as soon as every lane
// has read its last period, so the copy overlaps the second half of the
// arithmetic.  With two buffers (QEXT_F_RAW_PREFETCH), it is issued one whole
// sub-tile ahead.
//
// Block layout.  Block l is stream words [l*wpb, (l+1)*wpb), wpb = 2q.  A
// period yields WP words (b = 8: 2, b = 12: 3, b = 16: 4).  For b = 8 and 16
// a block is a whole number of periods.  For b = 12 (2q = 2 mod 3) a block is
// (2q-2)/3 whole periods plus two edge words, taken from the period before
// the whole ones (head) and the one after them (tail).  The order of words
// inside a block is free: the Gram-diagonal parities sum over slots, and x
// and y use the same order.  So group g (q words, 32 elements) is any half of
// the whole periods plus edge word g, and each lane reads its periods in a
// lane-rotated order that keeps a quarter-warp's 16-byte reads on distinct
// bank groups.
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_block.cuh"
#include "qext_internal.h"

using namespace qxd;

namespace {

// Warps per CTA, each an independent pipeline: q = 16 runs one CTA of up to
// kMaxWarps warps per SM (as many as the shared-memory buffers allow), q = 4
// several CTAs of kSmallWarps.
constexpr int kMaxWarps = 16;
constexpr int kSmallWarps = 4;

template <int Q, int B>
struct RawLayout {
    static constexpr int WP = PeriodOf<B>::kWords;
    static constexpr int WPB = 2 * Q;  // words per block (n_p = 64)
    // whole periods per block, per group, and how many of them rotate
    static constexpr int NPB = B == 12 ? (WPB - 2) / 3 : WPB / WP;
    static constexpr int NPG = NPB / 2;
    static constexpr int NR = NPB >= 16 ? 16 : NPB >= 8 ? 8 : NPB >= 4 ? 4 : NPB >= 2 ? 2 : 1;
    static_assert(B != 12 || (WPB % 3 == 2 && 3 * NPG + 1 == Q), "b = 12 layout needs 2q = 2 mod 3");
    static_assert(B == 12 || WP * NPG == Q, "whole periods per group");
    // rows of 32 blocks per sub-tile: small blocks take several rows so
    // that each bulk copy stays large
    static constexpr uint32_t kRows = Q == 4 ? 4 : 1;
    // raw periods per source and sub-tile (buffer capacity)
    static constexpr uint32_t kCap = (32u * kRows * WPB + WP - 1) / WP + 1;
};

struct RawArgs {
    StreamArgs s;
    const uint16_t *sx;
    const uint16_t *sy;
    uint64_t nsamples;
    uint64_t nsub;       // sub-tiles of 32 * L::kRows blocks
    uint32_t nbuf;       // raw buffers per warp: 1 or 2
    uint32_t max_polls;  // bound of every mbarrier wait
    int no_copy;         // test of failure detection: barriers armed, no copy issued
};

// Sub-tile t: blocks [32R t, min(32R (t+1), nblocks)) with R = kRows rows of
// 32 blocks, raw periods [p0, p0 + np).
template <int Q, int B>
struct SubTile {
    uint64_t b0;  // first block
    uint64_t p0;
    uint32_t np;
    uint32_t r0;  // words of period p0 before the sub-tile's first word
    bool tma;     // every period lies inside the sample arrays: bulk-copy it
    __device__ __forceinline__ SubTile(const RawArgs &a, uint64_t t) {
        using L = RawLayout<Q, B>;
        b0 = 32 * L::kRows * t;
        const uint64_t b_end = b0 + 32 * L::kRows < a.s.nblocks ? b0 + 32 * L::kRows : a.s.nblocks;
        const uint64_t w = b0 * L::WPB;
        p0 = w / L::WP;
        r0 = uint32_t(w - p0 * L::WP);
        np = uint32_t((b_end * L::WPB - 1) / L::WP - p0 + 1);
        tma = 8 * (p0 + np) <= a.nsamples;
    }
};

template <int Q, int B>
__device__ __forceinline__ void issue_sub(const RawArgs &a, const SubTile<Q, B> &st, uint4 *bx, uint4 *by,
                                          uint64_t *bar) {
    mbar_expect_tx(bar, 32u * st.np);
    if (a.no_copy) return;  // the completion never comes: the wait must give up
    tma_load_1d(bx, a.sx + 8 * st.p0, 16u * st.np, bar);
    tma_load_1d(by, a.sy + 8 * st.p0, 16u * st.np, bar);
}

// Lane rotation of the whole periods: with NR >= 8 and every block starting
// on the same bank group (b = 8, 16) the lane index itself; with fewer
// periods, the lanes that share a bank group spread over the NR rotations;
// for b = 12 the rotation cancels the block's own starting bank group.
template <int Q, int B>
__device__ __forceinline__ uint32_t lane_rotation(uint32_t lane, uint32_t fp_rel) {
    using L = RawLayout<Q, B>;
    if constexpr (B == 12) {
        return (lane - fp_rel) & uint32_t(L::NR - 1);
    } else if constexpr (L::NPB >= 8) {
        return lane & 7u;
    } else {
        return (lane * uint32_t(L::NPB) / 8u) & uint32_t(L::NR - 1);
    }
}

// Whole period number j (0 .. NPB-1) of the block, after rotation.
template <int Q, int B>
__device__ __forceinline__ uint32_t period_of(int j, uint32_t fp_rel, uint32_t rot) {
    using L = RawLayout<Q, B>;
    return fp_rel + (j < L::NR ? ((uint32_t(j) + rot) & uint32_t(L::NR - 1)) : uint32_t(j));
}

// Group G of the block: its whole periods, packed, plus (b = 12) edge word ex / ey.
template <int Q, int B, int G>
__device__ __forceinline__ void raw_group(const uint4 *bx, const uint4 *by, uint32_t fp_rel, uint32_t rot,
                                          uint32_t ex, uint32_t ey, uint32_t (&X)[Q], uint32_t (&Y)[Q]) {
    using L = RawLayout<Q, B>;
    constexpr int WP = L::WP;
#pragma unroll
    for (int jj = 0; jj < L::NPG; ++jj) {
        const uint32_t per = period_of<Q, B>(G * L::NPG + jj, fp_rel, rot);
        uint32_t wx[WP], wy[WP];
        pack_period8<B>(bx[per], wx);
        pack_period8<B>(by[per], wy);
#pragma unroll
        for (int i = 0; i < WP; ++i) {
            X[WP * jj + i] = wx[i];
            Y[WP * jj + i] = wy[i];
        }
    }
    if constexpr (B == 12) {
        X[Q - 1] = ex;
        Y[Q - 1] = ey;
    }
}

// b = 12 edge words: off = (first word of the block) mod 3.
//   off 0: no head word, tail words T0, T1;  off 1: head H1, H2, no tail;
//   off 2: head H2, tail T0.
// Word w of a period is a byte permute of its packed sample pairs w and w+1
// (pack_period8), so the four sample pairs behind the two edge words are
// picked first and only they are packed.
struct EdgeSel {
    uint32_t off, s1, s2;  // off, and the byte-permute selectors of the two edge words
    __device__ __forceinline__ explicit EdgeSel(uint32_t o)
        : off(o), s1(o == 0 ? 0x4210u : o == 1 ? 0x5421u : 0x6542u), s2(o == 0 ? 0x5421u : o == 1 ? 0x6542u : 0x4210u) {}
};

__device__ __forceinline__ void edge_words(uint4 h, uint4 t, const EdgeSel &es, uint32_t &e1, uint32_t &e2) {
    const uint32_t off = es.off;
    const uint32_t u0 = off == 0 ? t.x : off == 1 ? h.y : h.z;
    const uint32_t u1 = off == 0 ? t.y : off == 1 ? h.z : h.w;
    const uint32_t u2 = off == 0 ? t.y : off == 1 ? h.z : t.x;
    const uint32_t u3 = off == 0 ? t.z : off == 1 ? h.w : t.y;
    e1 = __byte_perm(pack_pair12(u0), pack_pair12(u1), es.s1);
    e2 = __byte_perm(pack_pair12(u2), pack_pair12(u3), es.s2);
}

template <int Q, int B>
__global__ void __launch_bounds__(Q == 16 ? 32 * kMaxWarps : 32 * kSmallWarps) extract_raw_kernel(const RawArgs a) {
    using L = RawLayout<Q, B>;
    extern __shared__ __align__(16) uint4 raw[];
    __shared__ __align__(8) uint64_t full[kMaxWarps][2];
    const StreamArgs &s = a.s;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint4 *const buf0 = raw + size_t(warp) * a.nbuf * 2 * L::kCap;  // [x periods | y periods] per buffer
    uint4 *const buf1 = buf0 + (a.nbuf > 1 ? 2 * L::kCap : 0);
    if (lane == 0) {
        mbar_init(&full[warp][0], 1);
        mbar_init(&full[warp][1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    pdl_prologue();

    // warp-major numbering: every CTA (one per SM at q = 16) gets the same
    // number of warps with the extra sub-tile of the last round
    const uint64_t gwarps = uint64_t(gridDim.x) * nwarps;
    uint64_t t = uint64_t(warp) * gridDim.x + blockIdx.x;
    uint32_t uses0 = 0, uses1 = 0;  // completed phases of full[warp][0], [1]
    bool next_issued = false;       // lane 0: the next sub-tile's copy is in flight
    if (t < a.nsub && lane == 0) {
        const SubTile<Q, B> st(a, t);
        if (st.tma) {
            issue_sub(a, st, buf0, buf0 + L::kCap, &full[warp][0]);
            next_issued = true;
        }
    }
    for (uint32_t k = 0; t < a.nsub; ++k, t += gwarps) {
        const int b = a.nbuf > 1 ? int(k & 1u) : 0;
        uint4 *const bx = b ? buf1 : buf0, *const by = bx + L::kCap;
        const SubTile<Q, B> st(a, t);
        const uint64_t tn = t + gwarps;
        if (a.nbuf > 1 && lane == 0) {
            // the other buffer was last read in iteration k-1, which ended with __syncwarp
            next_issued = false;
            if (tn < a.nsub) {
                const SubTile<Q, B> sn(a, tn);
                if (sn.tma) {
                    uint4 *const nx = b ? buf0 : buf1;
                    issue_sub(a, sn, nx, nx + L::kCap, &full[warp][b ^ 1]);
                    next_issued = true;
                }
            }
        }
        if (st.tma) {
            const uint32_t use = b ? uses1++ : uses0++;
            const bool ok = mbar_wait_bounded(&full[warp][b], use & 1u, a.max_polls);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    record_status(s.status, QEXT_E_TIMEOUT);
                    // give the copies in flight a bounded chance to land
                    mbar_wait_bounded(&full[warp][b], use & 1u, a.max_polls);
                    if (a.nbuf > 1 && next_issued)
                        mbar_wait_bounded(&full[warp][b ^ 1], (b ? uses0 : uses1) & 1u, a.max_polls);
                }
                return;
            }
        } else {
            // the stream's last sub-tiles: bounded plain loads (samples past
            // the arrays read as 0); no bulk copy follows into this buffer
            __syncwarp();
            const uint64_t left = a.nsamples > 8 * st.p0 ? a.nsamples - 8 * st.p0 : 0;
            const uint32_t avail = left > 0xFFFFFFF0ull ? 0xFFFFFFF0u : uint32_t(left);
            for (uint32_t j = lane; j < st.np; j += 32) {
                bx[j] = load_period8(a.sx + 8 * st.p0, 8 * j, avail);
                by[j] = load_period8(a.sy + 8 * st.p0, 8 * j, avail);
            }
            fence_proxy_async_smem();
            __syncwarp();
        }

        // rows of 32 blocks, one block per lane (lanes past the stream redo
        // the last block, unstored)
        const uint64_t row0 = uint64_t(L::kRows) * t;
        const uint64_t rows_left = (s.nblocks - 32 * row0 + 31) / 32;
        const uint32_t nrows = rows_left < L::kRows ? uint32_t(rows_left) : L::kRows;
        for (uint32_t r = 0; r < nrows; ++r) {
            const uint64_t base = 32 * (row0 + r), blk = base + lane;
            const uint64_t lb = blk < s.nblocks ? blk : s.nblocks - 1;
            // the block's first word, counted from the start of period p0
            const uint32_t w_rel = st.r0 + uint32_t(lb - st.b0) * uint32_t(L::WPB);
            const uint32_t fp_rel = (w_rel + L::WP - 1) / L::WP;  // first whole period
            const uint32_t rot = lane_rotation<Q, B>(lane, fp_rel);
            uint32_t ex1 = 0, ey1 = 0, ex2 = 0, ey2 = 0;
            if constexpr (B == 12) {
                const uint32_t off = w_rel % 3;
                const uint32_t hp = off ? fp_rel - 1 : fp_rel;             // head period (if any)
                const uint32_t tp = off != 1 ? fp_rel + L::NPB : fp_rel;  // tail period (if any)
                const EdgeSel es(off);
                edge_words(bx[hp], bx[tp], es, ex1, ex2);
                edge_words(by[hp], by[tp], es, ey1, ey2);
            }
            BlockAcc<Q> acc;
            {
                uint32_t X[Q], Y[Q];
                raw_group<Q, B, 0>(bx, by, fp_rel, rot, ex1, ey1, X, Y);
                slice<Q>(X);
                slice<Q>(Y);
                acc.add(X, Y);
            }
            {
                uint32_t X[Q], Y[Q];
                raw_group<Q, B, 1>(bx, by, fp_rel, rot, ex2, ey2, X, Y);
                if (r + 1 == nrows) {
                    // every lane has read its periods: the buffer may be refilled
                    __syncwarp();
                    if (a.nbuf == 1 && lane == 0) {
                        next_issued = false;
                        if (tn < a.nsub) {
                            const SubTile<Q, B> sn(a, tn);
                            if (sn.tma) {
                                issue_sub(a, sn, buf0, buf0 + L::kCap, &full[warp][0]);
                                next_issued = true;
                            }
                        }
                    }
                }
                slice<Q>(X);
                slice<Q>(Y);
                acc.add(X, Y);
            }
            uint64_t v = reduce_mod_p<Q>(acc.unreduced(s), s) & mask_m(s.m);
            if (blk >= s.nblocks) v = 0;
            store_warp(v, base, s.nblocks, s.m, s.out);
        }
    }
    (void)next_issued;
}

template <int Q, int B>
int launch_raw(const StreamArgs &s, const uint16_t *sx, const uint16_t *sy, uint64_t nsamples, cudaStream_t st,
               uint32_t flags) {
    using L = RawLayout<Q, B>;
    if (s.wpb != uint32_t(L::WPB)) return QEXT_E_UNSUPPORTED;
    static qext::DeviceSlots attr_set, occ[2], smem_optin;  // per device; occupancy by buffers per warp
    const int dev = qext::current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int sms = qext::sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    const int optin = smem_optin.get(dev, [dev] {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess ? v : 0;
    });
    if (optin <= 0) return QEXT_E_CUDA;
    const uint32_t nbuf = (flags & QEXT_F_RAW_PREFETCH) ? 2u : 1u;
    const size_t per_warp = size_t(nbuf) * 2 * L::kCap * sizeof(uint4);
    // warps per CTA: q = 16 fills one CTA per SM (as many warps as the
    // buffers allow), q = 4 keeps small CTAs
    size_t fit = (size_t(optin) - 1024) / per_warp;
    int W = Q == 16 ? int(fit < size_t(kMaxWarps) ? fit : size_t(kMaxWarps)) : kSmallWarps;
    if (W < 1) return QEXT_E_UNSUPPORTED;
    const size_t smem = size_t(W) * per_warp;
    if (attr_set.get(dev, [optin] {
            return cudaFuncSetAttribute(extract_raw_kernel<Q, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        optin - 1024) == cudaSuccess ? 1 : 0;
        }) <= 0)
        return QEXT_E_CUDA;
    int o = 1;
    if (Q != 16) {
        o = occ[nbuf - 1].get(dev, [&] {
            int v = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, extract_raw_kernel<Q, B>, 32 * W, smem) !=
                cudaSuccess)
                return 0;
            return v < 1 ? 1 : v;
        });
        if (o <= 0) return QEXT_E_CUDA;
    }
    RawArgs a;
    a.s = s;
    a.sx = sx;
    a.sy = sy;
    a.nsamples = nsamples;
    a.nsub = (s.nblocks + 32 * L::kRows - 1) / (32 * L::kRows);
    a.nbuf = nbuf;
    a.no_copy = (flags & QEXT_F_TEST_TIMEOUT) ? 1 : 0;
    a.max_polls = a.no_copy ? 256u : kMaxPolls;
    const uint64_t ctas = (a.nsub + W - 1) / W, cap = uint64_t(sms) * o;
    const int grid = int(ctas < cap ? ctas : cap);
    return qext::launch_pdl(extract_raw_kernel<Q, B>, grid, 32 * W, smem, st, a);
}

template <int Q>
int launch_raw_q(uint32_t b, const StreamArgs &s, const uint16_t *sx, const uint16_t *sy, uint64_t nsamples,
                 cudaStream_t st, uint32_t flags) {
    switch (b) {
        case 8: return launch_raw<Q, 8>(s, sx, sy, nsamples, st, flags);
        case 12: return launch_raw<Q, 12>(s, sx, sy, nsamples, st, flags);
        case 16: return launch_raw<Q, 16>(s, sx, sy, nsamples, st, flags);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace

namespace qext {

int launch_raw_samples(uint32_t q, uint32_t b, const StreamArgs &s, const uint16_t *sx, const uint16_t *sy,
                       uint64_t nsamples, qext_cuda_stream stream, uint32_t flags) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (s.nblocks == 0) return QEXT_OK;
    switch (q) {
        case 4: return launch_raw_q<4>(b, s, sx, sy, nsamples, st, flags);
        case 16: return launch_raw_q<16>(b, s, sx, sy, nsamples, st, flags);
        default: return QEXT_E_UNSUPPORTED;
    }
}

}  // namespace qext
