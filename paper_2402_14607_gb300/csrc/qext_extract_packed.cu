// Extraction from packed words for q = 16 with n_p = 64 (qext_extract's
// default for 16-byte aligned sources): Ext_IP (Definition 3.2) per block of
// Algorithm 1, one block per lane, one copy pipeline per warp.
//
// Each warp walks sub-tiles of 32 consecutive blocks: lane 0 bulk-copies the
// sub-tile's 128-byte blocks of both sources into the warp's shared-memory
// buffer (completion on the warp's mbarrier, bounded wait), every lane reads
// its block, and once every lane holds its last words the next sub-tile's
// copy is issued, overlapping the second half of the arithmetic.  One CTA of
// up to kMaxWarps warps runs per SM; warps are numbered warp-major across the
// CTAs so that every SM gets the same number of warps that take the last
// round's extra sub-tile.  The block computation is Acc16K2 (two Karatsuba
// levels, parities in byte fields; qext_block.cuh).
#include <cuda_runtime.h>

#include <cstdint>

#include "qext_block.cuh"
#include "qext_internal.h"

using namespace qxd;

namespace {

constexpr int kMaxWarps = 16;

// A sub-tile's blocks (128 bytes per source each) arrive by one bulk copy per
// source; lane l reads its block's eight 16-byte chunks starting at chunk
// l mod 8, so a quarter-warp's reads fall on eight distinct bank groups.
// Lanes past the last block of a partial sub-tile compute on stale buffer
// contents and store nothing.
struct PackedArgs {
    StreamArgs s;
    uint64_t nsub;       // sub-tiles of 32 blocks
    uint32_t max_polls;  // bound of every mbarrier wait
    int no_copy;         // test of failure detection: barriers armed, no copy issued
};

constexpr uint32_t kPackedWpb = 32;                 // words per block and source (q = 16, n_p = 64)
constexpr uint32_t kPackedChunks = kPackedWpb / 4;  // 16-byte chunks per block

__global__ void __launch_bounds__(32 * kMaxWarps) extract_packed16_kernel(const PackedArgs a) {
    extern __shared__ __align__(16) uint4 pk[];
    __shared__ __align__(8) uint64_t full[kMaxWarps];
    const StreamArgs &s = a.s;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint4 *const bx = pk + size_t(warp) * 2 * 32 * kPackedChunks, *const by = bx + 32 * kPackedChunks;
    if (lane == 0) {
        mbar_init(&full[warp], 1);
        fence_mbar_init();
    }
    __syncwarp();
    pdl_prologue();

    // warp-major numbering: every CTA (one per SM) gets the same number of
    // warps with the extra sub-tile of the last round
    const uint64_t gwarps = uint64_t(gridDim.x) * nwarps;
    uint64_t t = uint64_t(warp) * gridDim.x + blockIdx.x;
    auto issue = [&](uint64_t tt) {
        const uint64_t b0 = 32 * tt;
        const uint32_t nb = s.nblocks - b0 < 32 ? uint32_t(s.nblocks - b0) : 32u;
        const uint32_t bytes = nb * kPackedWpb * 4u;
        mbar_expect_tx(&full[warp], 2u * bytes);
        if (a.no_copy) return;  // the completion never comes: the wait must give up
        tma_load_1d(bx, s.x + b0 * kPackedWpb, bytes, &full[warp]);
        tma_load_1d(by, s.y + b0 * kPackedWpb, bytes, &full[warp]);
    };
    if (lane == 0 && t < a.nsub) issue(t);
    const uint4 *const px = bx + lane * kPackedChunks, *const py = by + lane * kPackedChunks;
    for (uint32_t k = 0; t < a.nsub; ++k, t += gwarps) {
        const bool ok = mbar_wait_bounded(&full[warp], k & 1u, a.max_polls);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                record_status(s.status, QEXT_E_TIMEOUT);
                if (!a.no_copy) mbar_wait_bounded(&full[warp], k & 1u, a.max_polls);  // let the copy in flight land
            }
            return;
        }
        Acc16K2 acc;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            uint32_t X[16], Y[16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t ch = (uint32_t(4 * g + c) + lane) & (kPackedChunks - 1);
                const uint4 vx = px[ch], vy = py[ch];
                X[4 * c] = vx.x;
                X[4 * c + 1] = vx.y;
                X[4 * c + 2] = vx.z;
                X[4 * c + 3] = vx.w;
                Y[4 * c] = vy.x;
                Y[4 * c + 1] = vy.y;
                Y[4 * c + 2] = vy.z;
                Y[4 * c + 3] = vy.w;
            }
            if (g == 1) {
                // every lane holds its block: the buffer may be refilled
                __syncwarp();
                if (lane == 0 && t + gwarps < a.nsub) issue(t + gwarps);
            }
            slice<16>(X);
            slice<16>(Y);
            acc.add(X, Y);
        }
        uint64_t v = reduce_mod_p<16>(acc.unreduced(s), s) & mask_m(s.m);
        if (32 * t + lane >= s.nblocks) v = 0;
        store_warp(v, 32 * t, s.nblocks, s.m, s.out);
    }
}

int launch_packed16(const StreamArgs &s, cudaStream_t st, uint32_t flags) {
    static qext::DeviceSlots attr_set, smem_optin;
    const int dev = qext::current_device();
    if (dev < 0) return QEXT_E_CUDA;
    const int sms = qext::sm_count(dev);
    if (sms <= 0) return QEXT_E_CUDA;
    const int optin = smem_optin.get(dev, [dev] {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess ? v : 0;
    });
    if (optin <= 0) return QEXT_E_CUDA;
    const size_t per_warp = size_t(2) * 32 * kPackedChunks * sizeof(uint4);
    const size_t fit = (size_t(optin) - 1024) / per_warp;
    const int W = int(fit < size_t(kMaxWarps) ? fit : size_t(kMaxWarps));
    if (attr_set.get(dev, [optin] {
            return cudaFuncSetAttribute(extract_packed16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        optin - 1024) == cudaSuccess ? 1 : 0;
        }) <= 0)
        return QEXT_E_CUDA;
    PackedArgs a;
    a.s = s;
    a.nsub = (s.nblocks + 31) / 32;
    a.no_copy = (flags & QEXT_F_TEST_TIMEOUT) ? 1 : 0;
    a.max_polls = a.no_copy ? 256u : kMaxPolls;
    const uint64_t ctas = (a.nsub + W - 1) / W;
    const int grid = int(ctas < uint64_t(sms) ? ctas : uint64_t(sms));
    return qext::launch_pdl(extract_packed16_kernel, grid, 32 * W, size_t(W) * per_warp, st, a);
}

}  // namespace

namespace qext {

int launch_extract_packed16(const StreamArgs &s, qext_cuda_stream stream, uint32_t flags) {
    if (s.nblocks == 0) return QEXT_OK;
    if (s.wpb != kPackedWpb) return QEXT_E_UNSUPPORTED;
    return launch_packed16(s, reinterpret_cast<cudaStream_t>(stream), flags);
}

}  // namespace qext
