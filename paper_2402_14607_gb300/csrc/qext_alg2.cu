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
// block l is k_l = q_l / 16 consecutive units (q_l <= 2048: k_l <= 128).
// The product Z^(l) = sum_i x_i y_i is taken unit by unit: with S_u = the
// slices of unit u over a group of 32 elements (slice<16>, elements i and
// i + 16 in word i: element e in slot e), each element is x = sum_u X_u w^u
// (w = t^16) and the generalised Karatsuba formula (Weimerskirch and Paar,
// 2006) gives
//     x y = sum_u P_uu w^2u + sum_{u<v} (P_uv + P_uu + P_vv) w^(u+v),
//     P_uv = (X_u + X_v)(Y_u + Y_v),
// k_l (k_l + 1) / 2 unit products instead of k_l^2.  Each is a 16 x 16 sliced
// Gram product whose 31 diagonal parities (parities are linear: XORed over
// groups) are placed at bit 16 (u + v) of the block's unreduced sum, P_uv for
// u < v directly; P_uu lands at every offset o = u + w, w < k_l, so the P_uu
// are collected in a per-block array D and placed by the second launch as
// window XORs, W_o = XOR of D_u over max(0, o - k_l + 1) <= u <= min(o, k_l - 1)
// (prefix XORs).  Work items of at most kItemProducts unit products of one
// (block, group) run as CTAs of one launch (alg2_products_kernel): each slices
// the group's 2 k_l units into shared memory, computes its products, XORs the
// parities into shared sums and those into the block's arrays in global
// memory.  A second launch (alg2_reduce_kernel, one CTA per block) adds the
// P_uu windows, reduces the sum mod P_{q_l} word-parallel (the part at and
// above x^{q_l} folded back by the taps until none is left) and writes the
// block's k_l output units.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
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
    uint64_t zoff;     // first word of the block's unreduced sum (k + 1 words), then D (k words)
};

// A work item: unit products p in [p0, p1) of one group of one block (p
// counts the pairs u <= v row by row: row u holds v = u .. k - 1).
struct Alg2Item {
    uint32_t block;
    uint32_t group;
    uint32_t p0, p1;
};

struct qext_alg2_plan {
    double delta;
    uint32_t b, q1, Delta, n_p, max_blocks;
    std::vector<Alg2Block> blocks;
    std::vector<Alg2Item> items;
    std::vector<uint32_t> item_prefix;  // items of blocks < l
    uint64_t zwords = 0;
    std::mutex mu;                      // the device tables, made on first use
    Alg2Block *d_blocks = nullptr;
    Alg2Item *d_items = nullptr;
    uint32_t *d_z = nullptr;
    int device = -1;
};

namespace {

constexpr int kAlg2Threads = 256;
constexpr uint32_t kMaxUnits = 128;       // q_l <= 2048
constexpr uint32_t kItemProducts = 1024;  // unit products per work item
constexpr uint32_t kRow = 20;             // words per sliced unit in shared memory

__global__ void __launch_bounds__(kAlg2Threads)
    alg2_products_kernel(const Alg2Item *__restrict__ items, const Alg2Block *__restrict__ table, uint32_t n_p,
                         const uint16_t *__restrict__ x, const uint16_t *__restrict__ y, uint32_t *__restrict__ zg,
                         const StreamArgs pm) {  // pm: the parity-assembly multipliers only
    // sliced units of the group; rows of 20 words, so that a quarter-warp's
    // 16-byte reads of consecutive rows fall on distinct bank groups
    __shared__ __align__(16) uint32_t S[2][kMaxUnits][kRow];
    __shared__ uint32_t z[kMaxUnits + 1];     // this item's share of the unreduced sum
    __shared__ uint32_t d[kMaxUnits];         // and of the P_uu parities
    pdl_prologue();
    const Alg2Item it = items[blockIdx.x];
    const Alg2Block blk = table[it.block];
    const uint32_t k = blk.k, tid = threadIdx.x;
    for (uint32_t i = tid; i <= k; i += blockDim.x) z[i] = 0;
    for (uint32_t i = tid; i < k; i += blockDim.x) d[i] = 0;
    if (tid < 2 * k) {
        const uint32_t src = tid / k, u = tid % k;
        const uint16_t *s = (src ? y : x) + blk.in_unit + u;
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint32_t ea = 32 * it.group + uint32_t(i), eb = ea + 16;
            const uint32_t a = ea < n_p ? s[uint64_t(ea) * k] : 0u;
            const uint32_t c = eb < n_p ? s[uint64_t(eb) * k] : 0u;
            w[i] = a | (c << 16);
        }
        slice<16>(w);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(&S[src][u][4 * c]) = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
    __syncthreads();
    for (uint32_t p = it.p0 + tid; p < it.p1; p += blockDim.x) {
        // row u starts at R(u) = u k - u (u - 1) / 2
        const float b2 = float(2 * k + 1);
        uint32_t u = uint32_t((b2 - sqrtf(b2 * b2 - 8.0f * float(p))) * 0.5f);
        auto row = [k](uint32_t r) { return r * k - r * (r - 1) / 2; };
        while (u > 0 && row(u) > p) --u;
        while (u + 1 < k && row(u + 1) <= p) ++u;
        const uint32_t v = u + (p - row(u));
        const uint32_t mask = u == v ? 0u : ~0u;
        uint32_t X[16], Y[16];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint4 xu = lds4(&S[0][u][4 * c]), xv = lds4(&S[0][v][4 * c]);
            const uint4 yu = lds4(&S[1][u][4 * c]), yv = lds4(&S[1][v][4 * c]);
            X[4 * c] = lop_and_xor(xv.x, mask, xu.x);
            X[4 * c + 1] = lop_and_xor(xv.y, mask, xu.y);
            X[4 * c + 2] = lop_and_xor(xv.z, mask, xu.z);
            X[4 * c + 3] = lop_and_xor(xv.w, mask, xu.w);
            Y[4 * c] = lop_and_xor(yv.x, mask, yu.x);
            Y[4 * c + 1] = lop_and_xor(yv.y, mask, yu.y);
            Y[4 * c + 2] = lop_and_xor(yv.z, mask, yu.z);
            Y[4 * c + 3] = lop_and_xor(yv.w, mask, yu.w);
        }
        const uint32_t c = gram16_parities(X, Y, pm);  // diagonal d at bit d (31 bits)
        if (u == v) {
            atomicXor(&d[u], c);
            continue;
        }
        const uint32_t off = u + v;  // in 16-bit units
        if (off & 1u) {
            atomicXor(&z[off >> 1], c << 16);
            atomicXor(&z[(off >> 1) + 1], c >> 16);
        } else {
            atomicXor(&z[off >> 1], c);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i <= k; i += blockDim.x)
        if (z[i]) atomicXor(&zg[blk.zoff + i], z[i]);
    for (uint32_t i = tid; i < k; i += blockDim.x)
        if (d[i]) atomicXor(&zg[blk.zoff + k + 1 + i], d[i]);
}

// W_o = XOR of D_u over max(0, o - k + 1) <= u <= min(o, k - 1), from the
// prefix XORs H[u] = D_0 ^ ... ^ D_{u-1}; 0 past the last offset 2k - 2.
__device__ __forceinline__ uint32_t puu_window(const uint32_t *H, uint32_t k, uint32_t o) {
    if (o > 2 * k - 2) return 0u;
    const uint32_t lo = o + 1 > k ? o + 1 - k : 0u, hi = o < k - 1 ? o : k - 1;
    return H[hi + 1] ^ H[lo];
}

__global__ void __launch_bounds__(128)
    alg2_reduce_kernel(const Alg2Block *__restrict__ table, const uint32_t *__restrict__ zg,
                       uint16_t *__restrict__ out) {
    __shared__ uint32_t z[kMaxUnits + 2], H[kMaxUnits + 2];
    pdl_prologue();  // the products launch has completed past this point
    const Alg2Block blk = table[blockIdx.x];
    const uint32_t q = blk.q, k = blk.k, nz = k + 1, tid = threadIdx.x;
    const uint32_t qw = q >> 5, qb = q & 31u, nh = nz - qw;
    // prefix XORs of the P_uu parities, H[u] = D_0 ^ ... ^ D_{u-1}: warp 0,
    // lane j holding D_{4j} .. D_{4j+3} (k <= 128), an XOR scan across lanes
    if (tid < 32) {
        uint32_t d[4], run = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t u = 4 * tid + uint32_t(i);
            d[i] = u < k ? zg[blk.zoff + nz + u] : 0u;
            run ^= d[i];
        }
        uint32_t incl = run;  // inclusive scan of the lanes' XORs
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= uint32_t(o)) incl ^= v;
        }
        uint32_t acc = incl ^ run;  // XOR of the lanes before this one
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t u = 4 * tid + uint32_t(i);
            if (u <= k) H[u] = acc;
            acc ^= d[i];
        }
        if (tid == 31 && k == kMaxUnits) H[kMaxUnits] = acc;  // the whole XOR
    }
    __syncthreads();
    // word i of the sum: W_o (31 bits at bit 16 o) for o = 2i - 1, 2i, 2i + 1
    for (uint32_t i = tid; i < nz; i += blockDim.x)
        z[i] = zg[blk.zoff + i] ^ puu_window(H, k, 2 * i) ^ (i ? puu_window(H, k, 2 * i - 1) >> 16 : 0u) ^
               (puu_window(H, k, 2 * i + 1) << 16);
    // fold the part at and above x^q back by P's taps until none is left
    // (each fold lowers the degree by q - c; bounded for safety)
    for (int fold = 0; fold < 64; ++fold) {
        __syncthreads();
        bool any = false;
        for (uint32_t i = tid; i < nh; i += blockDim.x) {
            uint32_t v = z[qw + i] >> qb;
            if (qb && qw + i + 1 < nz) v |= z[qw + i + 1] << (32 - qb);
            H[i] = v;
            any |= v != 0;
        }
        if (!__syncthreads_or(any)) break;
        for (uint32_t i = tid; i < nz; i += blockDim.x) {
            uint32_t v = z[i];
            if (i > qw || (i == qw && qb == 0)) v = 0;
            else if (i == qw) v &= (1u << qb) - 1u;
#pragma unroll
            for (uint32_t t = 0; t < 4; ++t) {
                if (t >= blk.ntaps) break;
                const uint32_t e = blk.taps[t], ew = e >> 5, eb = e & 31u;
                if (i >= ew && i - ew < nh) v ^= H[i - ew] << eb;
                if (eb && i >= ew + 1 && i - ew - 1 < nh) v ^= H[i - ew - 1] >> (32 - eb);
            }
            z[i] = v;
        }
    }
    __syncthreads();
    for (uint32_t u = tid; u < blk.k; u += blockDim.x) out[blk.out_unit + u] = uint16_t(z[u >> 1] >> (16 * (u & 1u)));
}

void release(qext_alg2_plan *p) {
    cudaFree(p->d_blocks);
    cudaFree(p->d_items);
    cudaFree(p->d_z);
    p->d_blocks = nullptr;
    p->d_items = nullptr;
    p->d_z = nullptr;
}

// The device tables (blocks, work items, sums), made on the first extraction
// on the plan's device.
int upload(qext_alg2_plan *p) {
    std::lock_guard<std::mutex> lock(p->mu);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return QEXT_E_CUDA;
    if (p->d_blocks) return dev == p->device ? QEXT_OK : QEXT_E_STATE;
    if (cudaMalloc(&p->d_blocks, sizeof(Alg2Block) * p->blocks.size()) != cudaSuccess ||
        cudaMalloc(&p->d_items, sizeof(Alg2Item) * p->items.size()) != cudaSuccess ||
        cudaMalloc(&p->d_z, sizeof(uint32_t) * p->zwords) != cudaSuccess ||
        cudaMemcpy(p->d_blocks, p->blocks.data(), sizeof(Alg2Block) * p->blocks.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(p->d_items, p->items.data(), sizeof(Alg2Item) * p->items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        release(p);
        return QEXT_E_CUDA;
    }
    p->device = dev;
    return QEXT_OK;
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
    // every block's field polynomial; the searches of distinct degrees run
    // on parallel host threads (the largest degrees take the longest)
    std::vector<int> ok(max_blocks, 0);
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const uint32_t nthreads = std::max(1u, std::min(max_blocks, hw ? hw : 4u));
        std::atomic<uint32_t> next{0};
        std::vector<std::thread> pool;
        for (uint32_t t = 0; t < nthreads; ++t)
            pool.emplace_back([&] {
                for (uint32_t i; (i = next.fetch_add(1)) < max_blocks;) {
                    const uint32_t l = max_blocks - 1 - i;  // largest degrees first
                    Alg2Block &blk = p->blocks[l];
                    blk.q = uint32_t(q1 + dq * l);
                    blk.k = blk.q / 16;
                    for (int j = 0; j < 4; ++j) blk.taps[j] = 0;
                    ok[l] = qext::field_poly(blk.q, blk.taps, &blk.ntaps) ? 1 : 0;
                }
            });
        for (auto &th : pool) th.join();
    }
    uint64_t bits = 0, obits = 0;
    for (uint32_t l = 0; l < max_blocks; ++l) {
        if (!ok[l]) {
            delete p;
            return QEXT_E_PARAM;
        }
        Alg2Block &blk = p->blocks[l];
        blk.in_unit = bits / 16;
        blk.out_unit = obits / 16;
        blk.zoff = p->zwords;
        bits += uint64_t(blk.q) * p->n_p;
        obits += blk.q;
        p->zwords += 2 * blk.k + 1;
        // work items: the block's k (k + 1) / 2 unit products, per group of 32 elements
        p->item_prefix.push_back(uint32_t(p->items.size()));
        const uint32_t pairs = blk.k * (blk.k + 1) / 2, groups = (p->n_p + 31) / 32;
        for (uint32_t g = 0; g < groups; ++g)
            for (uint32_t p0 = 0; p0 < pairs; p0 += kItemProducts)
                p->items.push_back(Alg2Item{l, g, p0, std::min(pairs, p0 + kItemProducts)});
    }
    p->item_prefix.push_back(uint32_t(p->items.size()));
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
    const int rc = upload(const_cast<qext_alg2_plan *>(p));
    if (rc != QEXT_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Alg2Block &last = p->blocks[nblocks - 1];
    if (cudaMemsetAsync(p->d_z, 0, sizeof(uint32_t) * (last.zoff + 2 * last.k + 1), st) != cudaSuccess)
        return QEXT_E_CUDA;
    StreamArgs pm;
    std::memset(&pm, 0, sizeof pm);
    pm.set_multipliers();
    const Alg2Item *const items = p->d_items;
    const Alg2Block *const table = p->d_blocks;
    uint32_t *const z = p->d_z;
    const uint32_t n_p = p->n_p;
    const int rp = qext::launch_pdl(alg2_products_kernel, int(p->item_prefix[nblocks]), kAlg2Threads, 0, st, items,
                                    table, n_p, x, y, z, pm);
    if (rp != QEXT_OK) return rp;
    return qext::launch_pdl(alg2_reduce_kernel, int(nblocks), 128, 0, st, table, static_cast<const uint32_t *>(z), out);
}

int qext_alg2_destroy(qext_alg2_plan *p) {
    if (!p) return QEXT_OK;
    release(p);
    delete p;
    return QEXT_OK;
}

}  // extern "C"
