/*
 * qext.h -- C ABI of the GB300 (sm_103a) implementation of the block-wise
 * seedless two-source extractor Ext_bs^eq of Li & Zhou, "Real-Time Seedless
 * Post-Processing for Quantum Random Number Generators" (arXiv 2402.14607).
 *
 * What is computed (Algorithm 1 with the inner-product gadget, Def. 3.2):
 *   two raw bit streams x, y are cut into consecutive, non-overlapping
 *   n-bit blocks; block l of each stream is read as n_p elements of GF(2^q)
 *   (n = q * n_p); the block pair maps to
 *       Z^(l) = Ext_IP^{n_p,q}(x_l, y_l) = sum_{i<n_p} x_{l,i} * y_{l,i}
 *   in GF(2^q); Z^(l) is truncated to its first m coefficients and the
 *   outputs are concatenated in block order.  All arithmetic is exact GF(2).
 *
 * Bit conventions (the paper fixes none; these are this library's):
 *   - streams are arrays of uint32 words, little-endian; stream bit t is bit
 *     (t mod 32) of word t/32;
 *   - block l is stream bits [l*n, (l+1)*n); element i of a block is bits
 *     [i*q, (i+1)*q) of the block; element bit j is the coefficient of
 *     alpha^j;
 *   - GF(2^q) = F_2[alpha]/P(alpha) with P the minimum-weight irreducible
 *     polynomial of degree q that comes first in the order x^q + x^a + 1
 *     (smallest a), then x^q + x^c + x^b + x^a + 1 (smallest c, then b,
 *     then a); q = 1 is F_2 itself;
 *   - output: Z^(l)'s coefficients alpha^0..alpha^(m-1) occupy output bits
 *     [l*m, (l+1)*m); bits of the last output word past nblocks*m are 0.
 *
 * Errors: every call returns QEXT_OK (0) or a negative QEXT_E_* code; no call
 * aborts or prints.  Calls that enqueue GPU work are asynchronous on the given
 * stream and report launch errors only; a kernel that gives up a bounded wait
 * records QEXT_E_TIMEOUT in a device status word read by qext_device_status.
 *
 * Threading: a plan is immutable after creation and may be used from several
 * host threads and streams at once.  A qext_stream is not thread-safe.
 */
#ifndef QEXT_H
#define QEXT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as the CUDA runtime's cudaStream_t; NULL = the legacy default
 * stream. */
typedef struct CUstream_st *qext_cuda_stream;

#define QEXT_OK 0
#define QEXT_E_INVAL (-1)       /* null / misaligned pointer, bad size or argument   */
#define QEXT_E_ENTROPY (-2)     /* min-entropy rate k/n <= 1/2: no guarantee (Sec. 5) */
#define QEXT_E_PARAM (-3)       /* no block factorisation meets eps (Thm 3.1)         */
#define QEXT_E_UNSUPPORTED (-4) /* field size q has no GPU kernel in this build       */
#define QEXT_E_CUDA (-5)        /* a CUDA runtime call failed                         */
#define QEXT_E_TIMEOUT (-6)     /* a kernel gave up a bounded wait                    */
#define QEXT_E_BUDGET (-7)      /* device-memory budget exhausted (admission)         */
#define QEXT_E_STATE (-8)       /* object used in a state that forbids the call       */
#define QEXT_E_NOSPACE (-9)     /* caller's output buffer too small                   */
#define QEXT_E_LIMIT (-10)      /* request exceeds a fixed capacity of the call       */

/* Human-readable name of a status code (static string, never NULL). */
const char *qext_status_string(int status);

/* ------------------------------------------------------------------------
 * Plans.
 * ------------------------------------------------------------------------ */
typedef struct qext_plan qext_plan; /* opaque, host-owned */

/*
 * qext_plan_create -- parameters of one block application of the extractor,
 * from Definition 2.3's (t, m, k, epsilon) with t = n.
 *   n    bits per block per source (the paper's q*n).  The GPU kernels need
 *        n to be a multiple of 32 (whole words per block).
 *   m    output bits per block, 1 <= m <= q; 0 selects m = q (Theorem 3.4's
 *        output length m = N b / n_p over a stream).
 *   k    min-entropy of one n-bit block of either source, in bits (the
 *        forward-block-source rate of Def. 3.1 gives k = delta * n).
 *   eps  per-block error target, 0 < eps < 1.
 * Choice (Algorithm 1 and Theorem 3.1): delta = k/n must exceed 1/2;
 * n_min = ceil(24/(2 delta - 1)); the divisors d of n with d >= n_min are
 * tried in increasing order with q = n/d and the first one with
 *   log2 eps_blk = log2 sqrt(3) - 1/4 - (k/4 - n/8) + 2q  <=  log2 eps
 * and m <= q is taken (n_p = d).  The field polynomial is generated and
 * checked for irreducibility here.
 * Host-only: touches no GPU.  *out receives a plan to free with qext_destroy.
 * Errors: INVAL (null out, n = 0, k outside (0, n], eps outside (0, 1)),
 * ENTROPY (k/n <= 1/2), PARAM (no divisor meets eps and m).  A plan with no
 * GPU kernel (q outside the built set, or n not a multiple of 32) is still
 * created; qext_extract then returns UNSUPPORTED (qext_plan_info reports it).
 */
int qext_plan_create(uint32_t n, uint32_t m, double k, double eps, qext_plan **out);

/* Frees a plan (NULL is accepted).  The plan must not be in use by queued
 * GPU work: synchronise the streams that used it first. */
int qext_destroy(qext_plan *p);

/*
 * qext_plan_info -- the chosen parameters.  Any output pointer may be NULL.
 *   q, n_p, m          as chosen (n = q * n_p);
 *   log2_eps_block     Theorem 3.1's per-block error, log2;
 *   poly_taps[4]       exponents of P below q, descending, then zeros
 *                      (the constant term 1 and x^q are implied);
 *   gpu_supported      1 if every GPU entry point has a kernel for this plan
 *                      (q in {1,2,4,8,16,32,64} and n a multiple of 32);
 *                      2 if only qext_extract and qext_extract_samples
 *                      (b = 16) have one: q = 80, any n_p (Sec. 4.2's field);
 *                      0 if none.
 * The error of a stream of L blocks is at most L * 2^log2_eps_block
 * (Theorem 3.3's sum with equal q).
 */
int qext_plan_info(const qext_plan *p, uint32_t *q, uint32_t *n_p, uint32_t *m, double *log2_eps_block,
                   uint64_t poly_taps[4], int *gpu_supported);

/*
 * qext_alg1_params -- Algorithm 1's own parameter line for N samples of b
 * bits, rate delta, whole-stream error eps:
 *   n_p = ceil(24 / (2 delta - 1)),  q = b * ceil(log2(N / (eps n_p)) / b).
 * Host-only.  Errors: INVAL (bad N, b, eps or null outputs), ENTROPY
 * (delta <= 1/2).
 */
int qext_alg1_params(double N_samples, uint32_t b, double delta, double eps, uint32_t *n_p, uint32_t *q);

/* ------------------------------------------------------------------------
 * Stateless extraction over whole blocks (Algorithm 1's loop body).
 * ------------------------------------------------------------------------ */

/*
 * qext_extract -- Z^(l) for l = 0 .. nblocks-1 (Algorithm 1, Def. 3.2).
 *   x, y   DEVICE pointers to nblocks*n bits each (nblocks*n/32 words),
 *          4-byte aligned; 16-byte alignment selects the vectorised path.
 *   out    DEVICE pointer to ceil(nblocks*m/32) words; fully written (the
 *          unused high bits of the last word are zero).  Must not overlap x
 *          or y.
 *   stream CUDA stream the kernel is enqueued on (asynchronous).
 * The caller owns all three buffers.  nblocks = 0 enqueues nothing.
 * Errors: INVAL (null plan or pointer, misalignment), UNSUPPORTED (q has no
 * kernel: this build covers q in {1, 2, 4, 8, 16, 32, 64} with n a multiple
 * of 32, and q = 80 with any n_p), CUDA (launch).
 */
int qext_extract(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                 qext_cuda_stream stream);

/* Flags of qext_extract_ex (launch shape only; the output never changes). */
#define QEXT_F_DIRECT 0x1u /* skip shared-memory staging: each thread reads its block from global memory */
#define QEXT_F_NBUF1 0x2u  /* one tile buffer per CTA (more CTAs per SM) instead of two (prefetch) */
#define QEXT_F_TILE32 0x4u /* at most 32 blocks per tile */
#define QEXT_F_TILE64 0x8u /* at most 64 blocks per tile (exclusive with TILE32) */
#define QEXT_F_TEST_TIMEOUT 0x10u /* test of failure detection: every CTA (or, in the per-warp kernels,
                                   every warp) arms its barrier but issues no copy, gives up its bounded
                                   wait after a few polls, records QEXT_E_TIMEOUT (qext_device_status) and
                                   returns; outputs are not written.  Needs 16-byte aligned x, y and a
                                   staged tile (else INVAL).  Alone it tests the default kernel of the
                                   plan (the per-warp kernel for q = 16 with n_p = 64; for q = 80,
                                   the blocks-in-lanes kernel, with nblocks a multiple of 32); with
                                   QEXT_F_CTA_TILES, the CTA-tile kernel.  qext_extract_samples_ex
                                   accepts it for its per-warp kernel (q = 4, 16 with n_p = 64) only. */
#define QEXT_F_ALL 0x1Fu

/*
 * qext_extract_ex -- qext_extract with launch options (flags, 0 = the
 * default path chosen by qext_extract).  Same arguments, ownership and errors;
 * INVAL also for unknown flag bits.  The output is identical for every flag
 * combination.  The default path for q = 16 with n_p = 64 and 16-byte
 * aligned x, y is a per-warp copy pipeline over sub-tiles of 32 blocks; any
 * flag but QEXT_F_TEST_TIMEOUT, including QEXT_F_CTA_TILES (below), selects
 * the CTA-tile kernel instead.  q = 80 plans take QEXT_F_TEST_TIMEOUT only.
 */
int qext_extract_ex(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                    qext_cuda_stream stream, uint32_t flags);

/*
 * qext_extract_samples -- fused ingest + extraction: the same output as
 * qext_pack_samples on each source followed by qext_extract, without the
 * packed streams ever reaching device memory.  Raw b-bit ADC samples (the low
 * b bits of each uint16; higher bits ignored) form the bit streams (Sec. 3,
 * sample s at stream bits [s*b, (s+1)*b)), which are cut into n-bit blocks.
 *   b          8, 12 or 16 (else UNSUPPORTED);
 *   x_samples, y_samples  DEVICE pointers to nsamples uint16 each, 16-byte
 *              aligned;
 *   nblocks    whole blocks to extract, nblocks * n <= nsamples * b;
 *   out        DEVICE pointer to ceil(nblocks*m/32) words, fully written.
 * Kernels exist for q in {4, 16, 64} (b = 8, 12, 16) and q = 80 (b = 16,
 * where the samples are the packed stream); other q return UNSUPPORTED.
 * Asynchronous on stream.  Errors: INVAL, UNSUPPORTED, CUDA.
 */
int qext_extract_samples(const qext_plan *p, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                         uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream);

/*
 * qext_extract_samples_ex -- qext_extract_samples with launch options (0 =
 * the default path).  The default for q = 4, 16 with n_p = 64 runs one copy
 * pipeline per warp: each warp TMA-copies the raw samples of 32 blocks into
 * its own shared-memory buffer and every lane packs its block's samples in
 * registers.  Other shapes use CTA-wide tiles of raw samples, TMA-copied and
 * packed in place in shared memory.  The output is identical for every flag
 * combination; INVAL for unknown flag bits.
 */
/* q = 4, 16: warp-specialised CTAs (producer warps pack from global memory
 * into shared memory while consumer warps extract). */
#define QEXT_F_WARP_SPECIALIZED 0x20u
/* Two raw-sample buffers (per warp, or per CTA with CTA-wide tiles), the next
 * copy issued one whole tile ahead (more shared memory, fewer warps per SM). */
#define QEXT_F_RAW_PREFETCH 0x40u
/* CTA-wide tiles (packed in place, for samples) even where the per-warp
 * kernel applies; also accepted by qext_extract_ex. */
#define QEXT_F_CTA_TILES 0x80u
int qext_extract_samples_ex(const qext_plan *p, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                            uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream,
                            uint32_t flags);

/*
 * qext_pack_samples -- ingest: raw ADC samples to a packed stream.  Sample s
 * (b bits, the low bits of samples[s]) occupies stream bits [s*b, (s+1)*b)
 * (Sec. 3: X = X_1 ... X_N in ({0,1}^b)^N).
 *   samples DEVICE pointer to nsamples uint16 values, 2-byte aligned; bits
 *           above b are ignored.
 *   out     DEVICE pointer to ceil(nsamples*b/32) words, fully written.
 *   1 <= b <= 16.  Asynchronous on stream.
 * Errors: INVAL, CUDA.
 */
int qext_pack_samples(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint32_t *out,
                      qext_cuda_stream stream);

/* ------------------------------------------------------------------------
 * Streams: Algorithm 1 over raw data that arrives in chunks.
 *
 * The paper's extractor consumes the two sources strictly in time order,
 * block l of x pairing with block l of y (Algorithm 1, the window I_l advanced
 * by one block per step; Algorithm 2 carries the same cursor).  A qext_stream
 * keeps, on the device, the unconsumed tail of each source (fewer than n
 * bits) and the output bits not yet forming a whole word (fewer than 32), so
 * that pushing a stream in pieces of any bit length yields exactly the output
 * of one push of the whole (its concatenation of Z^(l), Theorem 3.4's
 * m * floor(L/n) bits).  Not thread-safe; one CUDA stream per qext_stream.
 * ------------------------------------------------------------------------ */
typedef struct qext_stream qext_stream; /* opaque, host-owned, holds device memory */

/* Allocates the device state for a plan (which must outlive the stream).
 * Errors: INVAL, UNSUPPORTED (no GPU kernel for the plan), CUDA. */
int qext_stream_create(const qext_plan *p, qext_stream **out);

/* Frees the stream (NULL accepted).  Synchronise its CUDA stream first. */
int qext_stream_destroy(qext_stream *s);

/* Counters (host-side, exact): blocks output so far, tail bits held, output
 * bits pending.  Any pointer may be NULL. */
int qext_stream_info(const qext_stream *s, uint64_t *blocks_done, uint64_t *tail_bits, uint32_t *pending_bits);

/*
 * qext_stream_push -- appends nbits bits of each source and extracts every
 * block that becomes complete.
 *   x, y      DEVICE pointers to ceil(nbits/32) words each, 4-byte aligned;
 *             stream bits [0, nbits) of the chunk (LSB-first), the rest of
 *             the last word ignored.  16-byte alignment, with no tail or
 *             pending bits held, takes the in-place TMA-staged kernel.
 *   out       DEVICE pointer; receives the pending bits followed by the new
 *             blocks' m-bit outputs.  out_capacity_words must be at least
 *             ceil((pending + new_blocks*m)/32) (else NOSPACE, nothing done).
 *   *out_words  complete output words written; the remaining bits (fewer
 *             than 32) stay pending in the stream (out[*out_words] may have
 *             been written as well).
 * Asynchronous on `stream`: the caller's x, y, out must stay valid until it
 * completes.  Errors: INVAL, NOSPACE, UNSUPPORTED (general path, blocks over
 * 8192 bits), CUDA.
 */
int qext_stream_push(qext_stream *s, const uint32_t *x, const uint32_t *y, uint64_t nbits, uint32_t *out,
                     uint64_t out_capacity_words, uint64_t *out_words, qext_cuda_stream stream);

/*
 * qext_stream_push_samples -- qext_stream_push for raw ADC samples: appends
 * nsamples b-bit samples of each source (the low b bits of each uint16,
 * sample j at the next stream bits [j*b, (j+1)*b), LSB first; Sec. 3's
 * X_1 ... X_N fed in time order) and extracts every block that becomes
 * complete, with the same output, counters and state as qext_pack_samples
 * followed by qext_stream_push of the nsamples*b packed bits.
 *   b            1 .. 16 (else INVAL);
 *   x_samples, y_samples  DEVICE pointers to nsamples uint16 each, 2-byte
 *                aligned.
 * With no tail or pending bits held, b in {8, 12, 16}, q in {4, 16, 64}
 * and 16-byte aligned samples, the whole blocks run through the fused
 * ingest + extraction kernel of qext_extract_samples and only the leftover
 * bits are packed (into the new tail); otherwise the samples are packed into
 * the stream's own staging buffers (device memory owned by the stream, grown
 * on demand: a push that grows them synchronises `stream` first) and pushed
 * as bits.  out, out_capacity_words, *out_words and the asynchrony are as
 * for qext_stream_push.  Errors: INVAL, NOSPACE, UNSUPPORTED, CUDA.
 */
int qext_stream_push_samples(qext_stream *s, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                             uint64_t nsamples, uint32_t *out, uint64_t out_capacity_words, uint64_t *out_words,
                             qext_cuda_stream stream);

/*
 * qext_stream_flush -- ends the stream: writes the pending output bits (if
 * any) to out[0] (DEVICE, zero above *out_bits) and drops the incomplete
 * block (Algorithm 1 outputs whole blocks only).  Counters keep blocks_done.
 * Errors: INVAL, NOSPACE, CUDA.
 */
int qext_stream_flush(qext_stream *s, uint32_t *out, uint64_t out_capacity_words, uint32_t *out_bits,
                      qext_cuda_stream stream);

/* Bytes qext_stream_save writes for this stream (0 for NULL). */
size_t qext_stream_state_size(const qext_stream *s);

/*
 * qext_stream_save / qext_stream_restore -- checkpoint of a stream's state
 * (counters, tails, pending bits) into a HOST buffer, and a new stream from
 * one.  Save waits for `stream` (it copies device state to the host).  A
 * restored stream continues exactly where the saved one stood.  Restore
 * needs a plan with the same n, m, q, n_p (else STATE).
 * Errors: INVAL (bad buffer), NOSPACE, STATE, CUDA.
 */
int qext_stream_save(const qext_stream *s, void *host_buf, size_t capacity, size_t *size, qext_cuda_stream stream);
int qext_stream_restore(const qext_plan *p, const void *host_buf, size_t size, qext_stream **out,
                        qext_cuda_stream stream);

/* ------------------------------------------------------------------------
 * Batches: many stream pairs of uneven length and mixed block size in one
 * persistent kernel launch (blocks are independent, Sec. 3.3, so the blocks
 * of all streams can share one launch).
 * ------------------------------------------------------------------------ */
typedef struct qext_batch_item {
    const qext_plan *plan; /* this stream's plan (q, n, m); must outlive the batch */
    const uint32_t *x;     /* DEVICE, nblocks * n bits, 4-byte aligned (16: TMA staging) */
    const uint32_t *y;     /* DEVICE, same layout as x */
    uint64_t nblocks;      /* whole blocks of this stream */
    uint32_t *out;         /* DEVICE, ceil(nblocks*m/32) words, fully written */
} qext_batch_item;

/* Launch shape of a batch (the autotuner's search space). */
typedef struct qext_batch_config {
    uint32_t blocks_per_thread_small; /* q <= 4: 1, 2 or 4 blocks per thread per tile */
    uint32_t blocks_per_thread_mid;   /* 4 < q <= 16: 1, 2 or 4 */
    uint32_t ctas_per_sm;             /* 1 .. 3 persistent CTAs per SM */
    uint32_t order;                   /* 0: tiles by decreasing cost; 1: stream order */
} qext_batch_config;

typedef struct qext_batch qext_batch; /* opaque, host-owned, holds device memory */

/*
 * qext_batch_create -- builds the device descriptor and tile tables for the
 * items (pointers are recorded, not copied: the buffers must stay valid and
 * may be refilled between runs).  Default configuration; see autotune.
 * Errors: INVAL (null or misaligned pointers), UNSUPPORTED (a plan without a
 * GPU kernel, or blocks over 8192 bits), CUDA.
 */
int qext_batch_create(const qext_batch_item *items, uint32_t nitems, qext_batch **out);
int qext_batch_destroy(qext_batch *b);

/* One stream pair of raw ADC samples in a batch: the ingest of
 * qext_extract_samples (Sec. 3: sample s at stream bits [s*b, (s+1)*b), the
 * low b bits of each uint16) runs inside the batched kernel, which packs each
 * tile from the samples straight into shared memory; the packed stream never
 * reaches device memory. */
typedef struct qext_batch_samples_item {
    const qext_plan *plan;     /* q <= 64 with a GPU kernel (gpu_supported == 1); must outlive the batch */
    uint32_t b;                /* bits per sample: 8, 12 or 16 */
    const uint16_t *x_samples; /* DEVICE, nsamples uint16, 16-byte aligned */
    const uint16_t *y_samples; /* DEVICE, same layout as x_samples */
    uint64_t nsamples;         /* samples per source; nblocks * n <= nsamples * b */
    uint64_t nblocks;          /* whole blocks of this stream */
    uint32_t *out;             /* DEVICE, ceil(nblocks*m/32) words, fully written */
} qext_batch_samples_item;

/*
 * qext_batch_create_samples -- qext_batch_create for streams of raw samples
 * (same tiles, configuration, run, capture, launch and autotune; outputs
 * equal to qext_extract_samples per stream).  The items' arguments are
 * checked before the device is touched.  Errors: INVAL (null or misaligned
 * pointers, nblocks * n > nsamples * b), UNSUPPORTED (b not 8, 12 or 16, a
 * plan without a GPU kernel, or blocks over 8192 bits), CUDA.
 * qext_batch_run_ex with QEXT_F_TEST_TIMEOUT returns INVAL for such a batch
 * (its tiles take no bulk copy).
 */
int qext_batch_create_samples(const qext_batch_samples_item *items, uint32_t nitems, qext_batch **out);

/* Current configuration and tile count (either pointer may be NULL). */
int qext_batch_get_config(const qext_batch *b, qext_batch_config *cfg, uint32_t *ntiles);
/* Rebuilds the tile table for cfg (drops a captured graph).  Errors: INVAL. */
int qext_batch_set_config(qext_batch *b, const qext_batch_config *cfg);

/* One run: a memset of the tile counter and ONE kernel launch on `stream`,
 * every item's output written.  Asynchronous.  Errors: INVAL, CUDA. */
int qext_batch_run(qext_batch *b, qext_cuda_stream stream);

/* qext_batch_run with flags: 0, or QEXT_F_TEST_TIMEOUT (test of failure
 * detection: every CTA arms its tile barrier without issuing the bulk copy,
 * gives up its bounded wait after a few polls, records QEXT_E_TIMEOUT in the
 * device status word and returns; outputs are not written; every item with
 * blocks must be 16-byte aligned, else INVAL).  Errors: INVAL, CUDA. */
int qext_batch_run_ex(qext_batch *b, qext_cuda_stream stream, uint32_t flags);

/* Records one run into a CUDA graph (capture on `stream`, which must not be
 * capturing already); qext_batch_launch replays it.  Errors: STATE (launch
 * before capture), CUDA. */
int qext_batch_capture(qext_batch *b, qext_cuda_stream stream);
int qext_batch_launch(qext_batch *b, qext_cuda_stream stream);

/*
 * qext_batch_autotune -- times every configuration (tile shape for q <= 4 and
 * q <= 16, CTAs per SM, tile order) on this batch's own data, `reps` runs
 * each after a warm-up, keeps the fastest, and reports its time per run.
 * Synchronises `stream`.  The outputs are those of a normal run.
 */
int qext_batch_autotune(qext_batch *b, uint32_t reps, qext_cuda_stream stream, float *best_ms);

/*
 * qext_batch_run_noalloc -- the same outputs as qext_batch_create +
 * qext_batch_run on these items, for callers that cannot allocate device
 * memory: code that owns a fixed device-memory budget set at start-up (an
 * appliance or server whose admission control counts every byte), and code
 * in a latency-critical loop where cudaMalloc / cudaFree would synchronise
 * the device.  Nothing is allocated: the descriptors and the tile counter live
 * in one static device array of the library (about 200 KB, present on every
 * device that loads the library until the process exits).  The paper has no
 * counterpart; this is a calling convention, not part of the method.
 *   items, nitems  as for qext_batch_create; at most QEXT_NOALLOC_MAX_ITEMS
 *                  items (else QEXT_E_LIMIT, nothing done).
 * The first call on a device, with that device current, looks up the array's
 * device address and sets the kernel's shared-memory limit.  Every call
 * reuses the same array: it is rewritten (counter reset to 0) by each call,
 * so calls whose work overlaps on the GPU -- on different streams, or from
 * different host threads without ordering -- race and give wrong outputs;
 * order them on one stream.  The descriptors travel from a static host
 * buffer that the next call rewrites, staged before cudaMemcpyAsync returns
 * on an ordinary stream; a stream that is being captured into a CUDA graph
 * would instead record a copy that reads the buffer at replay time, so such
 * a stream is refused with STATE before anything is enqueued.  Default tile
 * configuration (no autotuning).  Errors: INVAL, UNSUPPORTED, LIMIT, STATE,
 * CUDA.
 */
#define QEXT_NOALLOC_MAX_ITEMS 1024
int qext_batch_run_noalloc(const qext_batch_item *items, uint32_t nitems, qext_cuda_stream stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of requests from many QRNG channels.
 *
 * A channel is a pair of raw streams with its own plan; a request carries the
 * next piece of a channel's streams in HOST memory (pinned memory lets the
 * copies overlap) and receives the m-bit outputs of the blocks it completes,
 * concatenated (a block straddling two requests completes in the later one;
 * the channel's chaining state stays on the device).  Requests of a channel
 * run one at a time in arrival order; requests of different channels that
 * arrive while others are on the GPU are admitted as soon as device memory
 * within the HBM budget frees up, and share batched kernel launches.
 * ------------------------------------------------------------------------ */
typedef struct qext_server qext_server;

typedef struct qext_server_config {
    uint64_t hbm_budget_bytes; /* device memory for requests in flight (one arena) */
    uint32_t max_batch;        /* requests per round, 1 .. QEXT_NOALLOC_MAX_ITEMS */
    uint32_t fake_executor;    /* 1: schedule only, no GPU (outputs not written) */
} qext_server_config;

typedef struct qext_completion {
    uint64_t request_id;
    uint32_t channel;
    int32_t status;      /* QEXT_OK or the error of this request */
    uint64_t out_bits;   /* output bits written to the request's buffer */
    uint64_t blocks;     /* blocks the request completed */
    double submit_s;     /* steady-clock seconds at submit */
    double done_s;       /* steady-clock seconds when the output was on the host */
    double latency_s;    /* done_s - submit_s */
    uint32_t batched;    /* 1 if it ran in the round's batched launch */
    uint32_t reserved;
} qext_completion;

typedef struct qext_server_stats {
    uint64_t submitted, completed, rounds, max_round;
    uint64_t bits_out;
    uint64_t bytes_in_use, peak_bytes, budget_bytes;
} qext_server_stats;

/* Starts the scheduler thread; allocates the whole budget as one device
 * arena (unless fake_executor).  Errors: INVAL, CUDA. */
int qext_server_create(const qext_server_config *cfg, qext_server **out);
/* Finishes every submitted request, stops the thread, frees everything. */
int qext_server_destroy(qext_server *s);
/* Adds a channel (plan must outlive the server); *channel receives its id.
 * Errors: INVAL, UNSUPPORTED, CUDA. */
int qext_server_add_channel(qext_server *s, const qext_plan *p, uint32_t *channel);
/*
 * qext_server_submit -- queues a request.
 *   b          0: x_host / y_host hold `count` stream bits as packed uint32
 *              words; 1..16: they hold `count` b-bit samples as uint16.
 *   out_host   HOST buffer of out_capacity_words >= ceil((count_bits/n + 2)
 *              * m / 32) words (else NOSPACE); written before completion.
 * The host buffers must stay valid until the request completes.
 * Errors: INVAL, NOSPACE, BUDGET (larger than the whole budget).
 */
int qext_server_submit(qext_server *s, uint32_t channel, uint32_t b, const void *x_host, const void *y_host,
                       uint64_t count, uint32_t *out_host, uint64_t out_capacity_words, uint64_t *request_id);
/* Moves up to max completions (oldest first) into out; *n receives the count. */
int qext_server_poll(qext_server *s, qext_completion *out, uint32_t max, uint32_t *n);
/* Waits until every submitted request has completed.  Errors: TIMEOUT. */
int qext_server_drain(qext_server *s, double timeout_s);
int qext_server_get_stats(qext_server *s, qext_server_stats *st);

/* ------------------------------------------------------------------------
 * Host-to-host extraction with overlapped copies.
 * ------------------------------------------------------------------------ */
typedef struct qext_pipeline qext_pipeline; /* opaque, holds device buffers and CUDA streams */

/*
 * qext_pipeline_create -- device buffers for two chunks of chunk_blocks
 * blocks (rounded up so that a chunk holds whole samples and whole output
 * words; qext_pipeline_info reports the value used).
 *   b   0: input is packed uint32 words; 8, 12 or 16: raw samples in uint16
 *       containers, extracted by qext_extract_samples (q in {4, 16, 64}).
 * Errors: INVAL, UNSUPPORTED, CUDA.
 */
int qext_pipeline_create(const qext_plan *p, uint32_t b, uint64_t chunk_blocks, qext_pipeline **out);
int qext_pipeline_info(const qext_pipeline *pp, uint64_t *chunk_blocks);
int qext_pipeline_destroy(qext_pipeline *pp);

/*
 * qext_pipeline_run -- extracts nblocks blocks from HOST streams x_host,
 * y_host (count samples, or count bits for b = 0; nblocks * n <= count
 * bits) into out_host (HOST, ceil(nblocks*m/32) words), chunk by chunk with
 * copies in, kernels and copies out overlapped.  Synchronous: returns when the
 * output is in out_host.  Page-locked host memory makes the copies
 * asynchronous (pageable memory works, slower).  Errors: INVAL, CUDA.
 */
int qext_pipeline_run(qext_pipeline *pp, const void *x_host, const void *y_host, uint64_t count, uint64_t nblocks,
                      uint32_t *out_host);

/*
 * qext_device_status -- reads and clears the device status word of the
 * current device (QEXT_OK or QEXT_E_TIMEOUT from a kernel that gave up a
 * bounded wait).  Synchronises the device.  Errors: CUDA.
 */
int qext_device_status(int *status);

/* ------------------------------------------------------------------------
 * Min-entropy monitoring.  The guarantees rest on the sources' min-entropy
 * H_min(X) = -log2 max_x P(X = x) (Sec. 2; the rate delta of Algorithms 1 and
 * 2); a stream whose sources drift is watched through the histogram of its
 * sample values.
 * ------------------------------------------------------------------------ */
/*
 * qext_sample_histogram -- counts[v] += the number of samples whose low b
 * bits equal v, for v < 2^b (bits above b ignored, as in the ingest).
 *   b        1 .. 16;
 *   samples  DEVICE pointer to nsamples uint16, 2-byte aligned (16-byte
 *            alignment enables vector loads);
 *   counts   DEVICE pointer to 2^b uint64, 8-byte aligned; the caller zeroes
 *            it to start and successive calls accumulate (e.g. per chunk).
 * Asynchronous on stream.  Errors: INVAL, CUDA.
 */
int qext_sample_histogram(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint64_t *counts,
                          qext_cuda_stream stream);
/* The plug-in estimate -log2(max_v counts[v] / sum_v counts[v]) of a HOST copy
 * of such a histogram (2^b entries); -1 if it is empty or b is out of range. */
double qext_min_entropy_estimate(uint32_t b, const uint64_t *counts_host);

/* ------------------------------------------------------------------------
 * Algorithm 2 (Ext_bs^neq, Sec. 3.3; error: Theorem 3.3): block sizes grow
 * with the block index, q_l = q_1 + l * Delta * b (l = 0, 1, ...), so that a
 * stream of unknown length can be extracted.  n = ceil(24 / (2 delta - 1))
 * elements per block (Algorithm 2's n); block l takes the next q_l * n bits of
 * each stream (the paper's cursor advances by q_l n / b samples), computes
 * Z^(l) = Ext_IP^{n, q_l} in GF(2^{q_l}) with that degree's field polynomial
 * (the convention of qext_plan_create) and outputs its q_l bits, concatenated
 * in block order.  With Delta = 0 this is Algorithm 1.
 * ------------------------------------------------------------------------ */
typedef struct qext_alg2_plan qext_alg2_plan;

/*
 * qext_alg2_plan_create -- the first max_blocks blocks of Algorithm 2 for
 * b-bit samples (1 <= b <= 16) of min-entropy rate delta.  q1 and Delta * b
 * must be multiples of 16 (the GPU works on 16-bit units), and
 * q1 + (max_blocks - 1) * Delta * b <= 2048 (the largest field built; at
 * q1 = Delta * b = 16 that is 128 blocks), else UNSUPPORTED.  Finds every
 * block's field polynomial on the host (the searches of the distinct degrees
 * run on parallel host threads and are kept for the process: seconds the
 * first time for fields up to 2048, nothing after that); touches no GPU.
 * The device tables are made by the first qext_alg2_extract, on the device
 * then current, which the plan is then bound to.  Caller owns *out.
 * Errors: INVAL, ENTROPY (delta <= 1/2), UNSUPPORTED, PARAM.
 */
int qext_alg2_plan_create(double delta, uint32_t b, uint32_t q1, uint32_t Delta, uint32_t max_blocks,
                          qext_alg2_plan **out);
/* n_p (Algorithm 2's n), max_blocks, and log2 of Theorem 3.3's bound
 * sqrt(3) sum_l 2^(-1/4 - (delta/4 - 1/8) q_l n + 2 q_l) over the plan's
 * blocks.  Any output pointer may be NULL.  Errors: INVAL. */
int qext_alg2_plan_info(const qext_alg2_plan *p, uint32_t *n_p, uint32_t *max_blocks, double *log2_error_bound);
/* Block l's q_l, window start (stream bit), output offset (bit) and
 * polynomial taps (as qext_plan_info); l = max_blocks gives the end of the
 * last block (q_l = 0).  Errors: INVAL. */
int qext_alg2_block_info(const qext_alg2_plan *p, uint32_t l, uint32_t *q_l, uint64_t *in_bit, uint64_t *out_bit,
                         uint64_t poly_taps[4]);
/*
 * qext_alg2_extract -- Z^(0) .. Z^(nblocks-1), nblocks <= max_blocks.
 *   x, y  DEVICE pointers to the streams as 16-bit units (unit u = stream
 *         bits [16u, 16u + 16), LSB first; for b = 16 the samples
 *         themselves), 2-byte aligned, at least in_bit(nblocks) / 16 units;
 *   out   DEVICE pointer to out_bit(nblocks) / 16 units, fully written.
 * Each block's unit products run as work items over many CTAs of one launch
 * into the plan's device sums, which a second launch reduces mod P_{q_l}, one
 * CTA per block.  Asynchronous on stream; calls on one plan that overlap on
 * the GPU share its sums and race (order them on one stream).  Errors: INVAL,
 * STATE (a device other than the one the plan's tables live on), CUDA.
 */
int qext_alg2_extract(const qext_alg2_plan *p, const uint16_t *x, const uint16_t *y, uint32_t nblocks, uint16_t *out,
                      qext_cuda_stream stream);
int qext_alg2_destroy(qext_alg2_plan *p);

#ifdef __cplusplus
}
#endif

#endif /* QEXT_H */
