// C ABI entry points that enqueue GPU work: argument checks, then the
// launchers of the .cu translation units.  Declarations and contracts are in
// include/qext.h.
#include <cstdint>

#include "qext_internal.h"
#include "qext_nvtx.h"

namespace {
bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
}  // namespace

extern "C" {

int qext_extract_ex(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                    qext_cuda_stream stream, uint32_t flags) {
    if (!p) return QEXT_E_INVAL;
    if (flags & ~uint32_t(QEXT_F_ALL | QEXT_F_CTA_TILES)) return QEXT_E_INVAL;
    if ((flags & QEXT_F_TILE32) && (flags & QEXT_F_TILE64)) return QEXT_E_INVAL;
    if (!p->gpu_supported && !p->gpu_q80) return QEXT_E_UNSUPPORTED;
    // q = 80: no launch options; QEXT_F_TEST_TIMEOUT tests the lanes kernel's bounded wait
    if (p->gpu_q80 && (flags & ~uint32_t(QEXT_F_TEST_TIMEOUT))) return QEXT_E_INVAL;
    if (nblocks == 0) return QEXT_OK;
    if (!x || !y || !out || !aligned(x, 4) || !aligned(y, 4) || !aligned(out, 4)) return QEXT_E_INVAL;
    if (nblocks > (UINT64_MAX / p->n)) return QEXT_E_INVAL;
    const qext::NvtxRange range("qext extract");
    if (p->gpu_q80) return qext::launch_extract_q80(p, x, y, nblocks, out, stream, flags);
    return qext::launch_extract(p, x, y, nblocks, out, stream, flags);
}

int qext_extract(const qext_plan *p, const uint32_t *x, const uint32_t *y, uint64_t nblocks, uint32_t *out,
                 qext_cuda_stream stream) {
    return qext_extract_ex(p, x, y, nblocks, out, stream, 0);
}

int qext_extract_samples(const qext_plan *p, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                         uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream) {
    return qext_extract_samples_ex(p, b, x_samples, y_samples, nsamples, nblocks, out, stream, 0);
}

int qext_extract_samples_ex(const qext_plan *p, uint32_t b, const uint16_t *x_samples, const uint16_t *y_samples,
                            uint64_t nsamples, uint64_t nblocks, uint32_t *out, qext_cuda_stream stream,
                            uint32_t flags) {
    if (!p) return QEXT_E_INVAL;
    if (flags & ~uint32_t(QEXT_F_WARP_SPECIALIZED | QEXT_F_RAW_PREFETCH | QEXT_F_CTA_TILES | QEXT_F_TEST_TIMEOUT))
        return QEXT_E_INVAL;
    // the test of failure detection exists for the per-warp kernel only
    if ((flags & QEXT_F_TEST_TIMEOUT) && (flags & (QEXT_F_WARP_SPECIALIZED | QEXT_F_CTA_TILES))) return QEXT_E_INVAL;
    if (!p->gpu_supported && !p->gpu_q80) return QEXT_E_UNSUPPORTED;
    if (b != 8 && b != 12 && b != 16) return QEXT_E_UNSUPPORTED;
    if (p->gpu_q80 ? b != 16 : (p->q != 4 && p->q != 16 && p->q != 64)) return QEXT_E_UNSUPPORTED;
    if (p->gpu_q80 && flags) return QEXT_E_INVAL;
    if (nblocks == 0) return QEXT_OK;
    if (nsamples > UINT64_MAX / 16 || nblocks > (nsamples * b) / p->n) return QEXT_E_INVAL;
    if (!x_samples || !y_samples || !out || !aligned(x_samples, 16) || !aligned(y_samples, 16) || !aligned(out, 4))
        return QEXT_E_INVAL;
    const qext::NvtxRange range("qext ingest+extract (fused)");
    if (p->gpu_q80)  // 16-bit samples are the packed stream (sample s = bits [16s, 16s + 16))
        return qext::launch_extract_q80(p, reinterpret_cast<const uint32_t *>(x_samples),
                                        reinterpret_cast<const uint32_t *>(y_samples), nblocks, out, stream);
    return qext::launch_extract_samples(p, b, x_samples, y_samples, nsamples, nblocks, out, stream, flags);
}

int qext_pack_samples(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint32_t *out,
                      qext_cuda_stream stream) {
    if (b < 1 || b > 16) return QEXT_E_INVAL;
    if (nsamples == 0) return QEXT_OK;
    if (!samples || !out || !aligned(samples, 2) || !aligned(out, 4)) return QEXT_E_INVAL;
    const qext::NvtxRange range("qext ingest (pack)");
    return qext::launch_pack(b, samples, nsamples, out, stream);
}

int qext_device_status(int *status) {
    if (!status) return QEXT_E_INVAL;
    return qext::read_device_status(status);
}

}  // extern "C"
