// hm_apply_noalloc: the apply of the compressed operator (same kernels and
// results as hm_apply) without any device allocation.
//
// Some callers cannot allocate device memory at the point where they apply
// the operator: a serving loop whose process has handed all free device
// memory to another framework's caching allocator, or a latency-critical loop
// that must not wait on cudaMalloc/cudaFree or risk an out-of-memory failure
// in the middle of a request.  For them this entry point takes its scratch
// (the permuted input and output vectors and the per-pair intermediate
// products) from one file-scope device array of HM_APPLY_NOALLOC_SCRATCH_BYTES
// bytes that the library holds on every GPU that loads it, until the process
// exits.  The offsets it needs were computed once by hm_compress.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current: the call switches to the
// context's device) and caches it.  The call is asynchronous on the context's
// stream.  Every call shares the array: calls that overlap on the GPU (on
// different streams or host threads) race on it.  Each call overwrites every
// part of the scratch it reads, so nothing has to start at zero.
#include "apply_kernels.cuh"

#include <mutex>

namespace hm {

static __device__ __align__(256) unsigned char g_apply_scratch[HM_APPLY_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_mutex;
void *g_ptr[64] = {nullptr};  // device address of the array, per device ordinal

Err scratch_base(unsigned char **out) {
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(HM_ENOTSUP, "apply_noalloc: device ordinal beyond 63");
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        HM_CUDA(cudaGetSymbolAddress(&p, g_apply_scratch));
        g_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_ptr[dev]);
    return ok();
}

// Bump allocator over the array: 256-byte aligned slices (byte offsets),
// bounds-checked before anything is launched.
struct Carve {
    size_t used = 0;
    Err take(size_t *off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        if (used + bytes > (size_t)HM_APPLY_NOALLOC_SCRATCH_BYTES)
            return fail(HM_ENOTSUP, "apply_noalloc: the request needs more than the " +
                                        std::to_string((size_t)HM_APPLY_NOALLOC_SCRATCH_BYTES >> 20) +
                                        " MiB scratch array; use hm_apply");
        *off = used;
        used += bytes;
        return ok();
    }
};

Err apply_noalloc(hm_ctx *c, const double *x, double *y, int nrhs, int trans) {
    Carve cv;
    size_t oxs = 0, oys = 0, ot = 0;
    const size_t vec = (size_t)c->n * nrhs * sizeof(double);
    HM_TRY(cv.take(&oxs, vec));
    HM_TRY(cv.take(&oys, vec));
    HM_TRY(cv.take(&ot, (size_t)std::max<int64_t>(c->plan.t_max, 1) * nrhs * sizeof(double)));
    unsigned char *base = nullptr;
    HM_TRY(scratch_base(&base));
    double *xs = reinterpret_cast<double *>(base + oxs), *ys = reinterpret_cast<double *>(base + oys),
           *t = reinterpret_cast<double *>(base + ot);
    HM_TRY(permute_rows(c, x, xs, nrhs, true));
    HM_TRY(apply_sorted_into(c, xs, ys, nrhs, trans, t));
    return permute_rows(c, ys, y, nrhs, false);
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_apply_noalloc(hm_ctx *c, const double *x_dev, double *y_dev, int64_t nrhs, int trans) {
    if (!c) return HM_EINVAL;
    if (c->stage < 2) {
        c->last_error = "apply_noalloc: compress first";
        return HM_ESTATE;
    }
    if (!x_dev || !y_dev || nrhs < 1 || nrhs > 64) {
        c->last_error = "apply_noalloc: bad vectors";
        return HM_EINVAL;
    }
    if (c->cfg.format == HM_FORMAT_H2) {
        c->last_error = "apply_noalloc: not available for HM_FORMAT_H2 (use hm_apply)";
        return HM_ENOTSUP;
    }
    hm::DeviceScope ds(c->dev);  // the scratch address and the kernels are those of the context's device
    hm::Err e = hm::apply_noalloc(c, x_dev, y_dev, (int)nrhs, trans ? 1 : 0);
    if (e) {
        c->last_error = e.msg;
        return e.code;
    }
    return HM_OK;
}
