// hm_apply_noalloc: the apply of the compressed operator (same kernels and
// results as hm_apply) without any device allocation.
//
// Some callers cannot allocate device memory at the point where they apply
// the operator: a serving loop whose process has handed all free device
// memory to another framework's caching allocator, or a latency-critical loop
// that must not wait on cudaMalloc/cudaFree or risk an out-of-memory failure
// in the middle of a request.  For them this entry point takes its scratch
// (the permuted input and output vectors, the per-pair intermediate products
// and their offsets, and the level table) from one file-scope device array of
// HM_APPLY_NOALLOC_SCRATCH_BYTES bytes that the library holds on every GPU
// that loads it, until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it, so that first
// call should come before any stream capture.  Every call shares the array:
// calls that overlap on the GPU (on different streams or host threads) race
// on it.  Each call overwrites every part of the scratch it reads, so nothing
// has to start at zero.
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

// Bump allocator over the array: 256-byte aligned slices, bounds-checked.
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <class T> Err take(T **p, size_t count) {
        const size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
        if (used + bytes > (size_t)HM_APPLY_NOALLOC_SCRATCH_BYTES)
            return fail(HM_ENOTSUP, "apply_noalloc: the request needs more than the " +
                                        std::to_string((size_t)HM_APPLY_NOALLOC_SCRATCH_BYTES >> 20) +
                                        " MiB scratch array; use hm_apply");
        *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return ok();
    }
};

Err apply_noalloc(hm_ctx *c, const double *x, double *y, int nrhs, int trans) {
    cudaStream_t st = c->st;
    unsigned char *base = nullptr;
    HM_TRY(scratch_base(&base));
    Carve cv{base};
    double *xs = nullptr, *ys = nullptr;
    HM_TRY(cv.take(&xs, (size_t)c->n * nrhs));
    HM_TRY(cv.take(&ys, (size_t)c->n * nrhs));
    std::vector<ApplyLevel> lv;
    ApplyLevel *lvd = nullptr;
    HM_TRY(cv.take(&lvd, (size_t)c->L + 1));
    HM_TRY(permute_rows(c, x, xs, nrhs, true));
    for (int l = 2; l <= c->L; ++l) {
        if (l >= (int)c->factors.size() || !c->factors[l].done || c->factors[l].n_pairs == 0) continue;
        const Factors &f = c->factors[l];
        const Coloring &g = c->colorings[l];
        const Cut &cu = c->cuts[l];
        const int64_t np = f.n_pairs;
        int64_t *sz = nullptr, *toff = nullptr;
        HM_TRY(cv.take(&sz, (size_t)np + 1));
        HM_TRY(cv.take(&toff, (size_t)np + 1));
        k_toff_sizes<<<ceil_div(np, 256), 256, 0, st>>>(f.kU.as<int>(), f.kV.as<int>(), np, nrhs, trans, sz);
        count_launch();
        HM_LAUNCH("apply_noalloc sizes");
        HM_TRY(scan_exclusive(sz, toff, np, st));
        int64_t tot = 0;
        HM_TRY(read_scalar(tot, toff + np, st));
        double *tq = nullptr;
        HM_TRY(cv.take(&tq, (size_t)std::max<int64_t>(tot, 1)));
        const size_t smem = (size_t)std::max(f.max_k, 1) * nrhs * sizeof(double);
        if (smem > 200 * 1024) return fail(HM_ENOTSUP, "apply_noalloc: too many right-hand sides");
        HM_CUDA(cudaFuncSetAttribute(k_apply_stage1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        k_apply_stage1<<<(int)np, 128, smem, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(), cu.ent.as<int>(), np,
                                                   f.kU.as<int>(), f.kV.as<int>(), f.offU.as<int64_t>(),
                                                   f.offV.as<int64_t>(), f.offB.as<int64_t>(), f.U.as<double>(),
                                                   f.V.as<double>(), f.B.as<double>(), xs, nrhs, trans, toff, tq);
        count_launch();
        HM_LAUNCH("apply_noalloc stage1");
        ApplyLevel a;
        a.pt2ent = cu.pt2ent.as<int>();
        a.ent = cu.ent.as<int>();
        a.int_ptr = cu.int_ptr.as<int>();
        a.int_idx = cu.int_idx.as<int>();
        a.pairT = g.pair_T.as<int>();
        a.kU = f.kU.as<int>();
        a.kV = f.kV.as<int>();
        a.offU = f.offU.as<int64_t>();
        a.offV = f.offV.as<int64_t>();
        a.U = f.U.as<double>();
        a.V = f.V.as<double>();
        a.toff = toff;
        a.tq = tq;
        lv.push_back(a);
    }
    if (!lv.empty())
        HM_CUDA(cudaMemcpyAsync(lvd, lv.data(), lv.size() * sizeof(ApplyLevel), cudaMemcpyHostToDevice, st));
    const Cut &cl = c->cuts[c->L];
    const Coloring &gl = c->colorings[c->L + 1];
    k_apply_stage2<<<cl.nc, 128, 0, st>>>(cl.ent.as<int>(), cl.nc, lvd, (int)lv.size(), cl.near_ptr.as<int>(),
                                          cl.near_idx.as<int>(), gl.pair_T.as<int>(), c->leaf.offD.as<int64_t>(),
                                          c->leaf.D.as<double>(), xs, nrhs, trans, ys);
    count_launch();
    HM_LAUNCH("apply_noalloc stage2");
    HM_TRY(permute_rows(c, ys, y, nrhs, false));
    HM_CUDA(cudaStreamSynchronize(st));
    return ok();
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
    hm::Err e = hm::apply_noalloc(c, x_dev, y_dev, (int)nrhs, trans ? 1 : 0);
    if (e) {
        c->last_error = e.msg;
        return e.code;
    }
    return HM_OK;
}
