// C ABI of include/hm.h: argument checks, call-order state machine, the
// level loop of Algorithm 4.1, apply, the Section 5 error estimate and exports.
#include "ctx.cuh"
#include "philox.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>

namespace hm {
thread_local cudaStream_t g_alloc_stream = nullptr;
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_allocs{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }
long long allocs_so_far() { return g_allocs.load(std::memory_order_relaxed); }

// allocations left before the injected failure; -1: injection off
static std::atomic<long long> g_alloc_countdown{[] {
    const char *s = getenv("HM_FAULT_ALLOC_AFTER");
    return s && *s ? atoll(s) : -1ll;
}()};
bool fault_alloc_now() {
    if (g_alloc_countdown.load(std::memory_order_relaxed) < 0) return false;
    return g_alloc_countdown.fetch_sub(1, std::memory_order_relaxed) == 0;  // fires once, then stays off
}
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}

using namespace hm;

namespace {

hm_status finish(hm_ctx *c, const Err &e) {
    if (e) {
        c->last_error = e.msg;
        return e.code;
    }
    return HM_OK;
}

hm_status bad(hm_ctx *c, hm_status code, const char *msg) {
    if (c) c->last_error = msg;
    return code;
}

__global__ void k_start_vector(int64_t n, unsigned long long seed, double *x) {
    // Philox Gaussian start vector, counter (0, i, 0, 2 << 8), duplicated in both columns
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double z = gauss(seed, 2, 0, 0, (int)i, 0);
    x[i * 2] = z;
    x[i * 2 + 1] = z;
}

__global__ void k_colsq(const double *x, int64_t n, int nrhs, double *out) {
    __shared__ double sh[32];
    for (int j = 0; j < nrhs; ++j) {
        double s = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            s = fma(x[i * nrhs + j], x[i * nrhs + j], s);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) atomicAdd(&out[j], s);
    }
}

__global__ void k_axpby2(const double *a, const double *b, int64_t n, double *out) {
    // out(:,0) = a(:,0) - b(:,0); out(:,1) = b(:,1)
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i * 2] = a[i * 2] - b[i * 2];
    out[i * 2 + 1] = b[i * 2 + 1];
}

__global__ void k_scale2(double *x, int64_t n, double s0, double s1) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i * 2] *= s0;
    x[i * 2 + 1] *= s1;
}

Err op_apply_vectors(hm_ctx *c, const hm_op *op, const double *x, double *y, int trans, DBuf &t1, DBuf &t2) {
    // y = A x or A^* x for row-major sorted [n][2] vectors
    if (op->kind == HM_OP_CALLBACK) {
        HM_TRY(ensure(t1, c->n * 2 * sizeof(double)));
        HM_TRY(ensure(t2, c->n * 2 * sizeof(double)));
        // sorted row-major -> original column-major
        HM_TRY(permute_rows(c, x, t1.as<double>(), 2, false));
        const int rc = op->apply(op->user, trans, t1.as<double>(), t2.as<double>(), 2, (void *)c->st);
        if (rc) return fail(HM_EOP, "black-box operator returned " + std::to_string(rc));
        return permute_rows(c, t2.as<double>(), y, 2, true);
    }
    return op_apply_dense_vectors(c, op, x, y, 2, trans);
}

}  // namespace

extern "C" {

hm_status hm_create(hm_ctx **out, const hm_config *cfg, void *stream) {
    if (!out || !cfg) return HM_EINVAL;
    *out = nullptr;
    if (cfg->d < 1 || cfg->d > 3 || cfg->leaf_size < 0 || cfg->r < 1 || cfg->r > 64) return HM_EINVAL;
    if (cfg->rank > cfg->r || cfg->rank < 0 || !(cfg->tol >= 0.0) || !(cfg->tol < INFINITY)) return HM_EINVAL;
    if (cfg->tol > 0.0 && (cfg->oversample < 0 || cfg->oversample >= cfg->r)) return HM_EINVAL;
    if (cfg->precision != HM_FP64 && cfg->precision != HM_MIXED_BF16X6 && cfg->precision != HM_MIXED_BF16X6_F32)
        return HM_EINVAL;
    if (cfg->uniform_depth < 0 || cfg->uniform_depth > QBITS) return HM_EINVAL;
    if (cfg->format != HM_FORMAT_H1 && cfg->format != HM_FORMAT_UNIFORM_H1 && cfg->format != HM_FORMAT_H2)
        return HM_EINVAL;
    if (cfg->format == HM_FORMAT_H2 && cfg->keep_samples) return HM_ENOTSUP;
    hm_ctx *c = new (std::nothrow) hm_ctx();
    if (!c) return HM_ENOMEM;
    c->cfg = *cfg;
    c->st = (cudaStream_t)stream;
    std::memset(&c->info, 0, sizeof(c->info));
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        c->dev = dev;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    cudaGetLastError();
    *out = c;
    return HM_OK;
}

hm_status hm_destroy(hm_ctx *c) {
    if (!c) return HM_OK;
    {
        DeviceScope ds(c->dev);
        StreamScope ss(c->st);
        cudaStream_t st = c->st, cst0 = c->color_st[0], cst1 = c->color_st[1];
        delete c;
        cudaStreamSynchronize(st);
        if (cst0) cudaStreamDestroy(cst0);
        if (cst1) cudaStreamDestroy(cst1);
    }
    cudaGetLastError();
    return HM_OK;
}

hm_status hm_tree_build(hm_ctx *c, const double *points_dev, int64_t n, int leaf_size) {
    if (!c) return HM_EINVAL;
    if (!points_dev || n < 1 || n > (1ll << 30)) return bad(c, HM_EINVAL, "tree_build: bad points or n");
    if (leaf_size < 0 || (leaf_size == 0 && c->cfg.leaf_size < 1))
        return bad(c, HM_EINVAL, "tree_build: leaf_size < 0, or 0 with no leaf size in the configuration");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    c->leaf_size = leaf_size > 0 ? leaf_size : c->cfg.leaf_size;
    c->colorings.clear();
    c->factors.clear();
    c->kept.clear();
    c->leaf = Leaf();
    c->plan = ApplyPlan();
    c->xdf.release();
    c->stage = 0;
    Err e = build_tree(c, points_dev, n);
    if (e) return finish(c, e);
    c->colorings.resize(c->L + 2);
    c->box_colorings.clear();
    c->box_colorings.resize(c->L + 1);
    c->factors.resize(c->L + 1);
    c->stage = 1;
    return HM_OK;
}

hm_status hm_color(hm_ctx *c, int level, int *n_colors) {
    if (!c) return HM_EINVAL;
    if (c->stage < 1) return bad(c, HM_ESTATE, "color: build the tree first");
    const bool leaf = level == HM_LEVEL_LEAF;
    if (!leaf && (level < 2 || level > c->L)) return bad(c, HM_EINVAL, "color: level out of range");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    Err e = color_cut(c, level, leaf);
    if (e) return finish(c, e);
    if (n_colors) *n_colors = c->colorings[leaf ? c->L + 1 : level].n_colors;
    return HM_OK;
}

hm_status hm_color_boxes(hm_ctx *c, int level, int *n_colors) {
    if (!c) return HM_EINVAL;
    if (c->stage < 1) return bad(c, HM_ESTATE, "color_boxes: build the tree first");
    if (level < 2 || level > c->L) return bad(c, HM_EINVAL, "color_boxes: level out of range");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    Err e = color_boxes(c, level, c->st, c->scan_tmp);
    if (e) return finish(c, e);
    if (n_colors) *n_colors = c->box_colorings[level].n_colors;
    return HM_OK;
}

hm_status hm_sample(hm_ctx *c, const hm_op *op, int level) {
    if (!c || !op) return HM_EINVAL;
    if (c->stage < 1) return bad(c, HM_ESTATE, "sample: build the tree first");
    const bool leaf = level == HM_LEVEL_LEAF;
    if (!leaf && (level < 2 || level > c->L)) return bad(c, HM_EINVAL, "sample: level out of range");
    const int idx = leaf ? c->L + 1 : level;
    if (!c->colorings[idx].done) return bad(c, HM_ESTATE, "sample: colour the level first");
    if (op->kind == HM_OP_CALLBACK && !op->apply) return bad(c, HM_EINVAL, "sample: null callback");
    if (op->kind == HM_OP_DENSE && !op->dense_dev) return bad(c, HM_EINVAL, "sample: null dense matrix");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    Err e;
    if (!leaf) e = make_gaussians(c, level);
    if (!e) e = sample_level(c, op, level, leaf);
    if (!e) {
        cudaError_t ce = cudaStreamSynchronize(c->st);
        if (ce != cudaSuccess) e = fail(HM_ECUDA, cudaGetErrorString(ce));
    }
    return finish(c, e);
}

static Err keep_current(hm_ctx *c, int idx, bool leaf) {
    if (!c->cfg.keep_samples) return ok();
    if ((int)c->kept.size() < c->L + 2) c->kept.resize(c->L + 2);
    Samples &k = c->kept[idx];
    const Samples &s = c->cur;
    k.level = s.level;
    k.chi = s.chi;
    k.cols = s.cols;
    const size_t bytes = (size_t)s.chi * c->n * s.cols * sizeof(double);
    HM_TRY(alloc(k.Y, bytes));
    HM_CUDA(cudaMemcpyAsync(k.Y.p, s.Y.p, bytes, cudaMemcpyDeviceToDevice, c->st));
    if (!leaf) {
        HM_TRY(alloc(k.Z, bytes));
        HM_CUDA(cudaMemcpyAsync(k.Z.p, s.Z.p, bytes, cudaMemcpyDeviceToDevice, c->st));
    }
    return ok();
}

// The colourings (Section 4.1.1) depend on the tree alone, so two host
// threads compute them while the calling thread samples, peels and compresses
// the levels already coloured: one colours levels 2..L in order, the other the
// leaf level, each on a stream of its own of the highest priority (their
// one-CTA DSatur launches get the next free SM).  wait(idx) returns once
// colouring idx is complete on the device; its Coloring is then only read.
class ColorAhead {
public:
    explicit ColorAhead(hm_ctx *c) : c_(c), state_(c->L + 2, 0), errs_(c->L + 2) {}
    ~ColorAhead() {
        stop_ = true;
        for (auto &t : th_)
            if (t.joinable()) t.join();
    }
    Err start() {
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        for (int w = 0; w < 2; ++w)
            if (!c_->color_st[w]) {
                int least = 0, greatest = 0;
                HM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
                HM_CUDA(cudaStreamCreateWithPriority(&c_->color_st[w], cudaStreamNonBlocking, greatest));
            }
        // worker 0: levels 2..L; worker 1: the leaf level at index L + 1
        std::vector<int> levels;
        for (int l = 2; l <= c_->L; ++l) levels.push_back(l);
        try {
            th_[0] = std::thread([this, dev, levels] { run(dev, 0, levels); });
            th_[1] = std::thread([this, dev] { run(dev, 1, std::vector<int>{c_->L + 1}); });
        } catch (const std::exception &e) {
            stop_ = true;
            return fail(HM_ENOMEM, std::string("colour: cannot start the colouring threads: ") + e.what());
        }
        return ok();
    }
    // blocks until colouring idx is done; adds the blocked host time to *secs
    Err wait(int idx, double *secs) {
        const auto t0 = std::chrono::steady_clock::now();
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return state_[idx] != 0; });
        *secs += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return state_[idx] == 2 ? errs_[idx] : ok();
    }

private:
    void run(int dev, int w, std::vector<int> order) {
        Err e;
        if (cudaSetDevice(dev) != cudaSuccess) e = fail(HM_ECUDA, "colour: cudaSetDevice failed");
        StreamScope ss(c_->color_st[w]);
        for (int idx : order) {
            const bool leaf = idx == c_->L + 1;
            if (!e && stop_) e = fail(HM_ECUDA, "colour: cancelled");
            if (!e && !c_->colorings[idx].done)
                e = color_cut(c_, leaf ? 0 : idx, leaf, c_->color_st[w], c_->color_scan_tmp[w]);
            if (!e && !leaf && c_->cfg.format != HM_FORMAT_H1 && !c_->box_colorings[idx].done)
                e = color_boxes(c_, idx, c_->color_st[w], c_->color_scan_tmp[w]);
            {
                std::lock_guard<std::mutex> lk(m_);
                state_[idx] = e ? 2 : 1;
                errs_[idx] = e;  // after a failure every later level of this worker reports it too
            }
            cv_.notify_all();
        }
    }
    hm_ctx *c_;
    std::thread th_[2];
    std::mutex m_;
    std::condition_variable cv_;
    std::vector<int> state_;  // 0 pending, 1 done, 2 failed
    std::vector<Err> errs_;
    std::atomic<bool> stop_{false};
};

static Err compress_all(hm_ctx *c, const hm_op *op) {
    const auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = launches_so_far();
    c->t_tc = 0.0;
    c->tc_evals = 0;
    c->bb_tc_levels = 0;
    c->bb_fp64_levels = 0;
    {  // the pool's high-water mark from here on
        cudaMemPool_t pool;
        uint64_t zero = 0;
        if (cudaDeviceGetDefaultMemPool(&pool, c->dev) == cudaSuccess)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
        cudaGetLastError();
    }
    for (auto &e : c->ev_update) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    c->ev_update.clear();
    if (c->peel_macs.p) HM_CUDA(cudaMemsetAsync(c->peel_macs.p, 0, sizeof(unsigned long long), c->st));
    // (phase, start event, end event) triples, read once at the end
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    int cur_phase = -1;
    cudaEvent_t cur_start = nullptr;
    auto begin = [&](int ph) -> Err {
        HM_CUDA(cudaEventCreate(&cur_start));
        HM_CUDA(cudaEventRecord(cur_start, c->st));
        cur_phase = ph;
        return ok();
    };
    auto end = [&]() -> Err {
        cudaEvent_t e;
        HM_CUDA(cudaEventCreate(&e));
        HM_CUDA(cudaEventRecord(e, c->st));
        ev.push_back({cur_phase, {cur_start, e}});
        cur_start = nullptr;
        return ok();
    };
#define PHASE(ph, expr)                        \
    do {                                       \
        if ((err = begin(ph))) break;          \
        if ((err = (expr))) { end(); break; }  \
        if ((err = end())) break;              \
    } while (0)
    Err err;
    int64_t cols_total = 0;
    double color_wait = 0.0;
    double phase_uniform[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // uniform levels time their phases themselves
    ColorAhead ahead(c);
    err = ahead.start();
    for (int l = 2; l <= c->L && !err; ++l) {
        if ((err = ahead.wait(l, &color_wait))) break;
        const Coloring &g = c->colorings[l];
        if (c->cfg.format == HM_FORMAT_H2) {  // Section 4.3: every cut, also one without pairs (its far field)
            if ((err = h2_level(c, op, l, phase_uniform))) break;
            if (g.n_pairs > 0 && g.n_colors > 0)
                cols_total += (int64_t)c->box_colorings[l].n_colors * c->cfg.r + (int64_t)g.n_colors * g.m_cols;
            continue;
        }
        if (g.n_pairs == 0 || g.n_colors == 0) {
            c->factors[l] = Factors();
            c->factors[l].done = true;
            continue;
        }
        if (c->cfg.format == HM_FORMAT_UNIFORM_H1) {  // Section 4.2: two stages per level
            if ((err = uniform_level(c, op, l, phase_uniform))) break;
            cols_total += (int64_t)c->box_colorings[l].n_colors * c->cfg.r + (int64_t)g.n_colors * g.m_cols;
            continue;
        }
        PHASE(1, make_gaussians(c, l));
        if (err) break;
        PHASE(2, sample_level(c, op, l, false));
        if (err) break;
        cols_total += 2ll * g.n_colors * g.m_cols;
        PHASE(3, peel_level(c, l, false));
        if (err) break;
        if ((err = keep_current(c, l, false))) break;
        PHASE(4, bases_and_cores(c, l));
    }
    if (!err) err = ahead.wait(c->L + 1, &color_wait);
    if (!err) {
        const Coloring &g = c->colorings[c->L + 1];
        PHASE(5, sample_level(c, op, HM_LEVEL_LEAF, true));
        if (!err) {
            cols_total += (int64_t)g.n_colors * g.m_cols;
            PHASE(6, peel_level(c, 0, true));
            if (!err) err = keep_current(c, c->L + 1, true);
            if (!err) PHASE(6, extract_leaf(c));
        }
    }
    if (!err && c->cfg.format == HM_FORMAT_H2) err = h2_finish(c);
    if (!err) err = build_apply_plan(c);
#undef PHASE
    if (cur_start) cudaEventDestroy(cur_start);
    cudaError_t ce = cudaStreamSynchronize(c->st);
    if (!err && ce != cudaSuccess) err = fail(HM_ECUDA, std::string("compress: ") + cudaGetErrorString(ce));
    double phase[8] = {color_wait, phase_uniform[1], phase_uniform[2], phase_uniform[3], phase_uniform[4], 0, 0, 0};
    for (auto &e : ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess) phase[e.first] += ms * 1e-3;
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    double t_update = 0.0;
    for (auto &e : c->ev_update) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) t_update += ms * 1e-3;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    c->ev_update.clear();
    unsigned long long macs = 0;
    if (!err && c->peel_macs.p && cudaMemcpy(&macs, c->peel_macs.p, sizeof(macs), cudaMemcpyDeviceToHost) != cudaSuccess)
        macs = 0;
    cudaGetLastError();
    if (err) return err;
    const double ts = phase[2] + phase[5];
    c->t_sample = ts;
    hm_info &in = c->info;
    std::memset(&in, 0, sizeof(in));
    for (int k = 0; k < 7; ++k) in.seconds_phase[k] = phase[k];
    in.seconds_phase[7] = c->t_tc;
    in.n = c->n;
    in.L = c->L;
    for (auto &lv : c->levels) in.n_boxes += lv.nb;
    int64_t floats = 0;
    in.kernel_launches = launches_so_far() - launches0;
    in.tc_kernel_evals = c->tc_evals;
    in.bb_tc_levels = c->bb_tc_levels;
    in.bb_fp64_levels = c->bb_fp64_levels;
    in.seconds_peel_update = t_update;
    in.peel_update_macs = (int64_t)macs;
    in.rank = c->rank_arg;
    in.tol = c->tol;
    for (int l = 2; l <= c->L && l < 31; ++l) {
        in.act_rows[l] = c->colorings[l].n_act_rows;
        in.colors[l] = c->colorings[l].n_colors;
        in.pairs[l] = c->colorings[l].n_pairs;
        in.vertices[l] = c->colorings[l].n_vertices;
        const Factors &f = c->factors[l];
        floats += f.nU + f.nV + f.nB + f.nUt + f.nVt;
        in.max_rank = std::max(in.max_rank, f.max_k);
    }
    if (c->L + 1 < 32) {
        in.act_rows[c->L + 1] = c->colorings[c->L + 1].n_act_rows;
        in.colors[c->L + 1] = c->colorings[c->L + 1].n_colors;
        in.pairs[c->L + 1] = c->colorings[c->L + 1].n_pairs;
        in.vertices[c->L + 1] = c->colorings[c->L + 1].n_vertices;
    }
    floats += c->leaf.nD;
    in.factor_floats = floats;
    in.matvec_cols = cols_total;
    in.seconds_sample = ts;
    in.seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return ok();
}

hm_status hm_compress(hm_ctx *c, const hm_op *op, double tol, int rank) {
    if (!c || !op) return HM_EINVAL;
    if (op->kind == HM_OP_CALLBACK && !op->apply) return bad(c, HM_EINVAL, "compress: null callback");
    if (op->kind == HM_OP_DENSE && !op->dense_dev) return bad(c, HM_EINVAL, "compress: null dense matrix");
    if (op->kind == HM_OP_KERNEL && (op->kernel < HM_K_LOG || op->kernel > HM_K_EXP))
        return bad(c, HM_EINVAL, "compress: unknown kernel");
    if (!(tol >= 0.0) || !(tol < INFINITY) || rank < 0) return bad(c, HM_EINVAL, "compress: tol < 0 or rank < 0");
    if (tol == 0.0 && rank == 0) {  // the configuration's defaults
        tol = c->cfg.tol;
        rank = c->cfg.rank;
    }
    const int r = c->cfg.r, p = c->cfg.oversample;
    if (tol == 0.0 && rank == 0) return bad(c, HM_EINVAL, "compress: neither a tolerance nor a rank");
    if (rank > r) return bad(c, HM_EINVAL, "compress: rank > r");
    if (tol > 0.0 && (p < 0 || p >= r)) return bad(c, HM_EINVAL, "compress: oversampling p not in 0..r-1");
    if (c->stage < 1) return bad(c, HM_ESTATE, "compress: build the tree first");
    c->tol = tol;
    c->rank_arg = rank;
    c->rank_fixed = tol > 0.0 ? 0 : rank;
    c->kcap = tol > 0.0 ? (rank > 0 ? std::min(r - p, rank) : r - p) : r;
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    c->stage = 1;
    c->kept.clear();
    Err e = compress_all(c, op);
    if (e) return finish(c, e);
    c->stage = 2;
    return HM_OK;
}

hm_status hm_apply(hm_ctx *c, const double *x, double *y, int64_t nrhs, int trans) {
    if (!c) return HM_EINVAL;
    if (c->stage < 2) return bad(c, HM_ESTATE, "apply: compress first");
    if (!x || !y || nrhs < 1 || nrhs > 64) return bad(c, HM_EINVAL, "apply: bad vectors");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    DBuf xs, ys;
    Err e = alloc(xs, c->n * nrhs * sizeof(double));
    if (!e) e = alloc(ys, c->n * nrhs * sizeof(double));
    if (!e) e = permute_rows(c, x, xs.as<double>(), (int)nrhs, true);
    if (!e) e = apply_sorted(c, xs.as<double>(), ys.as<double>(), (int)nrhs, trans ? 1 : 0);
    if (!e) e = permute_rows(c, ys.as<double>(), y, (int)nrhs, false);
    return finish(c, e);
}

hm_status hm_relerr(hm_ctx *c, const hm_op *op, int iters, double *err) {
    if (!c || !op || !err) return HM_EINVAL;
    if (c->stage < 2) return bad(c, HM_ESTATE, "relerr: compress first");
    if (iters < 1) return bad(c, HM_EINVAL, "relerr: iters < 1");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    const int64_t n = c->n;
    DBuf x, ax, hx, w, z1, z2, sq, t1, t2;
    Err e;
    auto run = [&]() -> Err {
        HM_TRY(alloc(x, n * 2 * sizeof(double)));
        HM_TRY(alloc(ax, n * 2 * sizeof(double)));
        HM_TRY(alloc(hx, n * 2 * sizeof(double)));
        HM_TRY(alloc(w, n * 2 * sizeof(double)));
        HM_TRY(alloc(sq, 2 * sizeof(double)));
        const int g = ceil_div(n, 256);
        k_start_vector<<<g, 256, 0, c->st>>>(n, (unsigned long long)c->cfg.seed + 1ull, x.as<double>()); ::hm::count_launch();
        HM_LAUNCH("start_vector");
        double lam[2] = {0, 0};
        {  // normalise the start vector
            HM_CUDA(cudaMemsetAsync(sq.p, 0, 2 * sizeof(double), c->st));
            k_colsq<<<64, 256, 0, c->st>>>(x.as<double>(), n, 2, sq.as<double>()); ::hm::count_launch();
            double h[2];
            HM_CUDA(cudaMemcpyAsync(h, sq.p, sizeof(h), cudaMemcpyDeviceToHost, c->st));
            HM_CUDA(cudaStreamSynchronize(c->st));
            k_scale2<<<g, 256, 0, c->st>>>(x.as<double>(), n, 1.0 / sqrt(h[0]), 1.0 / sqrt(h[1])); ::hm::count_launch();
        }
        for (int it = 0; it < iters; ++it) {
            // w = M x: col 0 (A~ - A) x0, col 1 A x1
            HM_TRY(op_apply_vectors(c, op, x.as<double>(), ax.as<double>(), 0, t1, t2));
            HM_TRY(apply_sorted(c, x.as<double>(), hx.as<double>(), 2, 0));
            k_axpby2<<<g, 256, 0, c->st>>>(hx.as<double>(), ax.as<double>(), n, w.as<double>()); ::hm::count_launch();
            // x = M^* w
            HM_TRY(op_apply_vectors(c, op, w.as<double>(), ax.as<double>(), 1, t1, t2));
            HM_TRY(apply_sorted(c, w.as<double>(), hx.as<double>(), 2, 1));
            k_axpby2<<<g, 256, 0, c->st>>>(hx.as<double>(), ax.as<double>(), n, x.as<double>()); ::hm::count_launch();
            HM_LAUNCH("power step");
            HM_CUDA(cudaMemsetAsync(sq.p, 0, 2 * sizeof(double), c->st));
            k_colsq<<<64, 256, 0, c->st>>>(x.as<double>(), n, 2, sq.as<double>()); ::hm::count_launch();
            double h[2];
            HM_CUDA(cudaMemcpyAsync(h, sq.p, sizeof(h), cudaMemcpyDeviceToHost, c->st));
            HM_CUDA(cudaStreamSynchronize(c->st));
            lam[0] = sqrt(h[0]);
            lam[1] = sqrt(h[1]);
            k_scale2<<<g, 256, 0, c->st>>>(x.as<double>(), n, lam[0] > 0 ? 1.0 / lam[0] : 0.0,
                                           lam[1] > 0 ? 1.0 / lam[1] : 0.0); ::hm::count_launch();
        }
        *err = lam[1] > 0.0 ? sqrt(lam[0]) / sqrt(lam[1]) : 0.0;
        return ok();
    };
    e = run();
    return finish(c, e);
}

hm_status hm_get_info(hm_ctx *c, hm_info *out) {
    if (!c || !out) return HM_EINVAL;
    *out = c->info;
    out->launches_total = launches_so_far();
    out->device_allocs = allocs_so_far();
    {
        cudaMemPool_t pool;
        uint64_t v = 0;
        if (c->dev >= 0 && cudaDeviceGetDefaultMemPool(&pool, c->dev) == cudaSuccess) {
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) == cudaSuccess) out->pool_used_bytes = v;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v) == cudaSuccess) out->pool_peak_bytes = v;
        }
        cudaGetLastError();
    }
    out->leaf_size = c->leaf_size;
    if (c->stage >= 1) {
        out->n = c->n;
        out->L = c->L;
        int nb = 0;
        for (auto &lv : c->levels) nb += lv.nb;
        out->n_boxes = nb;
    }
    return HM_OK;
}

hm_status hm_export(hm_ctx *c, int what, int level, void *host_buf, size_t *bytes) {
    if (!c || !bytes) return HM_EINVAL;
    if (c->stage < 1) return bad(c, HM_ESTATE, "export: build the tree first");
    DeviceScope ds(c->dev);
    StreamScope ss(c->st);
    const bool leaf = level == HM_LEVEL_LEAF;
    const int cl = leaf ? c->L : level;
    const int idx = leaf ? c->L + 1 : level;
    std::vector<std::pair<const void *, size_t>> parts;  // device pointers, bytes
    std::vector<char> hostpart;                          // prepared on the host instead
    auto need_cut = [&]() { return cl >= 0 && cl <= c->L; };
    switch (what) {
    case HM_X_PERM: parts.push_back({c->perm.p, (size_t)c->n * sizeof(int)}); break;
    case HM_X_LEVEL_BOXES:
        if (level < 0 || level > c->L) return bad(c, HM_EINVAL, "export: level");
        parts.push_back({c->levels[level].box.p, (size_t)c->levels[level].nb * BOX_FIELDS * sizeof(int)});
        break;
    case HM_X_CUT:
    case HM_X_NEAR:
    case HM_X_INTER: {
        if (!need_cut()) return bad(c, HM_EINVAL, "export: level");
        const Cut &cu = c->cuts[cl];
        if (what == HM_X_CUT) {
            std::vector<int> ent;
            Err e = to_host(ent, cu.ent.p, (size_t)cu.nc * ENT_FIELDS, c->st);
            if (e) return finish(c, e);
            std::vector<int> o(2 * (size_t)cu.nc);
            for (int i = 0; i < cu.nc; ++i) {
                o[2 * i] = ent[(size_t)i * ENT_FIELDS];
                o[2 * i + 1] = ent[(size_t)i * ENT_FIELDS + 1];
            }
            hostpart.assign((char *)o.data(), (char *)(o.data() + o.size()));
        } else {
            const bool nr = what == HM_X_NEAR;
            parts.push_back({nr ? cu.near_ptr.p : cu.int_ptr.p, (size_t)(cu.nc + 1) * sizeof(int)});
            parts.push_back({nr ? cu.near_idx.p : cu.int_idx.p, (size_t)(nr ? cu.n_near : cu.n_int) * sizeof(int)});
        }
        break;
    }
    case HM_X_PAIR_VERTEX:
    case HM_X_VERTEX_COLOR:
    case HM_X_VERTEX_BETA:
    case HM_X_VERTEX_DEGREE: {
        if (idx < 0 || idx >= (int)c->colorings.size() || !c->colorings[idx].done)
            return bad(c, HM_ESTATE, "export: level not coloured");
        const Coloring &g = c->colorings[idx];
        if (what == HM_X_PAIR_VERTEX) parts.push_back({g.pair_vertex.p, (size_t)g.n_pairs * sizeof(int)});
        if (what == HM_X_VERTEX_COLOR) parts.push_back({g.vertex_color.p, (size_t)g.n_vertices * sizeof(int)});
        if (what == HM_X_VERTEX_BETA) parts.push_back({g.vertex_beta.p, (size_t)g.n_vertices * sizeof(int)});
        if (what == HM_X_VERTEX_DEGREE) parts.push_back({g.vertex_degree.p, (size_t)g.n_vertices * sizeof(int)});
        break;
    }
    case HM_X_BOX_VERTEX_BOX:
    case HM_X_BOX_COLOR:
    case HM_X_BOX_DEGREE: {
        if (level < 2 || level >= (int)c->box_colorings.size() || !c->box_colorings[level].done)
            return bad(c, HM_ESTATE, "export: boxes of that level not coloured");
        const Coloring &g = c->box_colorings[level];
        const void *src = what == HM_X_BOX_VERTEX_BOX ? g.pair_alpha.p
                          : (what == HM_X_BOX_COLOR ? g.vertex_color.p : g.vertex_degree.p);
        parts.push_back({src, (size_t)g.n_vertices * sizeof(int)});
        break;
    }
    case HM_X_H2_RANKS:
    case HM_X_H2_SIGMA: {
        if (c->cfg.format != HM_FORMAT_H2 || c->stage < 2 || level < 2 || level > c->L ||
            !c->factors[level].has_bases)
            return bad(c, HM_ESTATE, "export: no H^2 bases at that level");
        const Factors &f = c->factors[level];
        if (what == HM_X_H2_RANKS) {
            parts.push_back({f.ekU.p, (size_t)f.nc * sizeof(int)});
            parts.push_back({f.ekV.p, (size_t)f.nc * sizeof(int)});
        } else {
            parts.push_back({f.eS.p, (size_t)f.nc * 2 * c->cfg.r * sizeof(double)});
        }
        break;
    }
    case HM_X_GAUSS:
        if (c->gauss_level != level) return bad(c, HM_ESTATE, "export: Gaussians of that level are not current");
        parts.push_back({c->GO.p, (size_t)c->n * c->cfg.r * sizeof(double)});
        parts.push_back({c->GP.p, (size_t)c->n * c->cfg.r * sizeof(double)});
        break;
    case HM_X_SAMPLE_Y:
    case HM_X_SAMPLE_Z: {
        const Samples *s = nullptr;
        if (c->cfg.keep_samples && idx < (int)c->kept.size() && c->kept[idx].Y.p) s = &c->kept[idx];
        else if (c->cur.level == level) s = &c->cur;
        if (!s) return bad(c, HM_ESTATE, "export: no samples for that level");
        if (what == HM_X_SAMPLE_Z && leaf) return bad(c, HM_EINVAL, "export: the leaf step has no Z");
        parts.push_back({what == HM_X_SAMPLE_Y ? s->Y.p : s->Z.p, (size_t)s->chi * c->n * s->cols * sizeof(double)});
        break;
    }
    case HM_X_PAIR_RANKS:
    case HM_X_FACTORS:
    case HM_X_FACTOR_OFFS: {
        if (level < 2 || level >= (int)c->factors.size() || !c->factors[level].done)
            return bad(c, HM_ESTATE, "export: no factors for that level");
        const Factors &f = c->factors[level];
        const int64_t np = f.n_pairs;
        if (what == HM_X_FACTORS) {
            parts.push_back({f.U.p, (size_t)f.nU * sizeof(double)});
            parts.push_back({f.V.p, (size_t)f.nV * sizeof(double)});
            parts.push_back({f.B.p, (size_t)f.nB * sizeof(double)});
        } else if (np > 0) {
            if (what == HM_X_PAIR_RANKS) {
                std::vector<int> ku, kv;
                Err e = to_host(ku, f.kU.p, np, c->st);
                if (!e) e = to_host(kv, f.kV.p, np, c->st);
                if (e) return finish(c, e);
                std::vector<int> o(2 * np);
                for (int64_t p = 0; p < np; ++p) {
                    o[2 * p] = ku[p];
                    o[2 * p + 1] = kv[p];
                }
                hostpart.assign((char *)o.data(), (char *)(o.data() + o.size()));
            } else {
                std::vector<int64_t> a, b, d;
                Err e = to_host(a, f.offU.p, np, c->st);
                if (!e) e = to_host(b, f.offV.p, np, c->st);
                if (!e) e = to_host(d, f.offB.p, np, c->st);
                if (e) return finish(c, e);
                std::vector<int64_t> o(3 * np);
                for (int64_t p = 0; p < np; ++p) {
                    o[3 * p] = a[p];
                    o[3 * p + 1] = b[p];
                    o[3 * p + 2] = d[p];
                }
                hostpart.assign((char *)o.data(), (char *)(o.data() + o.size()));
            }
        }
        break;
    }
    case HM_X_LEAF_D:
        if (!c->leaf.done) return bad(c, HM_ESTATE, "export: no leaf blocks");
        parts.push_back({c->leaf.D.p, (size_t)c->leaf.nD * sizeof(double)});
        break;
    default: return bad(c, HM_EINVAL, "export: unknown selector");
    }
    size_t need = hostpart.size();
    for (auto &pp : parts) need += pp.second;
    if (!host_buf) {
        *bytes = need;
        return HM_OK;
    }
    if (*bytes < need) return bad(c, HM_EINVAL, "export: buffer too small");
    char *dst = (char *)host_buf;
    if (!hostpart.empty()) {
        std::memcpy(dst, hostpart.data(), hostpart.size());
        dst += hostpart.size();
    }
    for (auto &pp : parts) {
        if (pp.second) {
            cudaError_t ce = cudaMemcpyAsync(dst, pp.first, pp.second, cudaMemcpyDeviceToHost, c->st);
            if (ce != cudaSuccess) return bad(c, HM_ECUDA, cudaGetErrorString(ce));
        }
        dst += pp.second;
    }
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return bad(c, HM_ECUDA, "export: copy failed");
    *bytes = need;
    return HM_OK;
}

const char *hm_last_error(const hm_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

}  // extern "C"
