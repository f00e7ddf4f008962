// Serving (include/hm.h, hm_server_*): a FIFO of compression jobs admitted by
// estimated device-memory footprint against a byte budget, compressed by a
// pool of worker threads each on the job's own CUDA stream (so the work of
// concurrent jobs overlaps on the GPU), kept resident afterwards for matvecs.
//
// A job's reservation is its estimated peak footprint while it compresses;
// when the compression ends the job's samples, Gaussians, peel copies and
// scratch are freed and the reservation shrinks to what the operator keeps,
// letting queued jobs start.  Admission is head-of-line: the next job in
// submission order starts when a worker is free and its estimate fits.
#include "ctx.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    hm_job_desc desc{};
    std::vector<double> points;  // host copy of the job's points
    size_t est = 0;              // estimated peak footprint while compressing
    int state = HM_JOB_QUEUED;
    hm_status status = HM_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t reserved = 0;
    hm_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    hm_info info{};
    std::mutex apply_mu;
};

// Estimated peak device bytes of one compression: the two sample buffers of
// the widest level (chi colours x n x r doubles each, chi bounded by the
// level's colour count seen on adaptive trees: 16 in 1D, 48 in 2D, 128 in 3D),
// the leaf sample (about 48 colours x n x leaf columns), the coarse-level
// products of the peel (T slots) and the factors (about 2 x 250 r doubles per
// point at most), the points and tree; then a 25% margin.
size_t estimate_bytes(const hm_job_desc &j) {
    const double n = (double)j.n, r = j.cfg.r, d = j.cfg.d;
    const double leaf = j.leaf_size > 0 ? j.leaf_size : std::max(1, j.cfg.leaf_size);
    const double chi = d == 1 ? 16 : (d == 2 ? 48 : 128);
    const double samples = 2.0 * chi * n * r * 8.0;
    const double leafs = 48.0 * n * std::min(2.0 * leaf, 128.0) * 8.0;
    const double peel = 2.0 * chi * n * r * 8.0;
    const double factors = 2.0 * 250.0 * r * n * 8.0;
    const double base = 512.0 * n + (64 << 20);
    return (size_t)(1.25 * (samples + leafs + peel + factors + base));
}

// The bytes a compressed job keeps: factors, leaf blocks, and about 512 bytes
// per point of tree, colouring and apply metadata.
size_t resident_bytes(const hm_info &in) { return (size_t)in.factor_floats * 8 + (size_t)in.n * 512 + (16 << 20); }

// Free what only the compression needed.
void trim_after_compress(hm_ctx *c) {
    hm::StreamScope ss(c->st);
    c->cur = hm::Samples();
    c->kept.clear();
    c->GO.release();
    c->GP.release();
    c->scratch_a.release();
    c->scratch_b.release();
    c->scratch_c.release();
    c->scratch_d.release();
    c->scan_tmp.release();
    c->xdf.release();
    for (auto &f : c->factors) {
        f.U32.release();
        f.V32.release();
        f.B32.release();
        f.U2.release();
        f.V2.release();
        f.B2.release();
    }
}

double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t k = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * (double)v.size()) - 1);
    return v[std::max<size_t>(k, 0)];
}

}  // namespace

struct hm_server {
    int dev = 0;
    size_t budget = 0;
    int slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<int64_t, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_id = 1;
    size_t reserved = 0, max_reserved = 0;
    int running = 0, max_running = 0;
    int64_t submitted = 0, completed = 0, failed = 0, released = 0;
    double first_submit = -1.0, last_done = 0.0;
    std::vector<double> job_lat, apply_lat;
    Clock::time_point t0 = Clock::now();

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void run_job(Job &j) {
        hm_status st = HM_OK;
        double *pts = nullptr;
        if (cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking) != cudaSuccess) st = HM_ECUDA;
        if (st == HM_OK) st = hm_create(&j.ctx, &j.desc.cfg, j.stream);
        const size_t bytes = (size_t)j.desc.n * j.desc.cfg.d * sizeof(double);
        if (st == HM_OK && cudaMallocAsync((void **)&pts, bytes, j.stream) != cudaSuccess) st = HM_ENOMEM;
        if (st == HM_OK &&
            cudaMemcpyAsync(pts, j.points.data(), bytes, cudaMemcpyHostToDevice, j.stream) != cudaSuccess)
            st = HM_ECUDA;
        if (st == HM_OK) st = hm_tree_build(j.ctx, pts, j.desc.n, j.desc.leaf_size);
        if (pts) cudaFreeAsync(pts, j.stream);
        if (st == HM_OK) st = hm_compress(j.ctx, &j.desc.op, j.desc.tol, j.desc.rank);
        if (st == HM_OK) {
            trim_after_compress(j.ctx);
            hm_get_info(j.ctx, &j.info);
            if (cudaStreamSynchronize(j.stream) != cudaSuccess) st = HM_ECUDA;
        }
        cudaGetLastError();
        j.status = st;
        std::vector<double>().swap(j.points);
    }

    void worker() {
        cudaSetDevice(dev);
        for (;;) {
            std::shared_ptr<Job> j;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop || (!queue.empty() && reserved + queue.front()->est <= budget);
                });
                if (stop) return;
                j = queue.front();
                queue.pop_front();
                j->state = HM_JOB_RUNNING;
                j->t_start = now();
                j->reserved = j->est;
                reserved += j->est;
                max_reserved = std::max(max_reserved, reserved);
                ++running;
                max_running = std::max(max_running, running);
            }
            run_job(*j);
            {
                std::lock_guard<std::mutex> lk(mu);
                --running;
                j->t_done = now();
                reserved -= j->reserved;
                if (j->status == HM_OK) {
                    j->state = HM_JOB_READY;
                    j->reserved = std::min(j->est, resident_bytes(j->info));
                    ++completed;
                    last_done = j->t_done;
                    job_lat.push_back(j->t_done - j->t_submit);
                } else {
                    j->state = HM_JOB_FAILED;
                    j->reserved = 0;
                    if (j->ctx) hm_destroy(j->ctx);
                    j->ctx = nullptr;
                    ++failed;
                }
                reserved += j->reserved;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

namespace {

void fill_stats(const Job &j, hm_job_stats *out) {
    if (!out) return;
    out->state = j.state;
    out->status = j.status;
    out->t_submit = j.t_submit;
    out->t_start = j.t_start;
    out->t_done = j.t_done;
    out->reserved_bytes = j.reserved;
    out->estimate_bytes = j.est;
    out->info = j.info;
}

void free_job(Job &j) {
    if (j.ctx) hm_destroy(j.ctx);
    j.ctx = nullptr;
    if (j.stream) cudaStreamDestroy(j.stream);
    j.stream = nullptr;
}

}  // namespace

extern "C" {

hm_status hm_server_create(hm_server **out, const hm_server_config *cfg) {
    if (!out || !cfg) return HM_EINVAL;
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64) return HM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HM_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return HM_ECUDA;
    }
    hm_server *s = new (std::nothrow) hm_server();
    if (!s) return HM_ENOMEM;
    s->dev = dev;
    s->budget = cfg->hbm_budget ? cfg->hbm_budget : (size_t)(0.85 * (double)free_b);
    s->slots = cfg->slots;
    try {
        for (int w = 0; w < s->slots; ++w) s->workers.emplace_back([s] { s->worker(); });
    } catch (const std::exception &) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        delete s;
        return HM_ENOMEM;
    }
    *out = s;
    return HM_OK;
}

hm_status hm_server_submit(hm_server *s, const hm_job_desc *job, int64_t *job_id) {
    if (!s || !job || !job_id || !job->points_host || job->n < 1 || job->n > (1ll << 30)) return HM_EINVAL;
    const hm_config &c = job->cfg;
    if (c.d < 1 || c.d > 3 || c.r < 1 || c.r > 64 || job->leaf_size < 0 || job->rank < 0 || !(job->tol >= 0.0))
        return HM_EINVAL;
    if (job->op.kind == HM_OP_CALLBACK ? !job->op.apply : (job->op.kind == HM_OP_DENSE ? !job->op.dense_dev : false))
        return HM_EINVAL;
    auto j = std::make_shared<Job>();
    j->desc = *job;
    j->est = estimate_bytes(*job);
    if (j->est > s->budget) return HM_ENOTSUP;
    try {
        j->points.assign(job->points_host, job->points_host + (size_t)job->n * c.d);
    } catch (const std::exception &) {
        return HM_ENOMEM;
    }
    j->desc.points_host = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->id = s->next_id++;
        j->t_submit = s->now();
        if (s->first_submit < 0) s->first_submit = j->t_submit;
        ++s->submitted;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_all();
    return HM_OK;
}

hm_status hm_server_wait(hm_server *s, int64_t job_id, double timeout_s, hm_job_stats *stats) {
    if (!s) return HM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return HM_EINVAL;
    std::shared_ptr<Job> j = it->second;
    auto done = [&] { return j->state == HM_JOB_READY || j->state == HM_JOB_FAILED; };
    if (timeout_s < 0) s->cv_done.wait(lk, done);
    else s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
    fill_stats(*j, stats);
    if (!done()) return HM_ETIMEOUT;
    return j->status;
}

hm_status hm_server_apply(hm_server *s, int64_t job_id, const double *x_dev, double *y_dev, int64_t nrhs,
                          int trans) {
    if (!s || !x_dev || !y_dev || nrhs < 1 || nrhs > 64) return HM_EINVAL;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return HM_EINVAL;
        j = it->second;
        if (j->state != HM_JOB_READY) return HM_ESTATE;
    }
    const double t0 = s->now();
    hm_status st;
    {
        std::lock_guard<std::mutex> lk(j->apply_mu);
        hm::DeviceScope ds(s->dev);
        st = hm_apply(j->ctx, x_dev, y_dev, nrhs, trans);
        if (st == HM_OK && cudaStreamSynchronize(j->stream) != cudaSuccess) {
            cudaGetLastError();
            st = HM_ECUDA;
        }
    }
    if (st == HM_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->apply_lat.push_back(s->now() - t0);
    }
    return st;
}

hm_status hm_server_release(hm_server *s, int64_t job_id) {
    if (!s) return HM_EINVAL;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return HM_EINVAL;
        j = it->second;
        if (j->state != HM_JOB_READY && j->state != HM_JOB_FAILED) return HM_ESTATE;
        s->jobs.erase(it);
    }
    {
        std::lock_guard<std::mutex> lk(j->apply_mu);  // no apply of this job is in flight
        hm::DeviceScope ds(s->dev);
        free_job(*j);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->reserved -= j->reserved;
        j->reserved = 0;
        ++s->released;
    }
    s->cv_work.notify_all();
    return HM_OK;
}

hm_status hm_server_get_info(hm_server *s, hm_server_info *out) {
    if (!s || !out) return HM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = hm_server_info{};
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->released = s->released;
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->max_running = s->max_running;
    out->budget = s->budget;
    out->reserved = s->reserved;
    out->max_reserved = s->max_reserved;
    const double span = s->last_done - s->first_submit;
    out->jobs_per_s = (s->completed > 0 && span > 0) ? (double)s->completed / span : 0.0;
    out->job_p50_s = pct(s->job_lat, 0.5);
    out->job_p99_s = pct(s->job_lat, 0.99);
    out->applies = (int64_t)s->apply_lat.size();
    out->apply_p50_s = pct(s->apply_lat, 0.5);
    out->apply_p99_s = pct(s->apply_lat, 0.99);
    return HM_OK;
}

hm_status hm_server_destroy(hm_server *s) {
    if (!s) return HM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    {
        hm::DeviceScope ds(s->dev);
        for (auto &kv : s->jobs) free_job(*kv.second);
    }
    delete s;
    return HM_OK;
}

}  // extern "C"
