// Serving loop for imaging requests (continuous batching on one GPU).
//
// A request is a whole imaging problem (Eq. 3) solved to a relative-change
// tolerance with log-sum reweighting (Sec. 2.2.3).  Requests are independent,
// like the spectral sub-cubes of the paper, so they overlap freely:
//  - set-up threads admit queued requests first-fit while their estimated
//    peak device footprint fits the budget, and build each problem on a
//    stream of its own (host sort, G build, power iteration);
//  - a stepping thread keeps every admitted problem busy: it replays chunks of
//    PDFB iterations (CUDA graphs) on the problem's stream, reads the
//    relative change back asynchronously (event + pinned copy, no blocking
//    sync), moves to the next reweighting stage or retires the request
//    (image to the caller's host buffer), which frees its memory with
//    stream-ordered frees and wakes the setup thread.
#include "fhs_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kSetupThreads = 3;

struct Req {
    long long id = 0;
    fhs_params params{};
    std::vector<double> omega, w, y, sigma, eps;
    std::vector<int64_t> vis_off, blk_off;
    int max_iter = 0, n_reweight = 0, check_every = 10;
    double rel_tol = 0.0;
    long long peak_bytes = 0, resident_bytes = 0;
    // progress
    fhs_request_result res{};
    std::vector<float> image;                   // result on the host
    fhs_problem *prob = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    double *h_red = nullptr;                    // pinned [3]: the two reductions, then the device error flag
    bool in_flight = false;
    int stage = 0, stage_iters = 0, per_stage = 0;
};

}  // namespace

struct fhs_server {
    long long budget = 0;
    int max_active = 1, chunk = 10;
    Clock::time_point t0 = Clock::now();
    std::mutex mu;
    std::condition_variable cv_setup, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::vector<std::shared_ptr<Req>> active;
    std::map<long long, std::shared_ptr<Req>> all;
    long long next_id = 1;
    long long bytes_in_use = 0;                 // admitted peak/resident footprint
    int setting_up = 0;
    bool stop = false;
    int device = 0;
    std::vector<std::thread> th_setup;          // set-up is host-heavy (sort, tables): several threads
    std::thread th_step;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(fhs_server *sv, const std::shared_ptr<Req> &r, int state, int status) {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->res.state = state;
    r->res.status = status;
    r->res.t_done = sv->now();
    sv->bytes_in_use -= r->resident_bytes;
    sv->active.erase(std::remove(sv->active.begin(), sv->active.end(), r), sv->active.end());
    sv->cv_setup.notify_all();
    sv->cv_done.notify_all();
}

void release(std::shared_ptr<Req> &r) {
    if (r->prob) fhs::destroy_on_stream(r->prob, r->stream);
    r->prob = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    if (r->h_red) cudaFreeHost(r->h_red);
    r->h_red = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
    // inputs are no longer needed
    std::vector<double>().swap(r->omega);
    std::vector<double>().swap(r->w);
    std::vector<double>().swap(r->y);
}

void setup_loop(fhs_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::shared_ptr<Req> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_setup.wait(lk, [&] {
                if (sv->stop) return true;
                if ((int)sv->active.size() + sv->setting_up >= sv->max_active) return false;
                for (auto &q : sv->queue)
                    if (sv->bytes_in_use + q->peak_bytes <= sv->budget) return true;
                return false;
            });
            if (sv->stop) return;
            for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
                if (sv->bytes_in_use + (*it)->peak_bytes <= sv->budget) {
                    r = *it;
                    sv->queue.erase(it);
                    break;
                }
            if (!r) continue;
            sv->bytes_in_use += r->peak_bytes;   // held at peak during set-up
            sv->setting_up++;
            r->res.state = FHS_REQ_RUNNING;
            r->res.t_start = sv->now();
        }
        fhs_status st = FHS_OK;
        if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&r->h_red, 3 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            st = FHS_ERR_CUDA;
        }
        if (st == FHS_OK)
            st = fhs_create_problem(&r->params, r->omega.data(), r->w.empty() ? nullptr : r->w.data(), r->y.data(),
                                    r->sigma.data(), r->vis_off.data(), r->blk_off.data(),
                                    r->eps.empty() ? nullptr : r->eps.data(), r->stream, &r->prob);
        fhs_info info{};
        if (st == FHS_OK) fhs_get_info(r->prob, &info);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->setting_up--;
            sv->bytes_in_use -= r->peak_bytes;
            if (st == FHS_OK) {
                r->resident_bytes = std::max<long long>(info.device_bytes, 0);
                sv->bytes_in_use += r->resident_bytes;
                r->res.device_bytes = info.device_bytes;
                r->per_stage = r->max_iter / (r->n_reweight + 1);
                sv->active.push_back(r);
            }
        }
        if (st != FHS_OK) {
            release(r);
            std::lock_guard<std::mutex> lk(sv->mu);
            r->res.state = FHS_REQ_FAILED;
            r->res.status = st;
            r->res.t_done = sv->now();
            sv->cv_done.notify_all();
            sv->cv_setup.notify_all();
        }
    }
}

// One scheduling pass over one active request; returns true if it did work.
bool step_one(fhs_server *sv, std::shared_ptr<Req> &r) {
    const int stage_len = (r->stage < r->n_reweight) ? r->per_stage : r->max_iter - r->per_stage * r->n_reweight;
    if (r->in_flight) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) return false;
        r->in_flight = false;
        if (q != cudaSuccess) {
            cudaGetLastError();
            release(r);
            finish(sv, r, FHS_REQ_FAILED, FHS_ERR_CUDA);
            return true;
        }
        int dev_err = 0;
        std::memcpy(&dev_err, r->h_red + 2, sizeof dev_err);
        if (dev_err != 0) {
            // a bounded device wait gave up during these iterations: the iterate is not to be trusted
            release(r);
            finish(sv, r, FHS_REQ_FAILED, FHS_ERR_TIMEOUT);
            return true;
        }
        const double rel = r->h_red[1] > 0 ? std::sqrt(r->h_red[0] / r->h_red[1]) : INFINITY;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->res.rel_change = rel;
        }
        if (rel < r->rel_tol || r->stage_iters >= stage_len) {
            if (r->stage < r->n_reweight) {
                if (fhs_reweight(r->prob, r->stream) != FHS_OK) {
                    release(r);
                    finish(sv, r, FHS_REQ_FAILED, FHS_ERR_CUDA);
                    return true;
                }
                r->stage++;
                r->stage_iters = 0;
            } else {
                const size_t n = (size_t)r->params.n_channels * r->params.ny * r->params.nx;
                r->image.resize(n);
                float *dimg = nullptr;
                cudaError_t e = cudaMallocAsync(&dimg, n * sizeof(float), r->stream);
                if (e == cudaSuccess &&
                    fhs_get_state(r->prob, FHS_STATE_IMAGE, dimg, r->stream) == FHS_OK)
                    e = cudaMemcpyAsync(r->image.data(), dimg, n * sizeof(float), cudaMemcpyDeviceToHost, r->stream);
                if (dimg) cudaFreeAsync(dimg, r->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
                release(r);
                finish(sv, r, e == cudaSuccess ? FHS_REQ_DONE : FHS_REQ_FAILED,
                       e == cudaSuccess ? FHS_OK : FHS_ERR_CUDA);
                return true;
            }
        }
    }
    const int len = (r->stage < r->n_reweight) ? r->per_stage : r->max_iter - r->per_stage * r->n_reweight;
    const int n = std::min(r->check_every, std::max(len - r->stage_iters, 0));
    if (n > 0 && fhs_pdfb_step(r->prob, n, nullptr, r->stream) != FHS_OK) {
        release(r);
        finish(sv, r, FHS_REQ_FAILED, FHS_ERR_CUDA);
        return true;
    }
    r->stage_iters += n;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->res.iterations += n;
    }
    // relative change of the last iteration, read back without blocking
    if (cudaMemcpyAsync(r->h_red, r->prob->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaMemcpyAsync(r->h_red + 2, r->prob->dev_err, sizeof(int), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaEventRecord(r->ev, r->stream) != cudaSuccess) {
        cudaGetLastError();
        release(r);
        finish(sv, r, FHS_REQ_FAILED, FHS_ERR_CUDA);
        return true;
    }
    r->in_flight = true;
    return true;
}

void step_loop(fhs_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<std::shared_ptr<Req>> act;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop && sv->active.empty() && sv->setting_up == 0) return;
            act = sv->active;
        }
        bool worked = false;
        for (auto &r : act) worked |= step_one(sv, r);
        if (!worked) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

fhs_status fhs_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t check_every,
                             fhs_server **out) {
    if (!out || hbm_budget_bytes <= 0 || max_active < 1) {
        fhs::set_last_error("fhs_server_create: need out != NULL, budget > 0, max_active >= 1");
        return FHS_ERR_ARG;
    }
    fhs_server *sv = new fhs_server();
    sv->budget = hbm_budget_bytes;
    sv->max_active = max_active;
    sv->chunk = check_every > 0 ? check_every : 10;
    cudaGetDevice(&sv->device);
    for (int k = 0; k < kSetupThreads; ++k) sv->th_setup.emplace_back(setup_loop, sv);
    sv->th_step = std::thread(step_loop, sv);
    *out = sv;
    return FHS_OK;
}

fhs_status fhs_server_submit(fhs_server *sv, const fhs_request *q, int64_t *id_out) {
    if (!sv || !q || !id_out || !q->omega || !q->y || !q->sigma || !q->vis_offsets || !q->block_offsets ||
        q->max_iter < 0 || q->n_reweight < 0) {
        fhs::set_last_error("fhs_server_submit: bad argument");
        return FHS_ERR_ARG;
    }
    auto r = std::make_shared<Req>();
    r->params = q->params;
    const int L = q->params.n_channels, B = q->params.n_blocks;
    if (L < 1 || B < 1) {
        fhs::set_last_error("fhs_server_submit: bad channel or block count");
        return FHS_ERR_ARG;
    }
    const int64_t M = q->vis_offsets[L];
    r->vis_off.assign(q->vis_offsets, q->vis_offsets + L + 1);
    r->blk_off.assign(q->block_offsets, q->block_offsets + (size_t)L * (B + 1));
    r->omega.assign(q->omega, q->omega + 2 * M);
    if (q->w) r->w.assign(q->w, q->w + M);
    r->y.assign(q->y, q->y + 2 * M);
    r->sigma.assign(q->sigma, q->sigma + L);
    if (q->eps) r->eps.assign(q->eps, q->eps + (size_t)L * B);
    r->max_iter = q->max_iter;
    r->n_reweight = q->n_reweight;
    r->rel_tol = q->rel_tol;
    r->check_every = q->check_every > 0 ? q->check_every : sv->chunk;
    int64_t res = 0, peak = 0;
    fhs_status st = fhs_estimate_bytes(&r->params, r->w.empty() ? nullptr : r->w.data(), M, &res, &peak);
    if (st != FHS_OK) return st;
    if (peak > sv->budget) {
        fhs::set_last_error("fhs_server_submit: request needs more device memory than the server budget");
        return FHS_ERR_OOM;
    }
    r->peak_bytes = peak;
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    r->res.state = FHS_REQ_QUEUED;
    r->res.t_submit = sv->now();
    sv->queue.push_back(r);
    sv->all[r->id] = r;
    *id_out = r->id;
    sv->cv_setup.notify_all();
    return FHS_OK;
}

fhs_status fhs_server_query(fhs_server *sv, int64_t id, fhs_request_result *res_out) {
    if (!sv || !res_out) return FHS_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) {
        fhs::set_last_error("fhs_server_query: unknown request");
        return FHS_ERR_ARG;
    }
    *res_out = it->second->res;
    return FHS_OK;
}

fhs_status fhs_server_wait(fhs_server *sv, int64_t id, double timeout_s, float *image_out,
                           fhs_request_result *res_out) {
    if (!sv) return FHS_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) {
        fhs::set_last_error("fhs_server_wait: unknown request");
        return FHS_ERR_ARG;
    }
    std::shared_ptr<Req> r = it->second;
    auto done = [&] { return r->res.state == FHS_REQ_DONE || r->res.state == FHS_REQ_FAILED; };
    if (timeout_s < 0) sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        fhs::set_last_error("fhs_server_wait: timed out");
        return FHS_ERR_TIMEOUT;
    }
    if (res_out) *res_out = r->res;
    if (r->res.state == FHS_REQ_DONE && image_out) std::memcpy(image_out, r->image.data(), r->image.size() * 4);
    return r->res.state == FHS_REQ_DONE ? FHS_OK : (fhs_status)r->res.status;
}

fhs_status fhs_server_stats(fhs_server *sv, int64_t *active, int64_t *queued, int64_t *bytes_in_use) {
    if (!sv) return FHS_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (active) *active = (int64_t)sv->active.size() + sv->setting_up;
    if (queued) *queued = (int64_t)sv->queue.size();
    if (bytes_in_use) *bytes_in_use = sv->bytes_in_use;
    return FHS_OK;
}

void fhs_server_destroy(fhs_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        // queued requests are dropped (FAILED, FHS_ERR_STATE); admitted ones run to the end
        for (auto &q : sv->queue) {
            q->res.state = FHS_REQ_FAILED;
            q->res.status = FHS_ERR_STATE;
            q->res.t_done = sv->now();
        }
        sv->queue.clear();
        sv->stop = true;
        sv->cv_setup.notify_all();
        sv->cv_done.notify_all();
    }
    for (auto &t : sv->th_setup) t.join();
    sv->th_step.join();
    delete sv;
}

}  // extern "C"
