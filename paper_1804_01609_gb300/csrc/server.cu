// Serving loop: transport solves (requests) arrive at any time and are run to completion on
// one GPU with continuous batching. A scheduler thread repeats ticks:
//   1. admit queued requests in arrival order while each fits the device-memory budget and a
//      slot is free (the head of the queue waits for memory rather than being overtaken);
//   2. advance every running request by one SL step: all local-stencil requests together in
//      the batch engine's single persistent launch, every RBF-PU request on its own stream,
//      so their work overlaps on the device;
//   3. retire requests that reached their step count (copy the field out, free the memory,
//      record the latency).
// Node sets, stencil state and fields stay on the device between steps.
#include <chrono>
#include <cstdio>
#include <string>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int method = RBFSL_LOCAL;
    int steps = 0;
    // owned host copies of the request's inputs
    std::vector<double> nodes, q0, centers;
    rbfsl_problem prob{};
    int64_t pu_Mp = 0;
    double pu_radius = 0.0;
    int pu_weight = RBFSL_PU_WENDLAND;
    size_t bytes = 0;  // admission estimate
    // state
    int state = 0;     // 0 queued, 1 running, 2 done, < 0 failed
    int batch_id = -1;
    rbfsl_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int done_steps = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int64_t failed_points = 0;
    std::vector<double> result;
    std::string err;
};

// Device bytes a request holds while it runs (nodes, departure points, status, two fields,
// grid index, stencil factors or patch factors).
size_t estimate_bytes(const rbfsl_request &r) {
    const double N = (double)r.problem.N, T = r.problem.T;
    const double es = 8.0;  // FP64 or FP32-pair weights
    const int M = (r.problem.ell + 1) * (r.problem.ell + 1);
    double b = N * (24 + 24 + 4) + 2.0 * N * T * 8.0 + N * 28.0 + 64.0 * 1024 * 1024;
    if (r.method == RBFSL_LOCAL) {
        const double m = r.problem.n + M;
        b += N * r.problem.n * (4 + es);
        if (r.problem.mode == RBFSL_CENTER) b += N * (m * m * 8.0 + m * 4.0 + r.problem.n * 4.0);
    } else {
        const double R = r.pu_radius > 0 ? r.pu_radius : 2.0 * std::sqrt(r.problem.n / N);
        const double per = N * R * R / 4.0 * 1.3;  // nodes per patch, with margin
        const double m = per + M;
        b += (double)r.pu_Mp * (m * m * 8.0 + m * 4.0 + m * T * 12.0) + N * T * 8.0;
    }
    return (size_t)b;
}

}  // namespace
}  // namespace rbfsl

struct rbfsl_server {
    int device = 0;
    size_t budget = 0, used = 0, peak = 0;
    int max_slots = 0, running = 0;
    cudaStream_t stream = nullptr;  // the batch's stream
    rbfsl_batch *batch = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<rbfsl::Req>> reqs;
    uint64_t next_ticket = 1;
    std::thread worker;
    bool stop = false;
    int64_t ticks = 0;
    rbfsl::Clock::time_point t0;
    std::string err;
};

namespace rbfsl {
namespace {

double now_s(const rbfsl_server *s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

int start_request(rbfsl_server *s, Req &r) {
    if (r.method == RBFSL_LOCAL) {
        int id = -1;
        const int rc = rbfsl_batch_add(s->batch, &r.prob, &id);
        if (rc) return rc;
        r.batch_id = id;
        return RBFSL_OK;
    }
    int rc;
    if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return RBFSL_ECUDA;
    }
    if ((rc = rbfsl_create(&r.ctx, s->device, r.stream))) return rc;
    const rbfsl_problem &p = r.prob;
    if ((rc = rbfsl_set_nodes(r.ctx, p.nodes, p.N, RBFSL_HOST))) return rc;
    const int nv = p.vel_kind == RBFSL_VEL_RIGID ? 4 : 2;
    if ((rc = rbfsl_set_velocity(r.ctx, p.vel_kind, p.vel_params, nv))) return rc;
    if ((rc = rbfsl_set_method(r.ctx, RBFSL_PU, RBFSL_DIRECT))) return rc;
    if ((rc = rbfsl_set_stencil_size(r.ctx, p.n))) return rc;
    if ((rc = rbfsl_set_sh_degree(r.ctx, p.ell))) return rc;
    if ((rc = rbfsl_set_kernel(r.ctx, RBFSL_PHS, p.phs_power))) return rc;
    if ((rc = rbfsl_set_pu(r.ctx, r.centers.data(), r.pu_Mp, r.pu_radius, r.pu_weight, RBFSL_HOST))) return rc;
    if ((rc = rbfsl_set_precision(r.ctx, p.precision))) return rc;
    if ((rc = rbfsl_set_dt(r.ctx, p.dt))) return rc;
    if ((rc = rbfsl_set_time(r.ctx, p.t0))) return rc;
    if ((rc = rbfsl_set_tracers(r.ctx, p.q0, p.N, p.T, RBFSL_F64, RBFSL_HOST))) return rc;
    return RBFSL_OK;
}

void release_request(rbfsl_server *s, Req &r) {
    if (r.batch_id >= 0) rbfsl_batch_remove(s->batch, r.batch_id);
    r.batch_id = -1;
    if (r.ctx) rbfsl_destroy(r.ctx);
    r.ctx = nullptr;
    if (r.stream) cudaStreamDestroy(r.stream);
    r.stream = nullptr;
}

void worker_loop(rbfsl_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Req *> to_start;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(1), [s] { return s->stop || !s->queue.empty() || s->running > 0; });
            if (s->stop) break;
            // admit in arrival order while the head fits
            while (!s->queue.empty()) {
                Req &r = *s->reqs[s->queue.front()];
                if (s->running >= s->max_slots || s->used + r.bytes > s->budget) break;
                s->queue.pop_front();
                s->used += r.bytes;
                s->peak = std::max(s->peak, s->used);
                ++s->running;
                r.state = 1;
                to_start.push_back(&r);
            }
        }
        for (Req *r : to_start) {
            r->t_admit = now_s(s);
            const int rc = start_request(s, *r);
            if (rc) {
                r->err = std::string("admission: ") + (r->ctx ? rbfsl_last_error(r->ctx) : get_error());
                release_request(s, *r);
                std::lock_guard<std::mutex> lk(s->mu);
                r->state = rc;
                r->t_finish = now_s(s);
                s->used -= r->bytes;
                --s->running;
                s->cv.notify_all();
            }
        }
        std::vector<Req *> active;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto &kv : s->reqs)
                if (kv.second->state == 1) active.push_back(kv.second.get());
        }
        if (active.empty()) continue;
        // one tick: every running request advances one SL step
        bool any_local = false;
        for (Req *r : active) {
            if (r->method == RBFSL_LOCAL) {
                any_local = true;
            } else {
                const int rc = rbfsl_step(r->ctx, 1);
                if (rc != RBFSL_OK) {
                    r->state = rc;
                    r->err = std::string("step: ") + rbfsl_last_error(r->ctx);
                }
            }
        }
        if (any_local) {
            const int rc = rbfsl_batch_step(s->batch, 1);
            if (rc != RBFSL_OK) {
                const std::string msg = std::string("batched step: ") + get_error();
                for (Req *r : active)
                    if (r->method == RBFSL_LOCAL) { r->state = rc; r->err = msg; }
            }
        }
        cudaStreamSynchronize(s->stream);
        for (Req *r : active)
            if (r->stream) cudaStreamSynchronize(r->stream);
        ++s->ticks;
        for (Req *r : active) {
            if (r->state == 1) ++r->done_steps;
            if (r->state == 1 && r->done_steps < r->steps) continue;
            if (r->state == 1) {
                r->result.resize((size_t)r->prob.N * r->prob.T);
                int rc;
                rbfsl_stats ps{};
                if (r->method == RBFSL_LOCAL) {
                    rc = rbfsl_batch_get_q(s->batch, r->batch_id, r->result.data());
                    if (!rc) rc = rbfsl_batch_problem_stats(s->batch, r->batch_id, &ps);
                } else {
                    rc = rbfsl_get_q(r->ctx, r->result.data(), RBFSL_F64, RBFSL_HOST);
                    if (!rc) rc = rbfsl_get_stats(r->ctx, &ps);
                }
                r->failed_points = ps.singular_points + ps.knn_failures + ps.uncovered_points;
                if (rc) {
                    r->state = rc;
                    r->err = std::string("result: ") + (r->ctx ? rbfsl_last_error(r->ctx) : get_error());
                }
            }
            release_request(s, *r);
            std::lock_guard<std::mutex> lk(s->mu);
            if (r->state == 1) r->state = 2;
            r->t_finish = now_s(s);
            s->used -= r->bytes;
            --s->running;
            s->cv.notify_all();
        }
    }
}

}  // namespace
}  // namespace rbfsl

using namespace rbfsl;

extern "C" {

int rbfsl_server_create(rbfsl_server **out, int device, size_t hbm_budget_bytes, int max_slots) {
    RBFSL_CHECK_ARG(out && hbm_budget_bytes > 0 && max_slots >= 1, "server_create: bad arguments");
    RBFSL_CUDA_TRY(cudaSetDevice(device));
    auto *s = new rbfsl_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->t0 = Clock::now();
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("server_create: stream creation failed");
        return RBFSL_ECUDA;
    }
    int rc = rbfsl_batch_create(&s->batch, device, s->stream);
    if (rc) {
        cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return RBFSL_OK;
}

int rbfsl_server_destroy(rbfsl_server *s) {
    if (!s) return RBFSL_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->reqs) release_request(s, *kv.second);
    rbfsl_batch_destroy(s->batch);
    cudaStreamDestroy(s->stream);
    delete s;
    return RBFSL_OK;
}

int rbfsl_server_submit(rbfsl_server *s, const rbfsl_request *r, uint64_t *ticket) {
    RBFSL_CHECK_ARG(s && r && ticket, "server_submit: null argument");
    const rbfsl_problem &p = r->problem;
    RBFSL_CHECK_ARG(r->method == RBFSL_LOCAL || r->method == RBFSL_PU, "server_submit: method must be LOCAL or PU");
    RBFSL_CHECK_ARG(r->steps >= 1, "server_submit: steps < 1");
    RBFSL_CHECK_ARG(p.N >= 1 && p.nodes && p.q0 && p.T >= 1 && p.dt > 0, "server_submit: bad problem");
    RBFSL_CHECK_ARG(r->method == RBFSL_LOCAL || (r->pu_centers && r->pu_Mp >= 1), "server_submit: PU needs centres");
    auto q = std::make_unique<Req>();
    q->method = r->method;
    q->steps = r->steps;
    q->nodes.assign(p.nodes, p.nodes + 3 * p.N);
    q->q0.assign(p.q0, p.q0 + p.N * p.T);
    q->prob = p;
    q->prob.nodes = q->nodes.data();
    q->prob.q0 = q->q0.data();
    if (r->method == RBFSL_PU) {
        q->centers.assign(r->pu_centers, r->pu_centers + 3 * r->pu_Mp);
        q->pu_Mp = r->pu_Mp;
        q->pu_radius = r->pu_radius;
        q->pu_weight = r->pu_weight;
    }
    q->bytes = estimate_bytes(*r);
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->bytes > s->budget) {
        set_error("server_submit: the request alone exceeds the device-memory budget");
        return RBFSL_ENOMEM;
    }
    q->ticket = s->next_ticket++;
    q->t_submit = now_s(s);
    *ticket = q->ticket;
    s->queue.push_back(q->ticket);
    s->reqs[q->ticket] = std::move(q);
    s->cv.notify_all();
    return RBFSL_OK;
}

int rbfsl_server_poll(rbfsl_server *s, uint64_t ticket, int *state) {
    RBFSL_CHECK_ARG(s && state, "server_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    RBFSL_CHECK_ARG(it != s->reqs.end(), "server_poll: unknown ticket");
    *state = it->second->state;
    return RBFSL_OK;
}

int rbfsl_server_result(rbfsl_server *s, uint64_t ticket, double *q_out, rbfsl_request_stats *st) {
    RBFSL_CHECK_ARG(s, "server_result: null server");
    std::unique_ptr<Req> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        RBFSL_CHECK_ARG(it != s->reqs.end(), "server_result: unknown ticket");
        if (it->second->state == 0 || it->second->state == 1) {
            set_error("server_result: request not finished");
            return RBFSL_EINVAL;
        }
        r = std::move(it->second);
        s->reqs.erase(it);
    }
    if (st) {
        st->submit_s = r->t_submit;
        st->admit_s = r->t_admit;
        st->finish_s = r->t_finish;
        st->steps = r->done_steps;
        st->node_updates = (int64_t)r->done_steps * r->prob.N;
        st->device_bytes = r->bytes;
        st->status = r->state == 2 ? RBFSL_OK : r->state;
        std::snprintf(st->message, sizeof(st->message), "%s", r->err.c_str());
        st->failed_points = r->failed_points;
    }
    if (r->state != 2) {
        set_error("server_result: the request failed");
        return r->state;
    }
    if (q_out) std::copy(r->result.begin(), r->result.end(), q_out);
    return RBFSL_OK;
}

int rbfsl_server_wait_idle(rbfsl_server *s, double timeout_s) {
    RBFSL_CHECK_ARG(s, "server_wait_idle: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                   [s] { return s->queue.empty() && s->running == 0; });
    if (!ok) {
        set_error("server_wait_idle: timed out");
        return RBFSL_ETIMEDOUT;
    }
    return RBFSL_OK;
}

int rbfsl_server_info(rbfsl_server *s, rbfsl_server_info_t *out) {
    RBFSL_CHECK_ARG(s && out, "server_info: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->ticks = s->ticks;
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->budget_bytes = s->budget;
    out->used_bytes = s->used;
    out->peak_bytes = s->peak;
    out->now_s = now_s(s);
    return RBFSL_OK;
}

}  // extern "C"
