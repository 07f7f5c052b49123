// Serving runtime (no counterpart in the paper): many independent runs on one
// GPU.  A worker thread admits queued requests in arrival order while a slot
// is free and the admitted runs' estimated device bytes fit the budget, gives
// every admitted run its own handle and stream, and each round issues the
// next step of every admitted run on its stream (the runs' kernels overlap on
// the device).  Optionally (batch_min_runs), groups of runs of one form are
// advanced by one batched step -- one persistent push launch and one regroup
// launch over the work items of all of them; measured, the independent
// streams serve faster.  Runs that arrive meanwhile join at the next round.  Finished runs are harvested:
// their diagnostics (and, on request, moments and fields) go to host memory
// and the handle and its device memory are freed before the next admission.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pic.h"

namespace {

struct Request {
    int64_t id = 0;
    pic_config cfg{};
    int32_t flags = 0;
    std::vector<int64_t> n;
    std::vector<std::vector<double>> data;  // per species [x | y | ux | uy | uz | w]
    pic_request_status st{};
    pic_t *h = nullptr;
    cudaStream_t stream = nullptr;
    int64_t count0 = 0;
    bool cancel = false;   // set under the server lock; the worker stops the run
    pic_diag diag{};
    std::vector<double> rho, S9, dj3, E3, H3;
};

int64_t node_count(const pic_config &c) { return (int64_t)(c.bc_x == PIC_BC_PERIODIC ? c.nx : c.nx + 1) * c.ny; }

}  // namespace

struct pic_server {
    pic_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request *> queue;     // queued, arrival order
    std::vector<Request *> running;  // admitted (worker thread only)
    uint64_t used = 0;               // admission estimate of the admitted runs
    int64_t next_id = 1;
    int active = 0;                  // queued + admitted
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void set_state(pic_server *srv, Request *r, int state, int err) {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->st.state = state;
    r->st.error = err;
    if (state == PIC_REQ_RUNNING) r->st.t_start = srv->now();
    if (state == PIC_REQ_DONE || state == PIC_REQ_FAILED || state == PIC_REQ_CANCELLED) {
        r->st.t_finish = srv->now();
        srv->active -= 1;
        srv->cv.notify_all();
    }
}

void free_run(Request *r) {
    if (r->h) pic_destroy(r->h);
    r->h = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
}

// Handle, stream and particles of an admitted request; the host copies of the
// particles are dropped once they are on the device.
int start_run(Request *r) {
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    pic_config c = r->cfg;
    c.cuda_stream = r->stream;
    for (int s = 0; s < c.n_species; ++s) c.capacity[s] = r->n[s];
    if (int rc = pic_init(&c, &r->h)) return rc;
    pic_species_data sd[PIC_MAX_SPECIES];
    for (int s = 0; s < c.n_species; ++s) {
        const int64_t n = r->n[s];
        const double *d = r->data[s].data();
        sd[s] = pic_species_data{n, d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, d + 5 * n};
    }
    if (int rc = pic_load_species(r->h, c.n_species, sd)) return rc;
    for (int s = 0; s < c.n_species; ++s) r->count0 += r->n[s];
    std::vector<std::vector<double>>().swap(r->data);
    return PIC_OK;
}

int harvest(Request *r) {
    if (int rc = pic_diagnostics(r->h, &r->diag)) return rc;
    r->st.particle_steps = 0.5 * (double)(r->count0 + r->diag.count) * (double)r->st.steps_total;
    if (r->flags & PIC_SUBMIT_KEEP_GRIDS) {
        const int64_t nn = node_count(r->cfg), nc = (int64_t)r->cfg.nx * r->cfg.ny;
        r->rho.resize(nn);
        r->S9.resize(9 * nn);
        r->dj3.resize(3 * nn);
        r->E3.resize(3 * nn);
        r->H3.resize(3 * nc);
        if (int rc = pic_moments(r->h, r->rho.data(), r->S9.data(), r->dj3.data())) return rc;
        if (int rc = pic_fields(r->h, r->E3.data(), r->H3.data())) return rc;
    }
    return PIC_OK;
}

void worker_loop(pic_server *srv) {
    cudaSetDevice(srv->device);
    const int per_round = srv->cfg.steps_per_round > 0 ? srv->cfg.steps_per_round : 1;
    const int min_batch = srv->cfg.batch_min_runs > 0 ? srv->cfg.batch_min_runs : (1 << 30);
    cudaStream_t bst = nullptr;
    cudaStreamCreateWithFlags(&bst, cudaStreamNonBlocking);
    std::map<int, pic_batch *> batches;   // form (2 * fp32 + deterministic) -> batch scratch
    for (;;) {
        std::vector<Request *> admit;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->running.empty())
                srv->cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return srv->stop || !srv->queue.empty(); });
            if (srv->stop) break;
            while (!srv->queue.empty() && (int)(srv->running.size() + admit.size()) < srv->cfg.max_slots) {
                Request *r = srv->queue.front();
                if (srv->used + r->st.device_bytes > srv->cfg.mem_budget) break;  // in order: wait for room
                srv->used += r->st.device_bytes;
                srv->queue.pop_front();
                admit.push_back(r);
            }
        }
        for (Request *r : admit) {
            int rc = start_run(r);
            if (rc) {
                free_run(r);
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    srv->used -= r->st.device_bytes;
                }
                set_state(srv, r, PIC_REQ_FAILED, rc);
                continue;
            }
            srv->running.push_back(r);
            set_state(srv, r, PIC_REQ_RUNNING, 0);
        }
        // one round: every admitted run advances, one batched step per form
        std::map<int, std::vector<Request *>> groups;
        std::vector<char> cancelled;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (Request *r : srv->running) cancelled.push_back(r->cancel ? 1 : 0);
        }
        for (size_t i = 0; i < srv->running.size(); ++i) {
            Request *r = srv->running[i];
            if (!cancelled[i] && !r->st.error && r->st.steps_done < r->st.steps_total)
                groups[4 * (r->cfg.shape > PIC_SHAPE_LINEAR) + 2 * (r->cfg.precision == PIC_FP32) +
                       (r->cfg.deposit == PIC_DEPOSIT_DETERMINISTIC)].push_back(r);
        }
        for (auto &kv : groups) {
            std::vector<Request *> &grp = kv.second;
            int64_t k = per_round;
            for (Request *r : grp) {
                const int64_t left = r->st.steps_total - r->st.steps_done;
                if (left < k) k = left;
            }
            if ((int)grp.size() < min_batch || kv.first >= 4) {
                // a lone run (or a run of a spline shape: no batched form) steps on its own stream
                for (Request *r : grp) {
                    const int rc = pic_step(r->h, (int)k);
                    std::lock_guard<std::mutex> lk(srv->mu);
                    if (rc) r->st.error = rc;
                    else r->st.steps_done += k;
                }
                continue;
            }
            pic_batch *&b = batches[kv.first];
            int rc = b ? PIC_OK : pic_batch_create(srv->cfg.max_slots, bst, &b);
            if (!rc) {
                std::vector<pic_t *> hs;
                for (Request *r : grp) hs.push_back(r->h);
                rc = pic_batch_step(b, hs.data(), (int)hs.size(), (int)k);
            }
            std::lock_guard<std::mutex> lk(srv->mu);
            for (Request *r : grp) {
                if (rc) r->st.error = rc;
                else r->st.steps_done += k;
            }
        }
        // harvest finished (or failed) runs and free their memory; drop cancelled ones
        std::vector<Request *> keep;
        for (size_t i = 0; i < srv->running.size(); ++i) {
            Request *r = srv->running[i];
            if (cancelled[i]) {
                if (r->stream) cudaStreamSynchronize(r->stream);
                free_run(r);
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    srv->used -= r->st.device_bytes;
                }
                set_state(srv, r, PIC_REQ_CANCELLED, 0);
                continue;
            }
            if (!r->st.error && r->st.steps_done < r->st.steps_total) {
                keep.push_back(r);
                continue;
            }
            int rc = r->st.error ? r->st.error : harvest(r);
            free_run(r);
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->used -= r->st.device_bytes;
            }
            set_state(srv, r, rc ? PIC_REQ_FAILED : PIC_REQ_DONE, rc);
        }
        srv->running.swap(keep);
    }
    for (Request *r : srv->running) free_run(r);
    srv->running.clear();
    for (auto &kv : batches) pic_batch_destroy(kv.second);
    if (bst) cudaStreamDestroy(bst);
}

}  // namespace

extern "C" PIC_API int pic_server_create(const pic_server_config *cfg, pic_server **out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    pic_server *srv = new pic_server();
    if (cfg) srv->cfg = *cfg;
    if (srv->cfg.max_slots <= 0) srv->cfg.max_slots = 64;
    if (srv->cfg.steps_per_round <= 0) srv->cfg.steps_per_round = 1;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return PIC_ERR_CUDA;
    }
    if (srv->cfg.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete srv;
            return PIC_ERR_CUDA;
        }
        srv->cfg.mem_budget = (uint64_t)(0.8 * (double)fr);
    }
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return PIC_OK;
}

extern "C" PIC_API int pic_server_destroy(pic_server *srv) {
    if (!srv) return PIC_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return PIC_OK;
}

extern "C" PIC_API int pic_server_submit(pic_server *srv, const pic_config *cfg, int32_t nsteps,
                                         const pic_species_data *species, int32_t flags, int64_t *id) {
    if (!srv || !cfg || !id || nsteps < 0 || cfg->n_species < 1 || cfg->n_species > PIC_MAX_SPECIES ||
        (!species && cfg->n_species > 0))
        return PIC_ERR_ARG;
    std::unique_ptr<Request> r(new Request());
    r->cfg = *cfg;
    r->cfg.cuda_stream = nullptr;
    r->flags = flags;
    r->st.steps_total = nsteps;
    r->n.assign(cfg->n_species, 0);
    r->data.resize(cfg->n_species);
    for (int s = 0; s < cfg->n_species; ++s) {
        const pic_species_data &d = species[s];
        if (d.n < 0 || (d.n > 0 && (!d.x || !d.y || !d.ux || !d.uy || !d.uz || !d.w))) return PIC_ERR_ARG;
        r->n[s] = d.n;
        std::vector<double> &v = r->data[s];
        v.resize(6 * d.n);
        const double *src[6] = {d.x, d.y, d.ux, d.uy, d.uz, d.w};
        for (int k = 0; k < 6; ++k)
            if (d.n) memcpy(v.data() + k * d.n, src[k], d.n * sizeof(double));
    }
    if (int rc = pic_estimate_bytes(&r->cfg, r->n.data(), &r->st.device_bytes)) return rc;
    std::lock_guard<std::mutex> lk(srv->mu);
    r->id = srv->next_id++;
    r->st.t_submit = srv->now();
    *id = r->id;
    Request *p = r.get();
    srv->reqs[r->id] = std::move(r);
    if (p->st.device_bytes > srv->cfg.mem_budget) {
        // can never be admitted
        p->st.state = PIC_REQ_FAILED;
        p->st.error = PIC_ERR_OOM;
        p->st.t_finish = p->st.t_submit;
        std::vector<std::vector<double>>().swap(p->data);
        return PIC_OK;
    }
    p->st.state = PIC_REQ_QUEUED;
    srv->queue.push_back(p);
    srv->active += 1;
    srv->cv.notify_all();
    return PIC_OK;
}

extern "C" PIC_API int pic_server_status(pic_server *srv, int64_t id, pic_request_status *out) {
    if (!srv || !out) return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return PIC_ERR_ARG;
    *out = it->second->st;
    return PIC_OK;
}

extern "C" PIC_API int pic_server_result(pic_server *srv, int64_t id, pic_diag *diag, double *rho, double *S9,
                                         double *dj3, double *E3, double *H3) {
    if (!srv) return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return PIC_ERR_ARG;
    Request *r = it->second.get();
    if (r->st.state != PIC_REQ_DONE) return PIC_ERR_STATE;
    if (diag) *diag = r->diag;
    const bool grids = (r->flags & PIC_SUBMIT_KEEP_GRIDS) != 0;
    if ((rho || S9 || dj3 || E3 || H3) && !grids) return PIC_ERR_STATE;
    auto cp = [](double *dst, const std::vector<double> &v) {
        if (dst && !v.empty()) memcpy(dst, v.data(), v.size() * sizeof(double));
    };
    cp(rho, r->rho);
    cp(S9, r->S9);
    cp(dj3, r->dj3);
    cp(E3, r->E3);
    cp(H3, r->H3);
    return PIC_OK;
}

extern "C" PIC_API int pic_server_release(pic_server *srv, int64_t id) {
    if (!srv) return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return PIC_ERR_ARG;
    const int st = it->second->st.state;
    if (st != PIC_REQ_DONE && st != PIC_REQ_FAILED && st != PIC_REQ_CANCELLED) return PIC_ERR_STATE;
    srv->reqs.erase(it);
    return PIC_OK;
}

extern "C" PIC_API int pic_server_cancel(pic_server *srv, int64_t id) {
    if (!srv) return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return PIC_ERR_ARG;
    Request *r = it->second.get();
    if (r->cancel) return PIC_ERR_STATE;
    if (r->st.state == PIC_REQ_QUEUED) {
        for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
            if (*q == r) {
                srv->queue.erase(q);
                std::vector<std::vector<double>>().swap(r->data);
                r->st.state = PIC_REQ_CANCELLED;
                r->st.t_finish = srv->now();
                srv->active -= 1;
                srv->cv.notify_all();
                return PIC_OK;
            }
        // taken off the queue and being started by the worker: it stops the run once started
        r->cancel = true;
        return PIC_OK;
    }
    if (r->st.state != PIC_REQ_RUNNING) return PIC_ERR_STATE;
    r->cancel = true;   // the worker stops it at the end of its round
    return PIC_OK;
}

extern "C" PIC_API int pic_server_wait_all(pic_server *srv, double timeout_s) {
    if (!srv) return PIC_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    const bool ok = srv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return srv->active == 0; });
    return ok ? PIC_OK : PIC_ERR_TIMEOUT;
}

extern "C" PIC_API double pic_server_now(pic_server *srv) { return srv ? srv->now() : 0.0; }
