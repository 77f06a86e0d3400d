// Continuous-batching generation server: many GIRG requests in flight on one GPU.
//
// A request is admitted as soon as a worker is free and its estimated device
// scratch fits the memory budget next to the requests already running; each
// worker runs the full generation pipeline of its request on its own CUDA stream,
// so the kernels of different requests overlap on the device while one request
// waits for a host step (the search for c, the work-list sizes).  Requests are
// taken in arrival order, except that a request that does not fit the remaining
// budget lets up to kSkipAhead later ones that do fit go first.  Every result is
// the same as that of a lone girg_generate call with the same parameters (all
// randomness is counter-based), whatever the mix it ran in.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "girg_gb300.h"

namespace {

constexpr size_t kSkipAhead = 16;

double now_us(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
    girg_params p;
    void* d_edges;
    int64_t cap;
    int64_t id;
    int64_t mem;
    double t_submit;
};

}  // namespace

struct girg_server {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    int running = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::deque<girg_request_result> done;
    std::vector<std::thread> workers;
    int first_error = GIRG_OK;

    // index of the first queued request that may start now, or -1
    long admissible() const {
        const size_t lim = std::min(queue.size(), kSkipAhead + 1);
        for (size_t i = 0; i < lim; ++i)
            if (running == 0 || in_use + queue[i].mem <= budget) return (long)i;
        return -1;
    }

    void work() {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            first_error = GIRG_E_CUDA;
            return;
        }
        for (;;) {
            Request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return (stop && queue.empty()) || admissible() >= 0; });
                if (stop && queue.empty()) break;
                const long i = admissible();
                r = queue[(size_t)i];
                queue.erase(queue.begin() + i);
                in_use += r.mem;
                ++running;
            }
            girg_request_result res;
            std::memset(&res, 0, sizeof(res));
            res.request_id = r.id;
            res.t_submit_us = r.t_submit;
            res.t_start_us = now_us(t0);
            int64_t m = 0;
            double c = 0.0;
            res.status = girg_generate(&r.p, r.d_edges, r.cap, &m, &c, st);
            int64_t stats[15];
            const int k = girg_last_stats(stats, 15);  // this thread's last call
            res.num_edges = m;
            res.c_used = c;
            res.checksum = k > 14 ? (uint64_t)stats[14] : 0u;
            res.t_done_us = now_us(t0);
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= r.mem;
                --running;
                done.push_back(res);
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        cudaStreamDestroy(st);
    }
};

extern "C" {

int64_t girg_scratch_bytes(const girg_params* p) {
    if (!p || p->n < 1 || p->d < 1 || p->d > 8) return -1;
    const int d = p->d;
    int64_t n3 = 1, n6 = 1;
    for (int k = 0; k < d; ++k) {
        n3 *= 3;
        n6 *= 6;
    }
    // per vertex: points, sort buffers, sorted arrays, cell offsets and work entries
    // (about 400 + 112 d bytes), type-I items with pair counts and prefixes (28 bytes
    // each, 1 + 0.75 3^d per vertex), and the partner segments (8 bytes each) at the
    // library's initial work-list sizes; more is allocated only when a list grows
    const int64_t seg = p->T > 0.0 ? (d == 1 ? 8 : d == 2 ? 28 : d == 3 ? 112 : d == 4 ? 448 : 4 * n6) : 0;
    const int64_t per_v = 400 + 112 * d + 21 * n3 + 8 * seg;
    return p->n * per_v + (64ll << 20);
}

int girg_server_create(int32_t workers, int64_t memory_budget_bytes, girg_server** out) {
    if (!out || workers < 1 || workers > 256 || memory_budget_bytes <= 0) return GIRG_E_PARAM;
    girg_server* s = new girg_server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return GIRG_E_CUDA;
    }
    s->budget = memory_budget_bytes;
    for (int i = 0; i < workers; ++i) s->workers.emplace_back([s] { s->work(); });
    *out = s;
    return GIRG_OK;
}

int girg_server_submit(girg_server* s, const girg_params* p, void* d_edges,
                       int64_t capacity_edges, int64_t request_id) {
    if (!s || !p || capacity_edges < 0) return GIRG_E_PARAM;
    const int64_t mem = girg_scratch_bytes(p);
    if (mem < 0) return GIRG_E_PARAM;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return GIRG_E_PARAM;
        s->queue.push_back(Request{*p, d_edges, capacity_edges, request_id, mem, now_us(s->t0)});
    }
    s->cv_work.notify_one();
    return GIRG_OK;
}

int girg_server_poll(girg_server* s, girg_request_result* out, int32_t max_results,
                     int32_t wait_for) {
    if (!s || !out || max_results < 0) return -GIRG_E_PARAM;
    std::unique_lock<std::mutex> lk(s->mu);
    if (wait_for > 0)
        s->cv_done.wait(lk, [&] {
            return (int32_t)s->done.size() >= std::min(wait_for, max_results) ||
                   (s->queue.empty() && s->running == 0);
        });
    int32_t k = 0;
    while (k < max_results && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    return k;
}

int girg_server_pending(girg_server* s) {
    if (!s) return -GIRG_E_PARAM;
    std::lock_guard<std::mutex> lk(s->mu);
    return (int)s->queue.size() + s->running;
}

double girg_server_clock_us(girg_server* s) { return s ? now_us(s->t0) : -1.0; }

int girg_server_destroy(girg_server* s) {
    if (!s) return GIRG_E_PARAM;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    const int err = s->first_error;
    delete s;
    return err;
}

}  // extern "C"
