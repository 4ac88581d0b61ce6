// adi_serve.cu -- the serving loop of libadi (include/adi.h, "Serving"): a FIFO of requests
// admitted by an HBM budget into a set of resident simulations that advance together as one
// batch, re-formed whenever a simulation joins or leaves.  Host code only: every step of the
// simulations runs in the batch's kernels (adi_batch_step).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <new>
#include <vector>

#include "../../include/adi.h"
#include "adi_internal.h"

namespace {

struct Request {
    adi_request r{};                       // pointers below replace the caller's
    std::vector<double> c, u, v, w;        // host copies (u, v, w empty: zeros)
    std::vector<double> ru, rv, rw;        // results
    size_t bytes = 0;                      // reserved device bytes while running
    int state = ADI_REQ_PENDING;
    int remaining = 0;                     // steps still to run
    adi_handle sim = nullptr;
    double t_submit = -1, t_start = -1, t_done = -1;
};

size_t field_count(int method, int nx, int ny, int which) {  // 0 U, 1 V, 2 W
    if (method == ADI_CFD) return (size_t)(ny + 1) * (nx + 1);
    if (which == 0) return (size_t)(ny + 2) * (nx + 2);
    if (which == 1) return (size_t)(ny + 2) * (nx + 1);
    return (size_t)(ny + 1) * (nx + 2);
}

}  // namespace

struct adi_server_t {
    size_t budget = 0, used = 0;
    int precision = ADI_FP32, quantum = 1, max_active = 1;
    std::vector<Request> reqs;             // indexed by ticket
    std::deque<int> pending;               // tickets in arrival order
    std::vector<int> running;              // tickets
    adi_batch batch = nullptr;             // over `running`, null when it must be re-formed
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void drop_batch(adi_server s) {
    if (s->batch) adi_batch_destroy(s->batch);
    s->batch = nullptr;
}

// Creates the simulation of a request; ADI_ENOMEM leaves the request waiting.
int start_request(adi_server s, Request &q) {
    const adi_request &r = q.r;
    adi_handle h = nullptr;
    int rc = adi_create(&h, r.method, r.nx, r.ny, r.h, r.dt, q.c.data(), q.u.empty() ? nullptr : q.u.data(),
                        q.v.empty() ? nullptr : q.v.data(), q.w.empty() ? nullptr : q.w.data(), s->precision);
    if (!rc && r.has_source) rc = adi_set_source(h, r.src_i, r.src_j, r.src_amp, r.src_f0, r.src_tdelay);
    if (rc) {
        adi_destroy(h);
        return rc;
    }
    q.sim = h;
    q.remaining = r.nsteps;
    q.state = ADI_REQ_RUNNING;
    q.t_start = s->now();
    return ADI_OK;
}

// Copies the fields of a finished simulation to the host and frees its device memory.
int retire_request(adi_server s, Request &q) {
    const adi_request &r = q.r;
    q.ru.resize(field_count(r.method, r.nx, r.ny, 0));
    q.rv.resize(field_count(r.method, r.nx, r.ny, 1));
    q.rw.resize(field_count(r.method, r.nx, r.ny, 2));
    int rc = adi_read_fields(q.sim, q.ru.data(), q.rv.data(), q.rw.data());
    adi_destroy(q.sim);
    q.sim = nullptr;
    s->used -= q.bytes;
    q.state = rc ? ADI_REQ_FAILED : ADI_REQ_DONE;
    q.t_done = s->now();
    return rc;
}

// Admits waiting requests in order while they fit; the first that does not fit waits.
int admit(adi_server s) {
    while (!s->pending.empty() && (int)s->running.size() < s->max_active) {
        Request &q = s->reqs[s->pending.front()];
        if (s->used + q.bytes > s->budget) break;
        int rc = start_request(s, q);
        if (rc == ADI_ENOMEM) break;  // the device is fuller than the budget says: wait
        const int ticket = s->pending.front();
        s->pending.pop_front();
        if (rc) {
            q.state = ADI_REQ_FAILED;
            q.t_done = s->now();
            continue;
        }
        s->used += q.bytes;
        if (q.remaining == 0) {
            retire_request(s, q);
            continue;
        }
        s->running.push_back(ticket);
        drop_batch(s);
    }
    return ADI_OK;
}

}  // namespace

extern "C" {

size_t adi_server_bytes(int method, int nx, int ny, int precision) {
    const size_t st = adi_state_bytes(method, nx, ny, precision);
    if (!st) return 0;
    const size_t xl = method == ADI_CFD ? (size_t)(ny - 1) : (size_t)ny;  // x-lines (nx cells each)
    const size_t yl = method == ADI_CFD ? (size_t)(nx - 1) : (size_t)nx;  // y-lines (ny cells each)
    // groups per line: one at most, or up to kFacMaxSplit sub-lines for a split line
    const size_t gx = adi::fac_split_line(method, nx) ? adi::kFacMaxSplit : 1;
    const size_t gy = adi::fac_split_line(method, ny) ? adi::kFacMaxSplit : 1;
    // the batch's own descriptor copies (two parities) and line-group table
    return st + 2 * (xl + yl) * sizeof(adi::LineDesc<double>) + (xl * gx + yl * gy) * sizeof(adi::FacGroup);
}

int adi_server_create(adi_server *out, size_t hbm_budget, int precision, int quantum, int max_active) {
    if (!out) return ADI_EINVAL;
    *out = nullptr;
    if ((precision != ADI_FP32 && precision != ADI_FP64) || quantum < 1 || max_active < 1 || hbm_budget == 0)
        return ADI_EINVAL;
    adi_server s = new (std::nothrow) adi_server_t;
    if (!s) return ADI_ENOMEM;
    s->budget = hbm_budget;
    s->precision = precision;
    s->quantum = quantum;
    s->max_active = max_active;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return ADI_ECUDA;
    }
    *out = s;
    return ADI_OK;
}

int adi_server_submit(adi_server s, const adi_request *req, int *ticket) {
    if (!s || !req || !ticket) return ADI_EINVAL;
    const adi_request &r = *req;
    if (r.nsteps < 0 || !r.c_field) return ADI_EINVAL;
    const size_t bytes = adi_server_bytes(r.method, r.nx, r.ny, s->precision);
    if (!bytes) return ADI_EINVAL;
    if (bytes > s->budget) return ADI_ENOMEM;
    Request q;
    q.r = r;
    q.bytes = bytes;
    q.c.assign(r.c_field, r.c_field + field_count(r.method, r.nx, r.ny, 0));
    if (r.u0) q.u.assign(r.u0, r.u0 + field_count(r.method, r.nx, r.ny, 0));
    if (r.v0) q.v.assign(r.v0, r.v0 + field_count(r.method, r.nx, r.ny, 1));
    if (r.w0) q.w.assign(r.w0, r.w0 + field_count(r.method, r.nx, r.ny, 2));
    q.r.c_field = q.r.u0 = q.r.v0 = q.r.w0 = nullptr;
    q.t_submit = s->now();
    *ticket = (int)s->reqs.size();
    s->reqs.push_back(std::move(q));
    s->pending.push_back(*ticket);
    return ADI_OK;
}

int adi_server_tick(adi_server s, int *n_running, int *n_pending) {
    if (!s) return ADI_EINVAL;
    int rc = admit(s);
    if (!rc && !s->running.empty()) {
        if (!s->batch) {
            std::vector<adi_handle> hs;
            for (int t : s->running) hs.push_back(s->reqs[t].sim);
            rc = adi_batch_create(&s->batch, hs.data(), (int)hs.size());
            if (!rc) rc = adi_batch_set_stream(s->batch, s->stream);
        }
        int q = s->quantum;
        for (int t : s->running) q = std::min(q, s->reqs[t].remaining);
        if (!rc) rc = adi_batch_step(s->batch, q);
        if (!rc) rc = adi_batch_sync(s->batch);
        if (!rc) {
            std::vector<int> still;
            bool left = false;
            for (int t : s->running) {
                s->reqs[t].remaining -= q;
                if (s->reqs[t].remaining > 0) still.push_back(t); else left = true;
            }
            if (left) {
                drop_batch(s);  // members leave: the batch is re-formed next round
                for (int t : s->running)
                    if (s->reqs[t].remaining == 0) {
                        int r2 = retire_request(s, s->reqs[t]);
                        if (!rc) rc = r2;
                    }
                s->running = still;
            }
        }
        if (!rc) rc = admit(s);
    }
    if (n_running) *n_running = (int)s->running.size();
    if (n_pending) *n_pending = (int)s->pending.size();
    return rc;
}

int adi_server_status(adi_server s, int ticket, int *state, double *t_submit, double *t_start, double *t_done) {
    if (!s || ticket < 0 || ticket >= (int)s->reqs.size()) return ADI_EINVAL;
    const Request &q = s->reqs[ticket];
    if (state) *state = q.state;
    if (t_submit) *t_submit = q.t_submit;
    if (t_start) *t_start = q.t_start;
    if (t_done) *t_done = q.t_done;
    return ADI_OK;
}

int adi_server_result(adi_server s, int ticket, double *u, double *v, double *w) {
    if (!s || ticket < 0 || ticket >= (int)s->reqs.size()) return ADI_EINVAL;
    const Request &q = s->reqs[ticket];
    if (q.state != ADI_REQ_DONE) return q.state == ADI_REQ_FAILED ? ADI_ECUDA : ADI_EBUSY;
    if (u) std::copy(q.ru.begin(), q.ru.end(), u);
    if (v) std::copy(q.rv.begin(), q.rv.end(), v);
    if (w) std::copy(q.rw.begin(), q.rw.end(), w);
    return ADI_OK;
}

size_t adi_server_used_bytes(adi_server s) { return s ? s->used : 0; }

int adi_server_destroy(adi_server s) {
    if (!s) return ADI_OK;
    drop_batch(s);
    for (int t : s->running) {
        adi_destroy(s->reqs[t].sim);
        s->reqs[t].sim = nullptr;
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    (void)cudaGetLastError();
    delete s;
    return ADI_OK;
}

}  // extern "C"
