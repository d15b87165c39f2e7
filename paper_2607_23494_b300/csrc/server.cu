// Request server: continuous batching of measurement requests on one GPU.
//
// Requests (a catalogue plus a statistic: xi, xi_l or zeta_l on some grid and
// shells) are queued by hermes_server_submit and executed by worker threads,
// each with its own CUDA stream, so the work of several requests overlaps on
// the device.  A request is admitted when its device footprint (estimated
// before it runs, measured after) fits in the server's HBM budget next to the
// requests in flight and the idle resident contexts; idle contexts are evicted
// least-recently-used first to make room.  A request that has been passed over
// by later, smaller requests too many times blocks further admissions until it
// fits, so large requests are not starved.
//
// Reconstructed fields stay resident: a context keeps the field of the last
// catalogue it assigned, keyed by the caller's field_id, and a later request
// with the same (L, N, p, field_id) skips the scatter and forward transform.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hermes.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Slot {
    hermes_ctx* ctx = nullptr;
    double L = 0;
    int N = 0, p = 0;
    int64_t field_id = -1;       // resident catalogue, -1: none
    std::vector<double> edges;   // shells of the resident tables
    int l_max = -1;
    int last_stat = -1;          // statistic of the last request (its buffers may still be held)
    bool busy = false;
    int64_t last_used = 0;
    int64_t bytes = 0;           // device footprint (measured after each use)
};

struct Request {
    int64_t ticket = 0;
    hermes_request r{};
    std::vector<double> edges;
    std::vector<int> ells;
    int64_t est = 0;              // estimated footprint
    int passed_over = 0;          // later requests admitted ahead of this one
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    hermes_result res{};
};

constexpr int kMaxPassOver = 8;

int request_l_max(const Request& q) {
    if (q.r.stat == HERMES_STAT_XI) return 0;
    if (q.r.stat == HERMES_STAT_ZETA) return q.r.l_max;
    return *std::max_element(q.ells.begin(), q.ells.end());
}

}  // namespace

struct hermes_server {
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;  // ticket -> request (until waited on)
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<std::thread> workers;
    int64_t next_ticket = 1;
    int64_t reserved = 0;        // footprints of busy requests plus idle slots
    int64_t clock = 0;
    int64_t completed = 0, in_flight = 0, peak_in_flight = 0, reused = 0, peak_reserved = 0, evicted = 0;
    std::vector<hermes_ctx*> graveyard;  // evicted contexts, destroyed outside the lock
    bool stop = false;
};

namespace {

int64_t idle_bytes(const hermes_server* s) {
    int64_t b = 0;
    for (auto& sl : s->slots)
        if (!sl->busy) b += sl->bytes;
    return b;
}

// Chooses a slot for q and the extra bytes it needs; -1 when none may be used
// now (its field is resident in a busy slot).  Called with the lock held.
int choose_slot(hermes_server* s, const Request& q, int64_t* extra) {
    int same_field = -1, same_grid = -1;
    for (int i = 0; i < (int)s->slots.size(); ++i) {
        const Slot& sl = *s->slots[i];
        if (sl.L != q.r.L || sl.N != q.r.N || sl.p != q.r.p) continue;
        if (q.r.field_id >= 0 && sl.field_id == q.r.field_id) {
            if (sl.busy) return -2;  // wait for the resident field instead of rebuilding it
            same_field = i;
        } else if (!sl.busy && (same_grid < 0 || sl.last_used < s->slots[same_grid]->last_used)) {
            same_grid = i;
        }
    }
    const int pick = same_field >= 0 ? same_field : same_grid;
    if (pick >= 0) {
        *extra = std::max<int64_t>(0, q.est - s->slots[pick]->bytes);
        return pick;
    }
    *extra = q.est;
    return (int)s->slots.size();  // a new slot
}

// Evicts idle slots (least recently used first, never `keep`) until `need`
// more bytes fit.  Returns true if they fit.  Lock held.
bool make_room(hermes_server* s, int64_t need, int keep) {
    while (s->reserved + need > s->budget) {
        int victim = -1;
        for (int i = 0; i < (int)s->slots.size(); ++i) {
            if (i == keep || s->slots[i]->busy) continue;
            if (victim < 0 || s->slots[i]->last_used < s->slots[victim]->last_used) victim = i;
        }
        if (victim < 0) return false;
        Slot* v = s->slots[victim].get();
        s->reserved -= v->bytes;
        s->graveyard.push_back(v->ctx);
        ++s->evicted;
        s->slots.erase(s->slots.begin() + victim);
    }
    return true;
}

// Next admissible request and its slot; nullptr if none.  Lock held.
Request* admit(hermes_server* s, int* slot_out, int64_t* extra_out) {
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Request* q = *it;
        int64_t extra = 0;
        int slot = choose_slot(s, *q, &extra);
        if (slot == -2) continue;
        if (q->est > s->budget) {  // can never fit: fail it now
            s->queue.erase(it);
            *slot_out = -1;
            return q;
        }
        const int keep = slot < (int)s->slots.size() ? slot : -1;
        bool fits = s->reserved + extra <= s->budget;
        if (!fits) {
            // evicting idle contexts is allowed only if the whole idle set would make room
            if (s->reserved - idle_bytes(s) + (keep >= 0 ? s->slots[keep]->bytes : 0) + extra <= s->budget &&
                make_room(s, extra, keep)) {
                slot = choose_slot(s, *q, &extra);  // indices shift when slots are evicted
                fits = slot >= 0 && s->reserved + extra <= s->budget;
            }
        }
        if (!fits) {
            if (q->passed_over >= kMaxPassOver) return nullptr;  // nobody overtakes it any more
            continue;
        }
        for (auto jt = s->queue.begin(); jt != it; ++jt) ++(*jt)->passed_over;
        s->queue.erase(it);
        *slot_out = slot;
        *extra_out = extra;
        return q;
    }
    return nullptr;
}

void set_result(Request* q, int status, const char* msg) {
    q->res.status = status;
    std::snprintf(q->res.msg, sizeof(q->res.msg), "%s", msg ? msg : "");
}

// Runs one request on slot sl, owned by this worker while busy.  Only the
// context, its stream and the resident shells are touched here; the slot's
// identity (L, N, p, field_id) is kept by the scheduler under the lock.
int execute(Slot* sl, Request* q, cudaStream_t st, bool reuse) {
    const hermes_request& r = q->r;
    int rc;
    if (!sl->ctx) {
        const int j = 31 - __builtin_clz((unsigned)r.N);
        hermes_ctx* c = nullptr;
        if ((rc = hermes_create(r.L, r.N, r.p, j, &c)) != HERMES_OK) {
            set_result(q, rc, "hermes_create failed");
            return rc;
        }
        sl->ctx = c;
    }
    hermes_ctx* c = sl->ctx;
    hermes_set_stream(c, st);
    // a context changing statistic first drops the other statistic's buffers (the harmonic
    // fields of zeta_l, the window batch of xi), so it never holds both: admission reserved
    // only the larger of its previous footprint and this request's estimate
    if (sl->last_stat >= 0 && (sl->last_stat == HERMES_STAT_ZETA) != (r.stat == HERMES_STAT_ZETA)) {
        if ((rc = hermes_release_buffers(c)) != HERMES_OK) {
            set_result(q, rc, hermes_last_error(c));
            return rc;
        }
    }
    sl->last_stat = r.stat;
    const int lmax = request_l_max(*q);
    if (sl->edges != q->edges || sl->l_max < lmax) {
        if ((rc = hermes_window_shells(c, q->edges.data(), (int)q->edges.size(), lmax)) != HERMES_OK) {
            set_result(q, rc, hermes_last_error(c));
            sl->edges.clear();
            sl->l_max = -1;
            return rc;
        }
        sl->edges = q->edges;
        sl->l_max = lmax;
    }
    if (!reuse) {
        if (!r.pos) {
            set_result(q, HERMES_ERR_ARG, "pos is NULL and no resident field has this field_id");
            return HERMES_ERR_ARG;
        }
        if ((rc = hermes_assign(c, r.pos, r.w, r.n, r.flags)) != HERMES_OK) {
            set_result(q, rc, hermes_last_error(c));
            return rc;
        }
    }
    if (r.stat == HERMES_STAT_XI) rc = hermes_xi(c, r.out);
    else if (r.stat == HERMES_STAT_XI_MULTIPOLES) rc = hermes_xi_multipoles(c, q->ells.data(), (int)q->ells.size(), r.out);
    else rc = hermes_zeta_multipoles(c, r.out);
    set_result(q, rc, rc == HERMES_OK ? "" : hermes_last_error(c));
    return rc;
}

void worker_main(hermes_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        Request* q = nullptr;
        int slot = -1;
        int64_t extra = 0;
        s->cv_work.wait(lk, [&] { return s->stop || (q = admit(s, &slot, &extra)) != nullptr; });
        if (!q) break;  // stopping
        q->t_start = Clock::now();
        if (slot < 0) {  // larger than the whole budget
            q->res.queue_ms = ms_between(q->t_submit, q->t_start);
            set_result(q, HERMES_ERR_NOMEM, "the request's device footprint exceeds the server's HBM budget");
            q->t_done = q->t_start;
            q->done = true;
            s->cv_done.notify_all();
            continue;
        }
        if (slot == (int)s->slots.size()) {
            s->slots.emplace_back(new Slot);
            s->slots.back()->L = q->r.L;
            s->slots.back()->N = q->r.N;
            s->slots.back()->p = q->r.p;
        }
        Slot* sl = s->slots[slot].get();
        sl->busy = true;
        const bool reuse = q->r.field_id >= 0 && sl->field_id == q->r.field_id;
        if (!reuse) sl->field_id = q->r.field_id;  // requests for this field now wait for the slot
        s->reserved += extra;
        const int64_t held = sl->bytes + extra;  // this request's share of `reserved`
        s->peak_reserved = std::max(s->peak_reserved, s->reserved);
        ++s->in_flight;
        s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
        std::vector<hermes_ctx*> dead;
        dead.swap(s->graveyard);
        lk.unlock();
        for (hermes_ctx* d : dead) {  // its last stream is some worker's: destroy on its own stream
            hermes_set_stream(d, nullptr);
            hermes_destroy(d);
        }

        int rc = HERMES_ERR_CUDA;
        if (st) rc = execute(sl, q, st, reuse);
        else set_result(q, HERMES_ERR_CUDA, "worker stream could not be created");
        const int64_t now_bytes = sl->ctx ? hermes_device_bytes(sl->ctx) : 0;
        q->t_done = Clock::now();

        lk.lock();
        if (rc != HERMES_OK && !reuse) sl->field_id = -1;  // the field may be partly built
        const bool reused = reuse && rc == HERMES_OK;
        s->reserved += now_bytes - held;
        sl->bytes = now_bytes;
        sl->busy = false;
        sl->last_used = ++s->clock;
        if (!sl->ctx) {  // creation failed: drop the slot
            for (size_t i = 0; i < s->slots.size(); ++i)
                if (s->slots[i].get() == sl) {
                    s->slots.erase(s->slots.begin() + i);
                    break;
                }
        }
        --s->in_flight;
        ++s->completed;
        if (reused) ++s->reused;
        q->res.reused_field = reused ? 1 : 0;
        q->res.queue_ms = ms_between(q->t_submit, q->t_start);
        q->res.latency_ms = ms_between(q->t_submit, q->t_done);
        q->res.device_bytes = now_bytes;
        q->done = true;
        s->cv_done.notify_all();
        s->cv_work.notify_all();  // memory or a resident field may have been freed
    }
    lk.unlock();
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int hermes_server_create(int device, int64_t hbm_budget, int n_streams, hermes_server** out) {
    if (!out || n_streams < 1 || n_streams > 64 || hbm_budget <= 0) return HERMES_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? HERMES_ERR_CUDA : HERMES_ERR_ARG;
    }
    hermes_server* s = new hermes_server;
    s->device = device;
    s->budget = hbm_budget;
    for (int i = 0; i < n_streams; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return HERMES_OK;
}

int hermes_server_submit(hermes_server* s, const hermes_request* r, int64_t* ticket) {
    if (!s || !r || !ticket) return HERMES_ERR_ARG;
    if (r->stat < HERMES_STAT_XI || r->stat > HERMES_STAT_ZETA || !r->r_edges || r->n_edges < 2 || !r->out)
        return HERMES_ERR_ARG;
    if (r->stat == HERMES_STAT_XI_MULTIPOLES && (!r->ells || r->n_ells < 1)) return HERMES_ERR_ARG;
    if (r->stat == HERMES_STAT_ZETA && r->l_max < 0) return HERMES_ERR_ARG;
    if (r->n < 0 || (r->n > 0 && !r->pos)) return HERMES_ERR_ARG;
    std::unique_ptr<Request> q(new Request);
    q->r = *r;
    q->edges.assign(r->r_edges, r->r_edges + r->n_edges);
    if (r->stat == HERMES_STAT_XI_MULTIPOLES) q->ells.assign(r->ells, r->ells + r->n_ells);
    const int lmax = request_l_max(*q);
    q->est = hermes_estimate_bytes(r->N, r->stat, r->n_edges - 1, lmax, r->n,
                                   (r->flags & HERMES_DEVICE_PTR) ? 0 : 1);
    if (q->est < 0) return HERMES_ERR_ARG;
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return HERMES_ERR_STATE;
    q->ticket = s->next_ticket++;
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs[q->ticket] = std::move(q);
    s->cv_work.notify_one();
    return HERMES_OK;
}

int hermes_server_wait(hermes_server* s, int64_t ticket, hermes_result* res) {
    if (!s || !res) return HERMES_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HERMES_ERR_ARG;
    Request* q = it->second.get();
    s->cv_done.wait(lk, [&] { return q->done; });
    *res = q->res;
    s->reqs.erase(it);
    return HERMES_OK;
}

int hermes_server_stats(hermes_server* s, int64_t* stats, int n) {
    if (!s || !stats || n < 1) return HERMES_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t v[9] = {s->completed, s->in_flight, (int64_t)s->queue.size(), s->reserved, s->peak_reserved,
                          s->peak_in_flight, s->reused, (int64_t)s->slots.size(), s->evicted};
    for (int i = 0; i < std::min(n, 9); ++i) stats[i] = v[i];
    return HERMES_OK;
}

int hermes_server_destroy(hermes_server* s) {
    if (!s) return HERMES_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests still queued fail; those running finish first
        for (Request* q : s->queue) {
            set_result(q, HERMES_ERR_STATE, "server destroyed before the request ran");
            q->done = true;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto& t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (auto& sl : s->slots)
        if (sl->ctx) {
            hermes_set_stream(sl->ctx, nullptr);
            hermes_destroy(sl->ctx);
        }
    for (hermes_ctx* d : s->graveyard) {
        hermes_set_stream(d, nullptr);
        hermes_destroy(d);
    }
    delete s;
    return HERMES_OK;
}

}  // extern "C"
