// vla_server.cu -- the assembly server: continuous batching over a device
// memory budget (host runtime around the batched assembly kernel).
//
// A request names a mesh (host arrays plus a client key) and a coefficient.
// The scheduler admits requests in arrival order while the budget has room,
// ingest threads build the meshes of admitted requests on their own streams
// (H2D copy, vla_mesh_create) while earlier requests assemble, and every
// scheduling step takes ALL requests whose meshes are ready and assembles
// them in one batched persistent launch on the assembly stream.  Requests
// that arrive while a launch runs join the next one.  Meshes stay resident
// under their key and later requests with the same key skip the ingest; idle
// resident meshes are evicted, least recently used first, when an admission
// needs room.  Results stay on the device until the client releases them.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vla_internal.cuh"

namespace vla {
namespace {

double now_s() {   // CLOCK_MONOTONIC seconds (the clock of time.monotonic())
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SMesh {                 // a mesh on the device, private to a request or resident under a key
    int64_t key = -1;
    vla_mesh *mesh = nullptr;
    int64_t charged = 0;       // budget charged (estimate until built, then the handle's device bytes)
    int refs = 0;              // requests holding it
    bool building = false, built = false;
    vla_status status = VLA_OK;
    uint64_t last_use = 0;
    bool resident = false;
};

enum State { QUEUED, WAIT_MESH, INGEST, READY, RUNNING, DONE, FAILED };

struct SReq {
    int64_t ticket = 0;
    vla_request_t r;
    State state = QUEUED;
    SMesh *m = nullptr;
    bool new_mesh = false;
    void *out = nullptr;       // K | M | vol on the device
    int64_t out_charged = 0;
    vla_status status = VLA_OK;
    double t_submit = 0, t_admit = 0, t_ready = 0, t_start = 0, t_done = 0;
    double t_ingest = 0, h2d_ms = 0, build_ms = 0;   // ingest split: pickup time, device copy and build
    int32_t batch_size = 0;
    int64_t batch_id = -1;
    bool holds_mesh = false;   // counted in m->refs
};

}  // namespace
}  // namespace vla

using namespace vla;

struct vla_server {
    vla_server_config_t cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable sched_cv, ingest_cv, done_cv, reap_cv;
    std::unordered_map<int64_t, SReq *> reqs;
    std::deque<SReq *> queue;          // submitted, not admitted (arrival order)
    std::deque<SReq *> ingest_q;       // admitted, their mesh needs a build
    std::vector<SReq *> ready;         // mesh built: waiting for the next launch
    std::unordered_map<int64_t, SMesh *> by_key;
    std::vector<SMesh *> meshes;       // every live mesh
    std::vector<SMesh *> dead;         // meshes to destroy (outside the lock)
    std::vector<void *> dead_out;      // output blocks to free
    int64_t used = 0, peak = 0;
    int64_t next_ticket = 0, next_batch = 0;
    uint64_t clock = 0;
    bool stop = false;
    bool inflight = false;
    int64_t n_done = 0, n_failed = 0, n_batches = 0, n_evicted = 0, n_ingested = 0, n_reused = 0;
    int64_t batched_reqs = 0, max_batch_seen = 0;
    double busy_s = 0, t_launch = 0;
    int64_t live = 0;                  // admitted requests not finished yet
    cudaStream_t astream = nullptr;    // assembly launches and output allocations
    cudaStream_t fstream = nullptr;    // frees
    std::thread sched, reaper;
    std::vector<std::thread> workers;
};

namespace {

struct Batch {   // one batched launch in flight
    vla_server *srv;
    std::vector<SReq *> reqs;
    int64_t id;
};

int nlb_of(int dim, int order) { return order == 1 ? dim + 1 : (dim + 1) * (dim + 2) / 2; }

// budget estimate of a mesh handle before it is built: an upper bound on the
// pattern (nnz <= ne nlb^2), tiles and build scratch
int64_t mesh_estimate(const vla_request_t &r) {
    const int64_t nlb = nlb_of(r.dim, r.order);
    return r.ne * (nlb * nlb * 16 + nlb * 40) + r.nn * 128 + r.nfb * 24 + (4 << 20);
}
int64_t out_bytes(int64_t nnz, int64_t ne) { return ((16 * nnz + 8 * ne + 255) / 256) * 256 + 256; }
int64_t out_estimate(const vla_request_t &r) {
    const int64_t nlb = nlb_of(r.dim, r.order);
    return out_bytes(std::min(r.ne * nlb * nlb, r.nn * r.nn), r.ne);
}

void charge(vla_server *s, int64_t b) {
    s->used += b;
    s->peak = std::max(s->peak, s->used);
}

// under the lock: evicts idle resident meshes (least recently used first)
// until `need` more bytes fit; returns whether they fit
bool make_room(vla_server *s, int64_t need) {
    while (s->used + need > s->cfg.hbm_budget_bytes) {
        SMesh *victim = nullptr;
        for (SMesh *m : s->meshes)
            if (m->resident && m->refs == 0 && m->built && (!victim || m->last_use < victim->last_use)) victim = m;
        if (!victim) return false;
        s->by_key.erase(victim->key);
        s->meshes.erase(std::find(s->meshes.begin(), s->meshes.end(), victim));
        s->used -= victim->charged;
        s->dead.push_back(victim);
        ++s->n_evicted;
    }
    return true;
}

void finish(vla_server *s, SReq *q, vla_status st) {   // under the lock
    if (q->t_admit > 0) --s->live;
    q->status = st;
    q->state = st == VLA_OK ? DONE : FAILED;
    q->t_done = now_s();
    if (st == VLA_OK) ++s->n_done;
    else ++s->n_failed;
}

// under the lock: admission in arrival order while the budget has room
void admit(vla_server *s) {
    while (!s->queue.empty()) {
        SReq *q = s->queue.front();
        const vla_request_t &r = q->r;
        SMesh *m = nullptr;
        if (r.key >= 0) {
            auto it = s->by_key.find(r.key);
            if (it != s->by_key.end()) m = it->second;
        }
        const int64_t mneed = m ? 0 : mesh_estimate(r);
        const int64_t oneed = (m && m->built) ? out_bytes(m->mesh->nnz, m->mesh->ne) : out_estimate(r);
        if (mneed + oneed > s->cfg.hbm_budget_bytes) {
            s->queue.pop_front();
            finish(s, q, VLA_ERR_BUDGET);
            s->done_cv.notify_all();
            continue;
        }
        if (s->cfg.max_inflight > 0 && s->live >= s->cfg.max_inflight) return;
        // the mesh this request reuses must not be the one evicted to make room for it
        if (m) m->refs++;
        const bool room = make_room(s, mneed + oneed);
        if (m) m->refs--;
        if (!room) return;   // head of line waits for memory
        s->queue.pop_front();
        ++s->live;
        q->t_admit = now_s();
        q->out_charged = oneed;
        charge(s, oneed);
        if (!m) {
            m = new SMesh();
            m->key = r.key;
            m->resident = r.key >= 0 && r.keep_resident;
            m->charged = mneed;
            m->building = true;
            charge(s, mneed);
            s->meshes.push_back(m);
            if (r.key >= 0) s->by_key[r.key] = m;
            q->new_mesh = true;
            q->m = m;
            q->holds_mesh = true;
            m->refs++;
            m->last_use = ++s->clock;
            q->state = INGEST;
            s->ingest_q.push_back(q);
            s->ingest_cv.notify_one();
        } else {
            q->m = m;
            q->holds_mesh = true;
            m->refs++;
            m->last_use = ++s->clock;
            if (r.keep_resident) m->resident = true;
            ++s->n_reused;
            if (m->built) {
                q->state = READY;
                q->t_ready = now_s();
                s->ready.push_back(q);
            } else {
                q->state = WAIT_MESH;   // its mesh is being built for an earlier request
            }
        }
    }
}

// host callback at the end of a batched launch (no CUDA calls here)
void CUDART_CB batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    vla_server *s = b->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        s->busy_s += t - s->t_launch;
        for (SReq *q : b->reqs) {
            finish(s, q, VLA_OK);
            q->t_done = t;
        }
        s->inflight = false;
    }
    s->done_cv.notify_all();
    s->sched_cv.notify_all();
    delete b;
}

void destroy_dead(vla_server *s, std::vector<SMesh *> &dead, std::vector<void *> &outs) {
    for (SMesh *m : dead) {
        if (m->mesh) {
            m->mesh->stream = s->fstream;   // free on the idle free stream, not the ingest stream that built it
            vla_mesh_destroy(m->mesh);
        }
        delete m;
    }
    for (void *o : outs) cudaFreeAsync(o, s->fstream);
    if (!outs.empty()) cudaStreamSynchronize(s->fstream);
}

void scheduler(vla_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (!s->dead.empty() || !s->dead_out.empty()) s->reap_cv.notify_one();
        if (s->stop && s->queue.empty() && s->ingest_q.empty() && s->ready.empty() && !s->inflight) {
            bool busy = false;
            for (auto &kv : s->reqs)
                if (kv.second->state == INGEST || kv.second->state == WAIT_MESH) busy = true;
            if (!busy) break;
        }
        admit(s);
        if (!s->dead.empty()) s->reap_cv.notify_one();   // evictions made room
        if (!s->inflight && !s->ready.empty()) {
            std::vector<SReq *> take;
            const size_t cap = s->cfg.max_batch > 0 ? (size_t)s->cfg.max_batch : s->ready.size();
            const size_t n = std::min(cap, s->ready.size());
            take.assign(s->ready.begin(), s->ready.begin() + n);
            s->ready.erase(s->ready.begin(), s->ready.begin() + n);
            s->inflight = true;
            const int64_t bid = s->next_batch++;
            lk.unlock();
            // outputs are allocated on the assembly stream, in stream order with the launch
            std::vector<vla_batch_job_t> jobs(n);
            vla_status st = VLA_OK;
            for (size_t i = 0; i < n && st == VLA_OK; ++i) {
                SReq *q = take[i];
                const vla_mesh *m = q->m->mesh;
                const size_t ob = (size_t)out_bytes(m->nnz, m->ne);
                if (pool_malloc((void **)&q->out, ob, s->astream) != cudaSuccess) {
                    cudaGetLastError();
                    q->out = nullptr;
                    st = fail(VLA_ERR_OOM, "server outputs: out of device memory");
                    break;
                }
                double *K = static_cast<double *>(q->out);
                vla_batch_job_t &j = jobs[i];
                memset(&j, 0, sizeof(j));
                j.mesh = m;
                j.coeff_kind = q->r.coeff_kind;
                j.ca = q->r.ca;
                j.cb = q->r.cb;
                j.K_vals = K;
                j.M_vals = K + m->nnz;
                j.vol = K + 2 * m->nnz;
            }
            const double t = now_s();
            if (st == VLA_OK) st = vla_batch_assemble(jobs.data(), (int32_t)n, s->cfg.precision, nullptr, s->astream);
            Batch *b = nullptr;
            if (st == VLA_OK) {
                b = new Batch{s, take, bid};
                for (SReq *q : take) {
                    q->batch_size = (int32_t)n;
                    q->batch_id = bid;
                }
            }
            lk.lock();
            s->t_launch = t;
            for (SReq *q : take) {
                q->t_start = t;
                q->state = RUNNING;
            }
            ++s->n_batches;
            s->batched_reqs += (int64_t)n;
            s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, (int64_t)n);
            if (st != VLA_OK) {
                for (SReq *q : take) finish(s, q, st);
                s->inflight = false;
                s->done_cv.notify_all();
                continue;
            }
            lk.unlock();
            if (cudaLaunchHostFunc(s->astream, batch_done, b) != cudaSuccess) {
                cudaGetLastError();
                cudaStreamSynchronize(s->astream);
                batch_done(b);
            }
            lk.lock();
            continue;
        }
        s->sched_cv.wait(lk);
    }
}

// frees evicted or released meshes and outputs off the scheduler's path
void reaper(vla_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        while (s->dead.empty() && s->dead_out.empty() && !s->stop) s->reap_cv.wait(lk);
        if (s->dead.empty() && s->dead_out.empty()) break;   // stopping, nothing left
        std::vector<SMesh *> dead;
        std::vector<void *> outs;
        dead.swap(s->dead);
        outs.swap(s->dead_out);
        lk.unlock();
        destroy_dead(s, dead, outs);
        lk.lock();
    }
}

void ingest_worker(vla_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t ws = nullptr;
    cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        while (s->ingest_q.empty() && !s->stop) s->ingest_cv.wait(lk);
        if (s->ingest_q.empty() && s->stop) break;
        SReq *q = s->ingest_q.front();
        s->ingest_q.pop_front();
        SMesh *sm = q->m;
        const vla_request_t r = q->r;
        q->t_ingest = now_s();
        lk.unlock();
        // H2D of the request's arrays into stream-ordered staging, then the device build
        const size_t cb = sizeof(double) * r.dim * r.nn, eb = sizeof(int32_t) * nlb_of(r.dim, r.order) * r.ne,
                     fb = sizeof(int32_t) * r.dim * r.nfb;
        void *stage = nullptr;
        vla_status st = VLA_OK;
        vla_mesh *mesh = nullptr;
        if (pool_malloc((void **)&stage, cb + eb + fb + 512, ws) != cudaSuccess) {
            cudaGetLastError();
            stage = nullptr;
            st = fail(VLA_ERR_OOM, "server staging: out of device memory");
        }
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
            }
        if (ev[0]) cudaEventRecord(ev[0], ws);
        if (st == VLA_OK) {
            unsigned char *p = static_cast<unsigned char *>(stage);
            double *dc = reinterpret_cast<double *>(p);
            int32_t *de = reinterpret_cast<int32_t *>(p + (cb + 255) / 256 * 256);
            int32_t *df = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(de) + (eb + 255) / 256 * 256);
            if (cudaMemcpyAsync(dc, r.coords, cb, cudaMemcpyDefault, ws) != cudaSuccess ||
                cudaMemcpyAsync(de, r.elems, eb, cudaMemcpyDefault, ws) != cudaSuccess ||
                (fb && cudaMemcpyAsync(df, r.faces, fb, cudaMemcpyDefault, ws) != cudaSuccess)) {
                st = cuda_fail(cudaGetLastError(), "server input copy");
            } else {
                if (ev[1]) cudaEventRecord(ev[1], ws);
                st = vla_mesh_create(r.dim, r.order, r.nn, r.ne, dc, de, r.nfb, fb ? df : nullptr, ws, &mesh);
                if (ev[2]) cudaEventRecord(ev[2], ws);
            }
        }
        if (stage) cudaFreeAsync(stage, ws);
        cudaStreamSynchronize(ws);
        float h2d_ms = 0.f, build_ms = 0.f;
        if (st == VLA_OK && ev[0] && ev[1] && ev[2]) {
            if (cudaEventElapsedTime(&h2d_ms, ev[0], ev[1]) != cudaSuccess ||
                cudaEventElapsedTime(&build_ms, ev[1], ev[2]) != cudaSuccess) {
                cudaGetLastError();
                h2d_ms = build_ms = 0.f;
            }
        }
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        lk.lock();
        ++s->n_ingested;
        q->h2d_ms = h2d_ms;
        q->build_ms = build_ms;
        sm->building = false;
        s->used -= sm->charged;
        if (st == VLA_OK) {
            sm->mesh = mesh;
            sm->built = true;
            sm->charged = mesh->device_bytes;
            charge(s, sm->charged);
        } else {
            sm->status = st;
            sm->charged = 0;
            if (sm->key >= 0) s->by_key.erase(sm->key);
        }
        // this request and every request that waited for the same mesh
        const double t = now_s();
        std::vector<SReq *> users;
        for (auto &kv : s->reqs)
            if (kv.second->m == sm && (kv.second->state == INGEST || kv.second->state == WAIT_MESH))
                users.push_back(kv.second);
        for (SReq *u : users) {
            if (st == VLA_OK) {
                s->used -= u->out_charged;   // the exact output size is known now
                u->out_charged = out_bytes(mesh->nnz, mesh->ne);
                charge(s, u->out_charged);
                u->state = READY;
                u->t_ready = t;
                s->ready.push_back(u);
            } else {
                s->used -= u->out_charged;
                u->out_charged = 0;
                sm->refs--;
                u->holds_mesh = false;
                finish(s, u, st);
            }
        }
        if (st != VLA_OK && sm->refs == 0) {
            s->meshes.erase(std::find(s->meshes.begin(), s->meshes.end(), sm));
            s->dead.push_back(sm);
        }
        s->sched_cv.notify_all();
        s->done_cv.notify_all();
    }
    lk.unlock();
    cudaStreamDestroy(ws);
}

}  // namespace

extern "C" vla_status vla_server_create(const vla_server_config_t *cfg, vla_server **out) {
    if (!cfg || !out) return fail(VLA_ERR_INVALID_ARG, "null config or out");
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0) return fail(VLA_ERR_INVALID_ARG, "hbm_budget_bytes must be positive");
    if (cfg->precision != VLA_PREC_FP64 && cfg->precision != VLA_PREC_MIXED)
        return fail(VLA_ERR_INVALID_ARG, "precision must be VLA_PREC_FP64 or VLA_PREC_MIXED");
    if (cfg->ingest_workers < 0 || cfg->ingest_workers > 64 || cfg->max_batch < 0 || cfg->max_inflight < 0)
        return fail(VLA_ERR_INVALID_ARG, "ingest_workers in [0, 64], max_batch and max_inflight >= 0");
    vla_server *s = new (std::nothrow) vla_server();
    if (!s) return fail(VLA_ERR_OOM, "host allocation failed");
    s->cfg = *cfg;
    if (s->cfg.ingest_workers == 0) s->cfg.ingest_workers = 4;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->astream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (s->astream) cudaStreamDestroy(s->astream);
        delete s;
        return cuda_fail(e, "server streams");
    }
    s->sched = std::thread(scheduler, s);
    s->reaper = std::thread(reaper, s);
    for (int i = 0; i < s->cfg.ingest_workers; ++i) s->workers.emplace_back(ingest_worker, s);
    *out = s;
    return VLA_OK;
}

extern "C" vla_status vla_server_submit(vla_server *s, const vla_request_t *r, int64_t *ticket) {
    if (!s || !r || !ticket) return fail(VLA_ERR_INVALID_ARG, "null server, request or ticket");
    if (r->dim != 2 && r->dim != 3) return fail(VLA_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (r->order != VLA_P1 && r->order != VLA_P2) return fail(VLA_ERR_INVALID_ARG, "order must be VLA_P1 or VLA_P2");
    if (r->nn < 1 || r->ne < 1 || r->nfb < 0 || !r->coords || !r->elems || (r->nfb > 0 && !r->faces))
        return fail(VLA_ERR_INVALID_ARG, "bad mesh arrays or sizes");
    if (r->coeff_kind != VLA_COEFF_POLY && r->coeff_kind != VLA_COEFF_EXP)
        return fail(VLA_ERR_INVALID_ARG, "unknown coefficient kind");
    SReq *q = new (std::nothrow) SReq();
    if (!q) return fail(VLA_ERR_OOM, "host allocation failed");
    q->r = *r;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete q;
            return fail(VLA_ERR_INVALID_ARG, "server is shutting down");
        }
        q->ticket = s->next_ticket++;
        s->reqs[q->ticket] = q;
        s->queue.push_back(q);
        *ticket = q->ticket;
    }
    s->sched_cv.notify_all();
    return VLA_OK;
}

extern "C" vla_status vla_server_poll(vla_server *s, int64_t ticket, double timeout_s, vla_result_t *res) {
    if (!s) return fail(VLA_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(VLA_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    SReq *q = it->second;
    if (timeout_s > 0) {
        const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
        while (q->state != DONE && q->state != FAILED)
            if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout) break;
    }
    if (q->state != DONE && q->state != FAILED) return VLA_PENDING;
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = q->status;
        res->new_mesh = q->new_mesh ? 1 : 0;
        res->batch_size = q->batch_size;
        res->batch_id = q->batch_id;
        res->t_submit = q->t_submit;
        res->t_admit = q->t_admit;
        res->t_ready = q->t_ready;
        res->t_start = q->t_start;
        res->t_done = q->t_done;
        res->t_ingest = q->t_ingest;
        res->h2d_ms = q->h2d_ms;
        res->build_ms = q->build_ms;
        if (q->state == DONE) {
            const vla_mesh *m = q->m->mesh;
            res->nn = m->nn;
            res->ne = m->ne;
            res->nnz = m->nnz;
            const double *K = static_cast<const double *>(q->out);
            res->K_vals = K;
            res->M_vals = K + m->nnz;
            res->vol = K + 2 * m->nnz;
            res->row_ptr = m->row_ptr;
            res->col_idx = m->col_idx;
        }
    }
    if (q->status < 0) return fail(q->status, "request %lld failed (status %d)", (long long)ticket, (int)q->status);
    return VLA_OK;
}

extern "C" vla_status vla_server_release(vla_server *s, int64_t ticket) {
    if (!s) return fail(VLA_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(VLA_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
        SReq *q = it->second;
        if (q->state != DONE && q->state != FAILED)
            return fail(VLA_ERR_INVALID_ARG, "request %lld is not finished", (long long)ticket);
        s->reqs.erase(it);
        s->used -= q->out_charged;
        if (q->out) s->dead_out.push_back(q->out);
        if (q->m && q->holds_mesh) {
            SMesh *m = q->m;
            q->holds_mesh = false;
            m->refs--;
            if (m->refs == 0 && !m->resident) {
                if (m->key >= 0) s->by_key.erase(m->key);
                s->meshes.erase(std::find(s->meshes.begin(), s->meshes.end(), m));
                s->used -= m->charged;
                s->dead.push_back(m);
            }
        }
        delete q;
    }
    s->sched_cv.notify_all();
    s->reap_cv.notify_one();
    return VLA_OK;
}

extern "C" vla_status vla_server_stats(vla_server *s, vla_server_stats_t *st) {
    if (!s || !st) return fail(VLA_ERR_INVALID_ARG, "null server or stats");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->used_bytes = s->used;
    st->peak_bytes = s->peak;
    st->budget_bytes = s->cfg.hbm_budget_bytes;
    st->n_done = s->n_done;
    st->n_failed = s->n_failed;
    st->n_batches = s->n_batches;
    st->n_ingested = s->n_ingested;
    st->n_reused = s->n_reused;
    st->n_evicted = s->n_evicted;
    st->max_batch = s->max_batch_seen;
    st->mean_batch = s->n_batches ? (double)s->batched_reqs / s->n_batches : 0.0;
    st->assembly_busy_s = s->busy_s;
    int64_t res = 0;
    for (SMesh *m : s->meshes)
        if (m->resident) ++res;
    st->n_resident = res;
    st->n_queued = (int64_t)s->queue.size();
    return VLA_OK;
}

extern "C" vla_status vla_server_destroy(vla_server *s) {
    if (!s) return VLA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests not admitted yet are dropped
        for (SReq *q : s->queue) finish(s, q, VLA_ERR_INVALID_ARG);
        s->queue.clear();
    }
    s->sched_cv.notify_all();
    s->ingest_cv.notify_all();
    s->done_cv.notify_all();
    for (auto &w : s->workers) w.join();
    if (s->sched.joinable()) s->sched.join();
    s->reap_cv.notify_all();
    if (s->reaper.joinable()) s->reaper.join();
    cudaStreamSynchronize(s->astream);
    std::vector<SMesh *> dead = s->meshes;
    dead.insert(dead.end(), s->dead.begin(), s->dead.end());
    std::vector<void *> outs = s->dead_out;
    for (auto &kv : s->reqs) {
        if (kv.second->out) outs.push_back(kv.second->out);
        delete kv.second;
    }
    destroy_dead(s, dead, outs);
    cudaStreamDestroy(s->astream);
    cudaStreamDestroy(s->fstream);
    delete s;
    return VLA_OK;
}
