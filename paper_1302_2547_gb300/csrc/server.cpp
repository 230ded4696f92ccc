// server.cpp -- a solve service on one GPU: requests (matrix, right-hand side, tolerance)
// are queued, admitted against a device-memory budget, served from a cache of device-
// resident hierarchies keyed by the matrix, and batched: a worker takes the queued requests
// of every idle matrix at once, requests for one matrix as the columns of one system and
// different matrices as the systems of one uaamg_solve_batch call (their K-cycles advance
// level step by level step together), and worker threads with their own CUDA streams keep
// several batches in flight.  Host-side orchestration only: every compute step is a
// libuaamg kernel.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "uaamg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Matrix {
    uint64_t key = 0;
    int32_t n = 0, nnz = 0;
    std::vector<int32_t> rowptr, col;
    std::vector<double> val;
};

struct Request {
    uint64_t ticket = 0;
    std::shared_ptr<Matrix> A;
    std::vector<double> b;
    double tol = 1e-8;
    Clock::time_point t_submit;
    // result
    std::vector<double> x;
    int32_t status = -1, iters = 0, batch = 0, cache_hit = 0;
    double relres = 0.0, latency_ms = 0.0;
    double queue_ms = 0.0, setup_ms = 0.0, solve_ms = 0.0;
    bool done = false;
};

struct CacheEntry {
    uint64_t key;
    uaamg_handle* h = nullptr;
    uint64_t bytes = 0;  // device bytes counted against the budget: the handle's own once it
                         // exists, plus what the batch using it reserved for its workspace
    int users = 0;       // workers currently solving with it
    cudaStream_t stream = nullptr;
};

// 64-bit FNV-1a over the CSR arrays: the cache key of a matrix when the caller gives none.
uint64_t fnv1a(const void* p, size_t bytes, uint64_t h) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; i++) {
        h ^= c[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

// The library-wide device-memory cap while services live: the sum of their budgets.
std::mutex g_budget_mu;
uint64_t g_budget_sum = 0;
int g_budget_servers = 0;

void add_budget(uint64_t b, int sign) {
    std::lock_guard<std::mutex> lk(g_budget_mu);
    if (sign > 0) {
        g_budget_sum += b;
        g_budget_servers++;
    } else {
        g_budget_sum -= b;
        g_budget_servers--;
    }
    uaamg_set_memory_budget(g_budget_servers > 0 ? g_budget_sum : 0);
}

}  // namespace

struct uaamg_server {
    uaamg_params params{};
    uint64_t budget = 0;
    int max_batch = 16;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    std::list<CacheEntry> cache;  // most recently used first
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int device = 0;
    // statistics
    uint64_t n_done = 0, n_batches = 0, n_hits = 0, n_setups = 0, n_rejected = 0;
    uint64_t n_cancelled = 0;

    CacheEntry* find(uint64_t key) {
        for (auto it = cache.begin(); it != cache.end(); ++it)
            if (it->key == key) {
                cache.splice(cache.begin(), cache, it);
                return &cache.front();
            }
        return nullptr;
    }
    // Device bytes this service's cached hierarchies may hold (their admission estimates).
    uint64_t held() const {
        uint64_t b = 0;
        for (auto& e : cache) b += e.bytes;
        return b;
    }
    // Evicts least recently used idle hierarchies until `need` more bytes fit the budget.
    bool make_room(uint64_t need) {
        if (!budget) return true;
        while (held() + need > budget) {
            auto victim = cache.end();
            for (auto it = cache.begin(); it != cache.end(); ++it)
                if (it->users == 0) victim = it;
            if (victim == cache.end()) return false;
            uaamg_free(victim->h);
            if (victim->stream) cudaStreamDestroy(victim->stream);
            cache.erase(victim);
        }
        return true;
    }
    void worker_main(int wid);
};

// Device bytes a hierarchy of this matrix may take (level 0 plus coarse levels, smoother
// data, setup scratch, and the solve workspace of `cols` right-hand sides): an upper bound
// used for admission before the setup or solve runs.
static uint64_t estimate_bytes(const Matrix& A, int cols) {
    const uint64_t n = (uint64_t)A.n, z = (uint64_t)A.nnz;
    return 2 * (16 * z + 120 * n) + (uint64_t)cols * n * 96 + (64ULL << 20);
}

// The device bytes a handle holds now.
static uint64_t handle_bytes(uaamg_handle* h) {
    uaamg_stats st{};
    return (h && uaamg_get_stats(h, &st) == UAAMG_OK) ? st.device_bytes : 0;
}

namespace {
// One system of a batch: the requests for one matrix (its columns) and its hierarchy.
struct Group {
    std::vector<std::shared_ptr<Request>> reqs;
    CacheEntry* entry = nullptr;
    bool need_setup = false;
    int status = UAAMG_OK;
};
}  // namespace

void uaamg_server::worker_main(int wid) {
    (void)wid;
    cudaSetDevice(device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    // the many-system solve needs one sweep before and after the coarse correction
    const bool cross = params.pre == 1 && params.post == 1;
    const int cols = std::min(max_batch, 32);
    while (true) {
        std::vector<Group> groups;
        int taken = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            // a handle serves one thread at a time: requests for a matrix another worker
            // is setting up or solving wait, and join a later batch
            auto idle = [&](uint64_t key) {
                for (auto& e : cache)
                    if (e.key == key && e.users > 0) return false;
                return true;
            };
            cv_work.wait(lk, [&] {
                if (stopping && queue.empty()) return true;
                for (auto& q : queue)
                    if (idle(q->A->key)) return true;
                return false;
            });
            if (stopping && queue.empty()) break;
            // continuous batching: in arrival order, every queued request of an idle matrix
            // with the first one's tolerance, up to max_batch requests; requests for one
            // matrix become the columns of one system, different matrices different systems
            // of one uaamg_solve_batch call
            double tol = 0.0;
            bool rejected = false, wait_memory = false;
            std::unordered_map<uint64_t, size_t> gi;
            // a group's entry counts at least the estimate for its columns so far
            auto reserve = [&](CacheEntry* e, const Matrix& A, int R) {
                const uint64_t need = estimate_bytes(A, R);
                if (e->bytes >= need) return true;
                if (!make_room(need - e->bytes)) return false;
                e->bytes = need;
                return true;
            };
            for (auto it = queue.begin(); it != queue.end() && taken < max_batch;) {
                std::shared_ptr<Request> q = *it;
                const uint64_t key = q->A->key;
                auto f = gi.find(key);
                const bool joins = f != gi.end();
                if ((!joins && !idle(key)) || (taken > 0 && q->tol != tol) ||
                    (joins && (int)groups[f->second].reqs.size() >= cols) ||
                    (!cross && taken > 0 && !joins)) {
                    ++it;
                    continue;
                }
                if (!joins) {  // a new system: cached, or set up by this worker within budget
                    Group g;
                    g.entry = find(key);
                    if (!g.entry) {
                        const uint64_t need = estimate_bytes(*q->A, 1);
                        if (budget && need > budget) {  // can never fit: reject
                            q->status = UAAMG_ERR_BUDGET;
                            q->done = true;
                            n_rejected++;
                            rejected = true;
                            it = queue.erase(it);
                            continue;
                        }
                        if (!make_room(need)) {
                            if (taken == 0) wait_memory = true;
                            if (taken == 0) break;
                            ++it;
                            continue;
                        }
                        cache.push_front(CacheEntry{key, nullptr, need, 0, nullptr});
                        g.entry = &cache.front();
                        g.need_setup = true;
                    } else if (!reserve(g.entry, *q->A, 1)) {
                        if (taken == 0) wait_memory = true;
                        if (taken == 0) break;
                        ++it;
                        continue;
                    }
                    g.entry->users++;
                    f = gi.emplace(key, groups.size()).first;
                    groups.push_back(std::move(g));
                } else if (!reserve(groups[f->second].entry, *q->A,
                                    (int)groups[f->second].reqs.size() + 1)) {
                    ++it;  // no room for one more column of this matrix now
                    continue;
                }
                Group& g = groups[f->second];
                if (!g.need_setup) {
                    q->cache_hit = 1;
                    n_hits++;
                }
                g.reqs.push_back(q);
                q->queue_ms =
                    std::chrono::duration<double, std::milli>(Clock::now() - q->t_submit).count();
                tol = q->tol;
                taken++;
                it = queue.erase(it);
            }
            if (rejected) cv_done.notify_all();
            if (groups.empty()) {
                if (wait_memory) cv_done.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        // set up the matrices this batch brings (outside the lock)
        for (Group& g : groups) {
            if (!g.need_setup) continue;
            const Matrix& A = *g.reqs[0]->A;
            uaamg_csr csr{A.n, A.nnz, A.rowptr.data(), A.col.data(), A.val.data(), 0};
            uaamg_handle* h = nullptr;
            const auto t0 = Clock::now();
            g.status = uaamg_setup(&csr, &params, stream, &h);
            const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
            for (auto& q : g.reqs) q->setup_ms = ms;
            std::lock_guard<std::mutex> lk(mu);
            n_setups++;
            if (g.status != UAAMG_OK) {
                for (auto it = cache.begin(); it != cache.end(); ++it)
                    if (&*it == g.entry) {
                        cache.erase(it);
                        break;
                    }
                g.entry = nullptr;
            } else {
                g.entry->h = h;
            }
        }
        // the systems whose setup succeeded, solved together
        std::vector<Group*> live;
        for (Group& g : groups)
            if (g.status == UAAMG_OK) live.push_back(&g);
        const int ns = (int)live.size();
        std::vector<int32_t> nr(ns);
        std::vector<std::vector<double>> B(ns), X(ns);
        std::vector<int32_t> its;
        std::vector<double> rr;
        int st = UAAMG_OK;
        for (int s = 0; s < ns; s++) {
            const Group& g = *live[s];
            const int R = (int)g.reqs.size(), n = g.reqs[0]->A->n;
            nr[s] = R;
            B[s].resize((size_t)n * R);
            X[s].assign((size_t)n * R, 0.0);
            for (int r = 0; r < R; r++)
                for (int i = 0; i < n; i++) B[s][(size_t)i * R + r] = g.reqs[r]->b[i];
        }
        size_t ncol = 0;
        for (int s = 0; s < ns; s++) ncol += nr[s];
        its.assign(ncol, 0);
        rr.assign(ncol, 0.0);
        const double tol = taken ? groups[0].reqs[0]->tol : 1e-8;
        const auto t_solve = Clock::now();
        if (ns == 1 && nr[0] == 1) {
            st = uaamg_solve(live[0]->entry->h, B[0].data(), X[0].data(), tol, 0, &its[0], &rr[0]);
        } else if (ns == 1) {
            st = uaamg_solve_many(live[0]->entry->h, nr[0], B[0].data(), X[0].data(), tol,
                                  its.data(), rr.data());
        } else if (ns > 1) {
            std::vector<uaamg_handle*> hs(ns);
            std::vector<const double*> bp(ns);
            std::vector<double*> xp(ns);
            for (int s = 0; s < ns; s++) {
                hs[s] = live[s]->entry->h;
                bp[s] = B[s].data();
                xp[s] = X[s].data();
            }
            st = uaamg_solve_batch(hs.data(), ns, nr.data(), bp.data(), xp.data(), tol,
                                   its.data(), rr.data(), stream);
        }
        const auto t_end = Clock::now();
        const double solve_ms = std::chrono::duration<double, std::milli>(t_end - t_solve).count();
        std::lock_guard<std::mutex> lk(mu);
        size_t c = 0;
        for (int s = 0; s < ns; s++) {
            Group& g = *live[s];
            const int R = nr[s], n = g.reqs[0]->A->n;
            for (int r = 0; r < R; r++, c++) {
                Request& q = *g.reqs[r];
                q.x.resize(n);
                for (int i = 0; i < n; i++) q.x[i] = X[s][(size_t)i * R + r];
                q.status = (st == UAAMG_ERR_NO_CONVERGENCE) ? (rr[c] <= q.tol ? UAAMG_OK : st) : st;
                q.iters = its[c];
                q.relres = rr[c];
            }
        }
        for (Group& g : groups) {
            if (g.entry) {
                g.entry->users--;
                // from now on the entry counts what its handle holds (below the estimate)
                if (g.entry->h) g.entry->bytes = handle_bytes(g.entry->h);
            }
            for (auto& q : g.reqs) {
                q->solve_ms = solve_ms;
                if (g.status != UAAMG_OK) q->status = g.status;
                q->batch = taken;
                q->latency_ms =
                    std::chrono::duration<double, std::milli>(t_end - q->t_submit).count();
                q->done = true;
                q->A.reset();  // the host copies of an answered request are no longer needed
                std::vector<double>().swap(q->b);
            }
        }
        n_done += taken;
        n_batches++;
        cv_done.notify_all();
        cv_work.notify_all();  // matrices became free: queued requests for them can run
    }
    cudaStreamDestroy(stream);
}

extern "C" {

int uaamg_server_create(const uaamg_params* p, uint64_t budget_bytes, int32_t workers,
                        int32_t max_batch, uaamg_server** out) {
    if (!out || workers < 1 || workers > 64 || max_batch < 1 || max_batch > 32)
        return UAAMG_ERR_INVALID_ARG;
    *out = nullptr;
    uaamg_server* s = new uaamg_server();
    if (p) s->params = *p;
    else uaamg_default_params(&s->params);
    s->budget = budget_bytes;
    s->max_batch = max_batch;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return UAAMG_ERR_CUDA;
    }
    if (budget_bytes) add_budget(budget_bytes, +1);
    for (int w = 0; w < workers; w++) s->workers.emplace_back(&uaamg_server::worker_main, s, w);
    *out = s;
    return UAAMG_OK;
}

int uaamg_server_submit(uaamg_server* s, const uaamg_csr* A, uint64_t matrix_key,
                        const double* b, double tol, uint64_t* ticket) {
    if (!s || !A || !b || !ticket || A->on_device || A->n < 1 || A->nnz < A->n || !(tol >= 0.0))
        return UAAMG_ERR_INVALID_ARG;
    auto req = std::make_shared<Request>();
    req->t_submit = Clock::now();
    uint64_t key = matrix_key;
    if (!key) {
        key = 0xcbf29ce484222325ULL;
        key = fnv1a(&A->n, sizeof(A->n), key);
        key = fnv1a(A->rowptr, sizeof(int32_t) * ((size_t)A->n + 1), key);
        key = fnv1a(A->col, sizeof(int32_t) * (size_t)A->nnz, key);
        key = fnv1a(A->val, sizeof(double) * (size_t)A->nnz, key);
    }
    std::shared_ptr<Matrix> M;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& q : s->queue)
            if (q->A->key == key) M = q->A;
    }
    if (!M) {
        M = std::make_shared<Matrix>();
        M->key = key;
        M->n = A->n;
        M->nnz = A->nnz;
        M->rowptr.assign(A->rowptr, A->rowptr + A->n + 1);
        M->col.assign(A->col, A->col + A->nnz);
        M->val.assign(A->val, A->val + A->nnz);
    }
    req->A = M;
    req->b.assign(b, b + A->n);
    req->tol = tol;
    std::lock_guard<std::mutex> lk(s->mu);
    req->ticket = s->next_ticket++;
    *ticket = req->ticket;
    s->tickets[req->ticket] = req;
    s->queue.push_back(req);
    s->cv_work.notify_one();
    return UAAMG_OK;
}

int uaamg_server_poll(uaamg_server* s, uint64_t ticket, int32_t* done) {
    if (!s || !done) return UAAMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return UAAMG_ERR_INVALID_ARG;
    *done = it->second->done ? 1 : 0;
    return UAAMG_OK;
}

int uaamg_server_wait(uaamg_server* s, uint64_t ticket, double* x, int32_t* iters,
                      double* relres, double* latency_ms, int32_t* batch) {
    if (!s) return UAAMG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return UAAMG_ERR_INVALID_ARG;
    std::shared_ptr<Request> req = it->second;
    s->cv_done.wait(lk, [&] { return req->done; });
    if (x && !req->x.empty()) memcpy(x, req->x.data(), sizeof(double) * req->x.size());
    if (iters) *iters = req->iters;
    if (relres) *relres = req->relres;
    if (latency_ms) *latency_ms = req->latency_ms;
    if (batch) *batch = req->batch;
    s->tickets.erase(it);
    return req->status;
}

int uaamg_server_cancel(uaamg_server* s, uint64_t ticket, int32_t* cancelled) {
    if (!s || !cancelled) return UAAMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return UAAMG_ERR_INVALID_ARG;
    *cancelled = 0;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
        if ((*q)->ticket != ticket) continue;
        (*q)->status = UAAMG_ERR_CANCELLED;
        (*q)->done = true;
        s->queue.erase(q);
        s->n_cancelled++;
        *cancelled = 1;
        s->cv_done.notify_all();
        break;
    }
    return UAAMG_OK;
}

int uaamg_server_wait_answer(uaamg_server* s, uint64_t ticket, double* x, uaamg_answer* a) {
    if (!s) return UAAMG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return UAAMG_ERR_INVALID_ARG;
    std::shared_ptr<Request> req = it->second;
    s->cv_done.wait(lk, [&] { return req->done; });
    if (x && !req->x.empty()) memcpy(x, req->x.data(), sizeof(double) * req->x.size());
    if (a) {
        a->status = req->status;
        a->iters = req->iters;
        a->batch = req->batch;
        a->cache_hit = req->cache_hit;
        a->relres = req->relres;
        a->latency_ms = req->latency_ms;
        a->queue_ms = req->queue_ms;
        a->setup_ms = req->setup_ms;
        a->solve_ms = req->solve_ms;
    }
    s->tickets.erase(it);
    return req->status;
}

int uaamg_server_stats(uaamg_server* s, uint64_t* done, uint64_t* batches, uint64_t* cache_hits,
                       uint64_t* setups, uint64_t* rejected, int32_t* cached) {
    if (!s) return UAAMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (done) *done = s->n_done;
    if (batches) *batches = s->n_batches;
    if (cache_hits) *cache_hits = s->n_hits;
    if (setups) *setups = s->n_setups;
    if (rejected) *rejected = s->n_rejected;
    if (cached) *cached = (int32_t)s->cache.size();
    return UAAMG_OK;
}

void uaamg_server_destroy(uaamg_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& e : s->cache) {
        if (e.h) uaamg_free(e.h);
    }
    s->cache.clear();
    if (s->budget) add_budget(s->budget, -1);
    delete s;
}

}  // extern "C"
