// api.cu -- the extern "C" boundary declared in include/uaamg.h.  Argument checking,
// device/stream bookkeeping and host copies only; every compute step is a kernel launched
// from setup.cu / solve.cu.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "pinned.cuh"
#include "kernels.cuh"

namespace uaamg {
int build_hierarchy(Handle* h, const uaamg_csr* A);
int solve(Handle* h, const double* b, double* x, double tol, int use_guess, int* iters,
          double* relres);
int apply_operator(Handle* h, int which, int l, const double* in, double* out);
int solve_many(Handle* h, int R, const double* B, double* X, double tol, int* iters,
               double* relres);
double profile_bytes(const Handle* h);

// Makes the handle's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Orders the handle's work after the caller's stream and the caller's stream after it.
static void enter(Handle* h) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->work, h->ev_in, 0);
}
static void leave(Handle* h) {
    cudaEventRecord(h->ev_out, h->work);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
}

static void destroy(Handle* h) {
    if (!h) return;
    if (h->work) cudaStreamSynchronize(h->work);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->loop_graph) cudaGraphExecDestroy(h->loop_graph);
    if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
    pinned_put(h->mos_host);
    for (auto& ps : h->prof_slots) {
        cudaEventDestroy(ps.a);
        cudaEventDestroy(ps.b);
    }
    if (h->work) {
        dfree_all(h);
        cudaStreamSynchronize(h->work);
        cudaStreamDestroy(h->work);
    }
    pinned_put(h->osc_host);
    cudaEvent_t evs[] = {h->ev_in, h->ev_out, h->ev_t0, h->ev_t1};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete h;
}

static bool params_ok(const uaamg_params* p) {
    return p->coarse_size >= 1 && p->max_levels >= 1 && p->max_levels <= kMaxLevels &&
           (p->max_agg_size == 0 || p->max_agg_size >= 2) &&
           (p->pass_mode == UAAMG_PASS_SINGLE_ROUND || p->pass_mode == UAAMG_PASS_MAXIMAL) &&
           p->pre >= 0 && p->pre <= 8 && p->post >= 0 && p->post <= 8 &&
           (p->kcycle_inner == 1 || p->kcycle_inner == 2) && p->kcycle_tau >= 0.0 &&
           (p->precision == UAAMG_FP64 || p->precision == UAAMG_MIXED) && p->max_iter >= 0 &&
           p->profile_class >= 0 && p->profile_class <= UAAMG_KCLASS_SRA &&
           (p->agg_repeat == 1 || p->agg_repeat == 2) && p->kcycle_ratio >= 0.0 &&
           p->min_coarsening >= 0.0 && p->fuse_below >= 0 && p->jacobi_omega >= 0.0 &&
           p->tma_rows >= 0 && p->sell_rows >= 0 && p->sra_rounds >= 0 && p->sra_rounds <= 64 &&
           p->wait_limit_ns >= 0 && p->cluster_below >= 0 && p->restrict_fuse_below >= 0 &&
           (p->autotune == 0 || p->autotune == 1);
}

}  // namespace uaamg

using namespace uaamg;

extern "C" {

void uaamg_default_params(uaamg_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->coarse_size = 64;
    p->max_levels = 25;
    p->max_agg_size = 5;
    p->pass_mode = UAAMG_PASS_SINGLE_ROUND;
    p->seed = 0x5EED;
    p->pre = 1;
    p->post = 1;
    p->kcycle_inner = 2;
    p->kcycle_tau = 0.0;
    p->precision = UAAMG_MIXED;
    p->max_iter = 200;
    p->use_graphs = 1;
    p->profile_class = 0;
    p->agg_repeat = 1;
    p->kcycle_ratio = 0.0;
    p->min_coarsening = 0.0;
    p->jacobi_omega = 0.0;
    p->tma_rows = 131072;
    p->sell_rows = 0;
    p->fuse_below = 0;
    p->sra_rounds = 0;
    p->restrict_fuse_below = 0;
    p->autotune = 0;
    p->cluster_below = 8192;
    p->wait_limit_ns = 0;
}

int uaamg_setup(const uaamg_csr* A, const uaamg_params* p, void* stream, uaamg_handle** out) {
    if (!out) return UAAMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!A || !A->rowptr || !A->col || !A->val || A->n < 1 || A->nnz < A->n)
        return UAAMG_ERR_INVALID_ARG;
    uaamg_params prm;
    if (p) prm = *p;
    else uaamg_default_params(&prm);
    if (!params_ok(&prm)) return UAAMG_ERR_INVALID_ARG;
    Handle* h = new Handle();
    h->p = prm;
    h->prof_class = prm.profile_class;
    h->user = (cudaStream_t)stream;
    int st = check_cuda(cudaGetDevice(&h->device));
    if (st == UAAMG_OK)
        st = check_cuda(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    if (st == UAAMG_OK) st = check_cuda(cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking));
    if (st == UAAMG_OK) st = check_cuda(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    if (st == UAAMG_OK) st = check_cuda(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    if (st == UAAMG_OK) st = check_cuda(cudaEventCreate(&h->ev_t0));
    if (st == UAAMG_OK) st = check_cuda(cudaEventCreate(&h->ev_t1));
    if (st != UAAMG_OK) {
        cudaGetLastError();
        destroy(h);
        return st;
    }
    enter(h);
    cudaEventRecord(h->ev_t0, h->work);
    st = build_hierarchy(h, A);
    cudaEventRecord(h->ev_t1, h->work);
    int st2 = check_cuda(cudaStreamSynchronize(h->work));
    if (st == UAAMG_OK) st = st2;
    if (st == UAAMG_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
        h->setup_ms = ms;
        for (auto& ps : h->prof_slots) {  // setup-phase kernel timings
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ps.a, ps.b) == cudaSuccess) {
                h->prof_ms += t;
                h->prof_launches++;
            }
            cudaEventDestroy(ps.a);
            cudaEventDestroy(ps.b);
        }
        h->prof_slots.clear();
    }
    if (st != UAAMG_OK) {
        cudaGetLastError();
        destroy(h);
        return st;
    }
    leave(h);
    *out = reinterpret_cast<uaamg_handle*>(h);
    return UAAMG_OK;
}

int uaamg_solve(uaamg_handle* hh, const double* b, double* x, double tol, int32_t use_guess,
                int32_t* iters, double* relres) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !b || !x || !iters || !relres || !(tol >= 0.0)) return UAAMG_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return UAAMG_ERR_CUDA;
    enter(h);
    int it = 0;
    double rr = 0.0;
    int st = solve(h, b, x, tol, use_guess, &it, &rr);
    *iters = it;
    *relres = rr;
    leave(h);
    return st;
}

int uaamg_solve_many(uaamg_handle* hh, int32_t nrhs, const double* B, double* X, double tol,
                     int32_t* iters, double* relres) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !B || !X || !iters || !relres || nrhs < 1 || !(tol >= 0.0))
        return UAAMG_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return UAAMG_ERR_CUDA;
    enter(h);
    std::vector<int> it(nrhs, 0);
    std::vector<double> rr(nrhs, 0.0);
    int st = solve_many(h, nrhs, B, X, tol, it.data(), rr.data());
    for (int r = 0; r < nrhs; r++) {
        iters[r] = it[r];
        relres[r] = rr[r];
    }
    leave(h);
    return st;
}

void uaamg_free(uaamg_handle* hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return;
    DeviceGuard g(h->device);
    destroy(h);
}

int uaamg_num_levels(const uaamg_handle* hh, int32_t* nlev) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !nlev) return UAAMG_ERR_INVALID_ARG;
    *nlev = h->nlev;
    return UAAMG_OK;
}

int uaamg_level_info(const uaamg_handle* hh, int32_t l, int32_t* n, int32_t* nnz,
                     int32_t* passes) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || l < 0 || l >= h->nlev) return UAAMG_ERR_INVALID_ARG;
    if (n) *n = h->lev[l].n;
    if (nnz) *nnz = (int32_t)h->lev[l].nnz;
    if (passes) *passes = h->lev[l].passes;
    return UAAMG_OK;
}

static int copy_out(const Handle* h, void* dst, const void* src, size_t bytes) {
    if (!src) return UAAMG_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return UAAMG_ERR_CUDA;
    int st = check_cuda(cudaStreamSynchronize(h->work));
    if (st == UAAMG_OK) st = check_cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return st;
}

int uaamg_get_aggregates(const uaamg_handle* hh, int32_t l, int32_t* agg) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !agg || l < 0 || l >= h->nlev - 1) return UAAMG_ERR_INVALID_ARG;
    return copy_out(h, agg, h->lev[l].agg, sizeof(int) * h->lev[l].n);
}

int uaamg_get_level_csr(const uaamg_handle* hh, int32_t l, int32_t* rowptr, int32_t* col,
                        double* val) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || l < 0 || l >= h->nlev || !rowptr || !col || !val) return UAAMG_ERR_INVALID_ARG;
    const Level& L = h->lev[l];
    int st = copy_out(h, rowptr, L.rowptr, sizeof(int) * (L.n + 1));
    if (st == UAAMG_OK) st = copy_out(h, col, L.col, sizeof(int) * L.nnz);
    if (st == UAAMG_OK) st = copy_out(h, val, L.val64, sizeof(double) * L.nnz);
    return st;
}

int uaamg_get_priorities(const uaamg_handle* hh, int32_t l, uint64_t* P) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !P || l < 0 || l >= h->nlev - 1) return UAAMG_ERR_INVALID_ARG;
    return copy_out(h, P, h->lev[l].prio, sizeof(uint64_t) * h->lev[l].n);
}

int uaamg_get_pass_of(const uaamg_handle* hh, int32_t l, int32_t* pass_of) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !pass_of || l < 0 || l >= h->nlev - 1) return UAAMG_ERR_INVALID_ARG;
    return copy_out(h, pass_of, h->lev[l].pass_of, sizeof(int) * h->lev[l].n);
}

int uaamg_level_kernel(const uaamg_handle* hh, int32_t l, int32_t* path, int32_t* rows,
                       double* us) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || l < 0 || l >= h->nlev) return UAAMG_ERR_INVALID_ARG;
    const Level& L = h->lev[l];
    int pth = L.path;
    if (pth < 0)  // by the size thresholds, as launch_rowblock decides
        pth = L.sl_ptr ? 2 : (h->p.tma_rows > 0 && L.n >= h->p.tma_rows ? 1 : 0);
    if (path) *path = pth;
    if (rows) *rows = L.rb_rows;
    if (us)
        for (int c = 0; c < 6; c++) us[c] = L.tune_us[c];
    return UAAMG_OK;
}

int uaamg_get_minv(const uaamg_handle* hh, int32_t l, double* minv) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !minv || l < 0 || l >= h->nlev) return UAAMG_ERR_INVALID_ARG;
    return copy_out(h, minv, h->lev[l].minv64, sizeof(double) * h->lev[l].n);
}

int uaamg_apply_B(uaamg_handle* hh, int32_t l, const double* in, double* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !in || !out || l < 0 || l >= h->nlev) return UAAMG_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return UAAMG_ERR_CUDA;
    return apply_operator(h, 0, l, in, out);
}

int uaamg_apply_K(uaamg_handle* hh, int32_t m, const double* in, double* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !in || !out || m < 1 || m >= h->nlev) return UAAMG_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return UAAMG_ERR_CUDA;
    return apply_operator(h, 1, m, in, out);
}

int uaamg_residual_history(const uaamg_handle* hh, double* hist, int32_t cap, int32_t* count) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !count || cap < 0 || (cap > 0 && !hist)) return UAAMG_ERR_INVALID_ARG;
    int k = (int)h->hist.size();
    if (k > cap) k = cap;
    for (int i = 0; i < k; i++) hist[i] = h->hist[i];
    *count = k;
    return UAAMG_OK;
}

int uaamg_get_stats(const uaamg_handle* hh, uaamg_stats* s) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !s) return UAAMG_ERR_INVALID_ARG;
    s->setup_ms = h->setup_ms;
    s->solve_ms = h->solve_ms;
    s->launches = h->launches;
    s->graph_nodes = h->loop_graph ? h->loop_nodes : h->graph_nodes;
    double z = 0, nn = 0;
    for (int l = 0; l < h->nlev; l++) {
        z += (double)h->lev[l].nnz;
        nn += h->lev[l].n;
    }
    s->opc = z / (double)h->lev[0].nnz;
    s->grid_complexity = nn / (double)h->lev[0].n;
    s->device_bytes = (uint64_t)h->bytes;
    s->tail_level = h->tail_level;
    s->tail_blocks = h->tail_level > 0 ? (h->tail_cluster ? h->tail_cl : 1) : 0;
    return UAAMG_OK;
}

int uaamg_set_profiling(uaamg_handle* hh, int32_t kclass) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || kclass < 0 || kclass > UAAMG_KCLASS_SRA) return UAAMG_ERR_INVALID_ARG;
    h->prof_class = kclass;
    h->prof_launches = 0;
    h->prof_ms = 0.0;
    return UAAMG_OK;
}

int uaamg_get_profile(const uaamg_handle* hh, int64_t* launches, double* total_ms,
                      double* bytes_per_launch) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h) return UAAMG_ERR_INVALID_ARG;
    if (launches) *launches = h->prof_launches;
    if (total_ms) *total_ms = h->prof_ms;
    if (bytes_per_launch) *bytes_per_launch = profile_bytes(h);
    return UAAMG_OK;
}

}  // extern "C"
