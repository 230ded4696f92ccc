// tune.cu -- the kernel autotuner: per level, the SpMV kernel family and the rows per
// block of the solve's fused sweeps (Sections 4.1, 4.4), chosen by timing.
//
// For every level of at least kTuneMinRows unknowns (except the coarsest), the kernels a
// visit of the level launches (the first l1-Jacobi sweep, the prolongation sweep, the SpMV
// with two inner products, and on level 0 the outer FP64 SpMV) are timed together with CUDA
// events on the handle's stream for each candidate: the row-block CSR kernel with 256,
// 128, 64 and 32 rows per block, the per-warp TMA-staged kernel, and the sliced ELLPACK
// kernel (Section 4.4: ELL suits uniform row lengths; its copy is built for the timing and
// kept only when it wins).  The fastest is kept for every SpMV-based kernel of that level
// in both precisions.  Every candidate computes the same arithmetic per entry (the TMA and
// ELLPACK kernels give the row-block kernel's one-thread-per-row bits; the lanes a row-block
// row is split into change only the rounding of the row sums).  Choices are remembered per
// matrix shape (n, nnz, precision) for the process, so repeated setups of one shape are
// not timed again.
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kTuneMinRows = 32768;  // smaller levels are latency-bound: thresholds decide
constexpr int kTuneReps = 5;

namespace {
struct TuneChoice {
    int path, rows;
    float us[6];
};
std::mutex g_tune_mu;
std::map<std::tuple<int, long long, int>, TuneChoice> g_tune;
}  // namespace

// The arguments of a level's SpMV-based kernels in precision U for kernel family `path`.
template <typename U>
static RBArgs<U> tune_args(Handle* h, Level& L, int path, int rows) {
    RBArgs<U> a{};
    a.path = path;
    a.n = L.n;
    a.nnz = L.nnz;
    a.rows = rows;
    a.rowptr = L.rowptr;
    a.col = L.col;
    if constexpr (sizeof(U) == 4) {
        a.val = L.val32;
        a.minv = L.minv32;
        if (path == 2) a.sval = L.sl_val32;
    } else {
        a.val = L.val64;
        a.minv = L.minv64;
        if (path == 2) a.sval = L.sl_val64;
    }
    if (path == 2) {
        a.sptr = L.sl_ptr;
        a.scol = L.sl_col;
        a.slen = L.sl_len;
        a.nslices = L.sl_ns;
    }
    a.partials = h->partials;
    a.counter = &h->ctrl->red_count;
    return a;
}

// One round of the level's kernels per visit of the cycle: the first sweep, the prolongation
// sweep and the SpMV with two inner products (in the cycle's precision T); on level 0 also
// the outer FP64 SpMV with its two inner products.
template <typename T>
static int run_level(Handle* h, int l, int path, int rows) {
    Level& L = h->lev[l];
    Level& C = h->lev[l + 1];
    RBArgs<T> a = tune_args<T>(h, L, path, rows);
    a.r = (const T*)L.rhs;
    a.y = (T*)L.w;
    a.y2 = (T*)L.s;
    int st = launch_rowblock<T>(h, RB_PRE1, 0, a);
    RBArgs<T> b = tune_args<T>(h, L, path, rows);
    b.r = (const T*)L.rhs;
    b.x = (const T*)L.w;
    b.agg = L.agg;
    b.e = (const T*)C.out;
    b.y = (T*)L.out;
    if (st == UAAMG_OK) st = launch_rowblock<T>(h, RB_PROSMOOTH, 0, b);
    RBArgs<T> c = tune_args<T>(h, L, path, rows);
    c.x = (const T*)L.out;
    c.y = (T*)L.s;
    c.d1 = (const T*)L.rhs;
    c.result = &L.sc->rho1;
    if (st == UAAMG_OK) st = launch_rowblock<T>(h, RB_SPMV, 2, c);
    if (l == 0 && st == UAAMG_OK) {
        RBArgs<double> d = tune_args<double>(h, L, path, rows);
        d.x = h->p_;
        d.y = h->q;
        d.d1 = h->r;
        d.result = &h->osc->pq;
        st = launch_rowblock<double>(h, RB_SPMV, 2, d);
    }
    return st;
}

template <typename T>
static int time_level(Handle* h, int l, int path, int rows, float* us) {
    Level& L = h->lev[l];
    L.path = path;
    L.rb_rows = rows;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = check_cuda(cudaEventCreate(&e0));
    if (st == UAAMG_OK) st = check_cuda(cudaEventCreate(&e1));
    for (int k = 0; k < 2 && st == UAAMG_OK; k++) st = run_level<T>(h, l, path, rows);
    if (st == UAAMG_OK) cudaEventRecord(e0, h->work);
    for (int k = 0; k < kTuneReps && st == UAAMG_OK; k++) st = run_level<T>(h, l, path, rows);
    if (st == UAAMG_OK) cudaEventRecord(e1, h->work);
    if (st == UAAMG_OK) st = check_cuda(cudaEventSynchronize(e1));
    float ms = 0.f;
    if (st == UAAMG_OK) st = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *us = 1000.f * ms / kTuneReps;
    return st;
}

template <typename T>
static int tune_level(Handle* h, int l, bool mixed) {
    Level& L = h->lev[l];
    const size_t es = sizeof(T);
    // finite operands for the timed kernels (the solve overwrites all of them)
    void* zero[] = {L.rhs, L.out, L.w, L.s, h->lev[l + 1].out};
    const size_t len[] = {es * L.n, es * L.n, es * L.n, es * L.n, es * h->lev[l + 1].n};
    int st = UAAMG_OK;
    for (int k = 0; k < 5 && st == UAAMG_OK; k++)
        if (zero[k]) st = check_cuda(cudaMemsetAsync(zero[k], 0, len[k], h->work));
    if (st == UAAMG_OK && l == 0) {
        const size_t b8 = sizeof(double) * L.n;
        st = check_cuda(cudaMemsetAsync(h->p_, 0, b8, h->work));
        if (st == UAAMG_OK) st = check_cuda(cudaMemsetAsync(h->q, 0, b8, h->work));
        if (st == UAAMG_OK) st = check_cuda(cudaMemsetAsync(h->r, 0, b8, h->work));
    }
    if (st) return st;
    const bool had_sell = L.sl_ptr != nullptr;
    if (st == UAAMG_OK && !had_sell) st = build_sell(h, L, mixed);  // kept only if it wins
    if (st) return st;
    static const int rows[4] = {256, 128, 64, 32};
    int best_path = 0, best_rows = L.rb_rows;
    float best = 1e30f;
    for (int c = 0; c < 6 && st == UAAMG_OK; c++) {
        float us = -1.f;
        if (c < 4) st = time_level<T>(h, l, 0, rows[c], &us);
        else if (c == 4) st = time_level<T>(h, l, 1, kRowsPerBlock, &us);
        else if (L.sl_ptr) st = time_level<T>(h, l, 2, kRowsPerBlock, &us);
        L.tune_us[c] = us;
        if (us >= 0.f && us < best) {
            best = us;
            best_path = c < 4 ? 0 : (c == 4 ? 1 : 2);
            best_rows = c < 4 ? rows[c] : kRowsPerBlock;
        }
    }
    if (st) return st;
    L.path = best_path;
    L.rb_rows = best_rows;
    if (best_path != 2 && !had_sell) drop_sell(h, L);
    return UAAMG_OK;
}

int autotune_levels(Handle* h) {
    const bool mixed = h->p.precision == UAAMG_MIXED;
    int st = UAAMG_OK;
    for (int l = 0; l < h->nlev - 1 && st == UAAMG_OK; l++) {
        Level& L = h->lev[l];
        if (L.n < kTuneMinRows) continue;
        const auto key = std::make_tuple(L.n, L.nnz, mixed ? 1 : 0);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                L.path = it->second.path;
                L.rb_rows = it->second.rows;
                for (int c = 0; c < 6; c++) L.tune_us[c] = it->second.us[c];
                if (L.path == 2 && !L.sl_ptr) st = build_sell(h, L, mixed);
                if (st == UAAMG_OK && L.path == 2 && !L.sl_ptr) L.path = -1;  // not buildable
                continue;
            }
        }
        st = mixed ? tune_level<float>(h, l, mixed) : tune_level<double>(h, l, mixed);
        if (st == UAAMG_OK) {
            TuneChoice c{L.path, L.rb_rows, {}};
            for (int k = 0; k < 6; k++) c.us[k] = L.tune_us[k];
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = c;
        }
    }
    return st;
}

}  // namespace uaamg
