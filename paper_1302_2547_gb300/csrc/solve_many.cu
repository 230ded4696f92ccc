// solve_many.cu -- uaamg_solve_many: R right-hand sides of one hierarchy at once.  Every
// column runs the same algorithm as uaamg_solve (K-cycle of Section 4.3 inside flexible CG)
// with its own scalars and its own convergence test; the kernels of kern_multi.cu read
// each level's matrix once per sweep for all columns.
#include <math.h>

#include "common.cuh"
#include "pinned.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kMaxRhs = 32;

template <typename T>
struct MPrec;
template <>
struct MPrec<float> {
    static const float* val(const Level& L) { return L.val32; }
    static const float* minv(const Level& L) { return L.minv32; }
};
template <>
struct MPrec<double> {
    static const double* val(const Level& L) { return L.val64; }
    static const double* minv(const Level& L) { return L.minv64; }
};

// Workspace of R interleaved columns on every level (kept by the handle; uaamg_solve_batch
// uses it too).
int ensure_multi(Handle* h, int R) {
    if (h->multi_R >= R) return UAAMG_OK;
    int st = UAAMG_OK;
    const size_t es = (h->p.precision == UAAMG_MIXED) ? sizeof(float) : sizeof(double);
    const int n0 = h->lev[0].n;
    if (h->mgraph) {  // its nodes name the buffers released below
        cudaGraphExecDestroy(h->mgraph);
        h->mgraph = nullptr;
        h->mgraph_R = 0;
    }
    if (h->multi_R > 0) {  // the narrower workspace goes (after the work queued on it)
        const int R0 = h->multi_R;
        for (int l = 0; l < h->nlev; l++) {
            MultiLevel& M = h->mlev[l];
            const size_t bytes = es * (size_t)h->lev[l].n * R0;
            void* vs[] = {M.rhs, M.out, M.w, M.s, M.c1, M.v1, M.rt, M.c2, M.v2};
            for (void* v : vs) dfree_one(h, v, bytes);
            dfree_one(h, M.sc, sizeof(double) * 7 * (size_t)R0);
        }
        double* os[] = {h->mb, h->mx, h->mr, h->mp, h->mq};
        for (double* v : os) dfree_one(h, v, sizeof(double) * (size_t)n0 * R0);
        dfree_one(h, h->mos, sizeof(double) * 8 * (size_t)R0);
        h->multi_R = 0;
    }
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        MultiLevel& M = h->mlev[l];
        const bool coarsest = (l == h->nlev - 1);
        const size_t bytes = es * (size_t)L.n * R;
        M = MultiLevel{};
        M.rhs = dalloc_bytes(h, bytes, &st);
        M.out = dalloc_bytes(h, bytes, &st);
        if (!coarsest) {
            M.w = dalloc_bytes(h, bytes, &st);
            M.s = dalloc_bytes(h, bytes, &st);
        }
        if (l >= 1 && !coarsest) {
            M.c1 = dalloc_bytes(h, bytes, &st);
            M.v1 = dalloc_bytes(h, bytes, &st);
            M.rt = dalloc_bytes(h, bytes, &st);
            M.c2 = dalloc_bytes(h, bytes, &st);
            M.v2 = dalloc_bytes(h, bytes, &st);
        }
        M.sc = dalloc<double>(h, 7 * (size_t)R, &st);
    }
    h->mb = dalloc<double>(h, (size_t)n0 * R, &st);
    h->mx = dalloc<double>(h, (size_t)n0 * R, &st);
    h->mr = dalloc<double>(h, (size_t)n0 * R, &st);
    h->mp = dalloc<double>(h, (size_t)n0 * R, &st);
    h->mq = dalloc<double>(h, (size_t)n0 * R, &st);
    h->mos = dalloc<double>(h, 8 * (size_t)R, &st);
    const size_t pneed = (size_t)16 * h->num_sms * 3 * kMaxRhs;
    if (st == UAAMG_OK && h->partials_cap < pneed) {  // the old buffer stays valid for its graph
        h->partials = dalloc<double>(h, pneed, &st);
        h->partials_cap = pneed;
    }
    if (st) return st;
    if (h->mos_host) {
        cudaStreamSynchronize(h->work);
        pinned_put(h->mos_host);
        h->mos_host = nullptr;
    }
    h->mos_host = static_cast<double*>(pinned_get(sizeof(double) * 8 * R));
    if (!h->mos_host) return UAAMG_ERR_OOM;
    h->multi_R = R;
    return UAAMG_OK;
}

template <typename T>
static MArgs<T> margs(Handle* h, const Level& L, int R) {
    MArgs<T> a{};
    a.n = L.n;
    a.R = R;
    a.rowptr = L.rowptr;
    a.col = L.col;
    a.val = MPrec<T>::val(L);
    a.minv = MPrec<T>::minv(L);
    a.partials = h->partials;
    a.counter = &h->ctrl->red_count;
    return a;
}

template <typename T>
static int mK(Handle* h, int R, int m, const T* in, T* out);

// out = B_l(in): one pre-sweep from zero, restriction, K_{l+1}, prolongation + post-sweep
template <typename T>
static int mB(Handle* h, int R, int l, const T* in, T* out) {
    if (l == h->nlev - 1) return launch_mdense<T>(h, h->nco, R, h->coarse_inv, in, out);
    Level& L = h->lev[l];
    MultiLevel& M = h->mlev[l];
    MultiLevel& C = h->mlev[l + 1];
    int st;
    MArgs<T> a = margs<T>(h, L, R);
    a.r = in;
    a.y = (T*)M.w;
    a.y2 = (T*)M.s;
    if ((st = launch_mrow<T>(h, RB_PRE1, 0, a))) return st;
    if ((st = launch_mrestrict<T>(h, L.nc, R, L.aggptr, L.members, (const T*)M.s, (T*)C.rhs)))
        return st;
    if ((st = mK<T>(h, R, l + 1, (const T*)C.rhs, (T*)C.out))) return st;
    MArgs<T> b = margs<T>(h, L, R);
    b.r = in;
    b.x = (const T*)M.w;
    b.agg = L.agg;
    b.e = (const T*)C.out;
    b.y = out;
    return launch_mrow<T>(h, RB_PROSMOOTH, 0, b);
}

template <typename T>
static int mK(Handle* h, int R, int m, const T* in, T* out) {
    if (m == h->nlev - 1) return launch_mdense<T>(h, h->nco, R, h->coarse_inv, in, out);
    Level& L = h->lev[m];
    MultiLevel& M = h->mlev[m];
    T *c1 = (T*)M.c1, *v1 = (T*)M.v1, *rt = (T*)M.rt, *c2 = (T*)M.c2, *v2 = (T*)M.v2;
    int st;
    if ((st = mB<T>(h, R, m, in, c1))) return st;
    MArgs<T> a = margs<T>(h, L, R);
    a.x = c1;
    a.y = v1;
    a.d1 = in;
    a.result = M.sc;  // rho1 (row 0), alpha1 (row 1)
    if ((st = launch_mrow<T>(h, RB_SPMV, 2, a))) return st;
    int inner = h->p.kcycle_inner;
    if (inner == 2 && h->p.kcycle_ratio > 0.0 &&
        (double)h->lev[m - 1].n < h->p.kcycle_ratio * (double)L.n)
        inner = 1;
    if (inner >= 2) {
        const bool tau = h->p.kcycle_tau > 0.0;
        if ((st = launch_mkc_rt<T>(h, L.n, R, in, v1, rt, M.sc, tau))) return st;
        if ((st = mB<T>(h, R, m, rt, c2))) return st;
        MArgs<T> b = margs<T>(h, L, R);
        b.x = c2;
        b.y = v2;
        b.d1 = v1;
        b.d2 = rt;
        b.result = M.sc + 2 * R;  // beta, gamma, alpha2
        if ((st = launch_mrow<T>(h, RB_SPMV, 3, b))) return st;
    }
    return launch_mkc_combine<T>(h, L.n, R, c1, c2, out, M.sc, inner >= 2, h->p.kcycle_tau);
}

template <typename T>
static int m_iteration(Handle* h, int R) {
    Level& L0 = h->lev[0];
    const int n = L0.n;
    MultiLevel& M0 = h->mlev[0];
    int st;
    const T* rin;
    if constexpr (sizeof(T) == 4) {
        if ((st = launch_mcast(h, (long long)n * R, h->mr, (float*)M0.rhs))) return st;
        rin = (const T*)M0.rhs;
    } else {
        rin = (const T*)h->mr;
    }
    T* z = (T*)M0.out;
    if ((st = mB<T>(h, R, 0, rin, z))) return st;
    if ((st = launch_mouter<T>(h, n, R, z, h->mp, h->mq, h->mos))) return st;
    MArgs<double> a{};
    a.n = n;
    a.R = R;
    a.rowptr = L0.rowptr;
    a.col = L0.col;
    a.val = L0.val64;
    a.x = h->mp;
    a.y = h->mq;
    a.d1 = h->mr;
    a.partials = h->partials;
    a.counter = &h->ctrl->red_count;
    a.result = h->mos;  // pq (row 0), pr (row 1)
    if ((st = launch_mrow<double>(h, RB_SPMV, 2, a))) return st;
    if ((st = launch_mxr(h, n, R, h->mx, h->mr, h->mp, h->mq, h->mos))) return st;
    return check_cuda(cudaMemcpyAsync(h->mos_host, h->mos, sizeof(double) * 8 * R,
                                      cudaMemcpyDeviceToHost, h->work));
}

static int m_run(Handle* h, int R) {
    if (h->p.precision == UAAMG_MIXED) return m_iteration<float>(h, R);
    return m_iteration<double>(h, R);
}

static int m_true_residual(Handle* h, int R) {
    Level& L0 = h->lev[0];
    MArgs<double> a{};
    a.n = L0.n;
    a.R = R;
    a.rowptr = L0.rowptr;
    a.col = L0.col;
    a.val = L0.val64;
    a.x = h->mx;
    a.r = h->mb;
    a.y = h->mr;
    a.partials = h->partials;
    a.counter = &h->ctrl->red_count;
    a.result = h->mos + 3 * R;  // rr
    int st = launch_mrow<double>(h, RB_RESID, 1, a);
    if (st == UAAMG_OK)
        st = check_cuda(cudaMemcpyAsync(h->mos_host, h->mos, sizeof(double) * 8 * R,
                                        cudaMemcpyDeviceToHost, h->work));
    if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
    return st;
}

int solve_many(Handle* h, int R, const double* B, double* X, double tol, int* iters,
               double* relres) {
    if (R < 1 || R > kMaxRhs || h->p.pre != 1 || h->p.post != 1) return UAAMG_ERR_UNSUPPORTED;
    int st = ensure_multi(h, R);
    if (st) return st;
    const int n = h->lev[0].n;
    const size_t bytes = sizeof(double) * (size_t)n * R;
    cudaEventRecord(h->ev_t0, h->work);
    if ((st = check_cuda(cudaMemcpyAsync(h->mb, B, bytes, cudaMemcpyDefault, h->work)))) return st;
    cudaMemsetAsync(h->mx, 0, bytes, h->work);
    cudaMemsetAsync(h->mp, 0, bytes, h->work);
    cudaMemsetAsync(h->mq, 0, bytes, h->work);
    double* os = h->mos_host;
    for (int r = 0; r < R; r++) {
        for (int k = 0; k < 8; k++) os[k * R + r] = 0.0;
        os[6 * R + r] = 1.0;  // active
        os[7 * R + r] = 1.0;  // first direction
    }
    cudaMemcpyAsync(h->mos, os, sizeof(double) * 8 * R, cudaMemcpyHostToDevice, h->work);
    if ((st = launch_mnorm(h, n, R, h->mb, h->mos + 4 * R))) return st;
    if ((st = m_true_residual(h, R))) return st;  // r = b, rr
    std::vector<double> bn(R), rn(R);
    std::vector<int> active(R, 1);
    int nactive = R;
    for (int r = 0; r < R; r++) {
        iters[r] = 0;
        bn[r] = sqrt(os[4 * R + r]);
        rn[r] = sqrt(os[3 * R + r]);
        if (bn[r] == 0.0) bn[r] = 1.0;
        if (rn[r] <= tol * bn[r]) {
            active[r] = 0;
            nactive--;
        }
    }
    auto push_active = [&]() {
        for (int r = 0; r < R; r++) os[6 * R + r] = active[r] ? 1.0 : 0.0;
        return check_cuda(cudaMemcpyAsync(h->mos + 6 * R, os + 6 * R, sizeof(double) * R,
                                          cudaMemcpyHostToDevice, h->work));
    };
    if ((st = push_active())) return st;
    if (nactive > 0 && h->p.use_graphs && (!h->mgraph || h->mgraph_R != R)) {
        if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
        h->mgraph = nullptr;
        cudaGraph_t g = nullptr;
        h->capturing = true;
        long long nodes0 = h->graph_nodes;
        st = check_cuda(cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal));
        if (st == UAAMG_OK) {
            int st2 = m_run(h, R);
            st = check_cuda(cudaStreamEndCapture(h->work, &g));
            if (st2) st = st2;
        }
        h->capturing = false;
        h->mgraph_nodes = h->graph_nodes - nodes0;
        h->graph_nodes = nodes0;
        if (st == UAAMG_OK) st = check_cuda(cudaGraphInstantiate(&h->mgraph, g, 0));
        if (g) cudaGraphDestroy(g);
        if (st) return st;
        h->mgraph_R = R;
    }
    int k = 0;
    while (nactive > 0 && k < h->p.max_iter) {
        if (h->mgraph) {
            st = check_cuda(cudaGraphLaunch(h->mgraph, h->work));
            count_launch(h, h->mgraph_nodes);
        } else {
            st = m_run(h, R);
        }
        if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
        if (st) return st;
        k++;
        bool check = false;
        for (int r = 0; r < R; r++) {
            if (!active[r]) continue;
            iters[r] = k;
            rn[r] = sqrt(os[3 * R + r]);
            if (rn[r] <= tol * bn[r]) check = true;
        }
        if (check) {  // confirm with the recomputed residual b - A x (all columns)
            if ((st = m_true_residual(h, R))) return st;
            bool changed = false;
            for (int r = 0; r < R; r++) {
                if (!active[r]) continue;
                rn[r] = sqrt(os[3 * R + r]);
                if (rn[r] <= tol * bn[r]) {
                    active[r] = 0;
                    nactive--;
                    changed = true;
                }
            }
            if (changed && (st = push_active())) return st;
        }
    }
    // final residuals of every column from the true residual
    if ((st = m_true_residual(h, R))) return st;
    int status = UAAMG_OK;
    for (int r = 0; r < R; r++) {
        relres[r] = sqrt(os[3 * R + r]) / bn[r];
        if (!(relres[r] <= tol)) status = UAAMG_ERR_NO_CONVERGENCE;
    }
    if ((st = check_cuda(cudaMemcpyAsync(X, h->mx, bytes, cudaMemcpyDefault, h->work)))) return st;
    cudaEventRecord(h->ev_t1, h->work);
    if ((st = check_cuda(cudaStreamSynchronize(h->work)))) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
    h->solve_ms = ms;
    return status;
}

}  // namespace uaamg
