// solve_batch.cu -- uaamg_solve_batch and uaamg_setup_batch: many systems, each with its own
// hierarchy, solved together level step by level step.
//
// The K-cycle (Section 4.3) of every system is the same recursion over its own levels;
// systems differ in depth and in the levels that take one flexible-CG step instead of two.
// The host walks the union of the systems' recursions once and emits, at every node, one
// launch per step for the systems that take that step there (a system whose coarsest level
// the node reaches takes the exact solve instead).  The emitted launches form the plan of
// one outer iteration, which is captured once as a CUDA graph and replayed; per-column
// convergence is tested on the host after each replay, as in uaamg_solve_many.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "batch.cuh"
#include "pinned.cuh"
#include "kernels.cuh"

namespace uaamg {

int ensure_multi(Handle* h, int R);

namespace {

struct Rec {
    int kind, mode, ndots, level;
    int s_r, s_x, s_y, s_y2, s_d1, s_d2, s_e;
    int res_os, res_row, outer;
    bool dbl;    // FP64 kernel whatever the cycle's precision
    long long off;  // offset of the launch's per-block table in the table buffer (int4s)
    int nseg, tiles;
};

Rec rec(int kind, int level) {
    Rec r;
    memset(&r, 0, sizeof(r));
    r.kind = kind;
    r.level = level;
    r.s_r = r.s_x = r.s_y = r.s_y2 = r.s_d1 = r.s_d2 = r.s_e = -1;
    return r;
}

struct Plan {
    const std::vector<BLevel>* lev = nullptr;  // [nsys][kMaxLevels]
    std::vector<int> nlev;
    std::vector<int4> tab;  // per launch, per block: system, tile, tiles, first tile
    std::vector<Rec> recs;
    long long max_part = 0;  // doubles of partial sums the widest launch needs

    const BLevel& L(int s, int l) const { return (*lev)[(size_t)s * kMaxLevels + l]; }

    int tiles_of(const Rec& r, int s) const {
        const BLevel& B = L(s, r.level);
        if (r.kind == BK_DENSE) return B.n;
        if (r.kind == BK_RESTRICT) return b_tiles(B.nc, B.R);
        return b_tiles(B.n, B.R);
    }

    // Appends the launch's per-block table and returns the record with its offset and grid.
    Rec table(Rec r, const std::vector<int>& parts, std::vector<int4>* out) const {
        r.off = (long long)out->size();
        r.nseg = (int)parts.size();
        int acc = 0;
        for (int s : parts) {
            const int nt = tiles_of(r, s);
            for (int t = 0; t < nt; t++) out->push_back(make_int4(s, t, nt, acc));
            acc += nt;
        }
        r.tiles = acc;
        return r;
    }

    // The union of the systems' K-cycles is exponential in the depth of levels that take
    // two steps; a plan beyond kMaxRecs launches per outer iteration is refused.
    static constexpr size_t kMaxRecs = 1 << 16;
    bool too_big = false;

    void emit(Rec r, const std::vector<int>& parts) {
        if (parts.empty() || too_big) return;
        if (recs.size() >= kMaxRecs) {
            too_big = true;
            return;
        }
        r = table(r, parts, &tab);
        long long need = (long long)r.tiles * 3 * kBPartStride;
        if (need > max_part) max_part = need;
        recs.push_back(r);
    }

    // out = K_m(in) for the systems `parts` (level m exists for each of them).
    void K(int m, const std::vector<int>& parts, int s_in, int s_out) {
        if (too_big) return;
        std::vector<int> dense, fcg, two;
        for (int s : parts) (m == nlev[s] - 1 ? dense : fcg).push_back(s);
        {
            Rec r = rec(BK_DENSE, m);
            r.s_r = s_in;
            r.s_y = s_out;
            emit(r, dense);
        }
        if (fcg.empty()) return;
        B(m, fcg, s_in, BS_C1);
        {
            Rec r = rec(BK_ROW, m);
            r.mode = RB_SPMV;
            r.ndots = 2;
            r.s_x = BS_C1;
            r.s_y = BS_V1;
            r.s_d1 = s_in;
            r.res_row = 0;  // rho1, alpha1
            emit(r, fcg);
        }
        for (int s : fcg)
            if (L(s, m).inner >= 2) two.push_back(s);
        if (!two.empty()) {
            Rec r = rec(BK_KC_RT, m);
            r.s_r = s_in;
            emit(r, two);
            B(m, two, BS_RT, BS_C2);
            Rec q = rec(BK_ROW, m);
            q.mode = RB_SPMV;
            q.ndots = 3;
            q.s_x = BS_C2;
            q.s_y = BS_V2;
            q.s_d1 = BS_V1;
            q.s_d2 = BS_RT;
            q.res_row = 2;  // beta, gamma, alpha2
            emit(q, two);
        }
        Rec c = rec(BK_COMBINE, m);
        c.s_y = s_out;
        emit(c, fcg);
    }

    // out = B_l(in): one pre-sweep from zero, restriction, K_{l+1}, prolongation and one
    // post-sweep (every system has a level below l).
    void B(int l, const std::vector<int>& parts, int s_in, int s_out) {
        Rec a = rec(BK_ROW, l);
        a.mode = RB_PRE1;
        a.s_r = s_in;
        a.s_y = BS_W;
        a.s_y2 = BS_S;
        emit(a, parts);
        emit(rec(BK_RESTRICT, l), parts);
        K(l + 1, parts, BS_RHS, BS_OUT);
        Rec b = rec(BK_ROW, l);
        b.mode = RB_PROSMOOTH;
        b.s_r = s_in;
        b.s_x = BS_W;
        b.s_e = BS_OUT;
        b.s_y = s_out;
        emit(b, parts);
    }

    // One outer flexible-CG iteration of every system.
    void outer(const std::vector<int>& all, bool mixed) {
        if (mixed) emit(rec(BK_CAST, 0), all);
        const int s_in = mixed ? BS_RHS : BS_R;
        std::vector<int> dense, rest;
        for (int s : all) (nlev[s] == 1 ? dense : rest).push_back(s);
        Rec d = rec(BK_DENSE, 0);
        d.s_r = s_in;
        d.s_y = BS_OUT;
        emit(d, dense);
        if (!rest.empty()) B(0, rest, s_in, BS_OUT);
        emit(rec(BK_ZQ, 0), all);
        emit(rec(BK_P, 0), all);
        Rec q = rec(BK_ROW, 0);
        q.mode = RB_SPMV;
        q.ndots = 2;
        q.s_x = BS_P;
        q.s_y = BS_Q;
        q.s_d1 = BS_R;
        q.res_os = 1;
        q.res_row = 0;  // pq, pr
        q.outer = 1;
        q.dbl = true;
        emit(q, all);
        Rec x = rec(BK_XR, 0);
        x.dbl = true;
        emit(x, all);
    }
};

// The FP64 residual r = b - A x with (r, r) into os row 3, for the systems `parts`.
Rec resid_rec() {
    Rec r = rec(BK_ROW, 0);
    r.mode = RB_RESID;
    r.ndots = 1;
    r.s_r = BS_B;
    r.s_x = BS_X;
    r.s_y = BS_R;
    r.res_os = 1;
    r.res_row = 3;
    r.outer = 1;
    r.dbl = true;
    return r;
}

struct Batch {
    Handle bh;  // the batch's own allocations, stream and launch count
    bool mixed = false;
    int nsys = 0;
    BLevel* d_lev = nullptr;
    int4* d_tab = nullptr;
    int4* d_chk = nullptr;  // tables of the convergence checks
    int* d_active = nullptr;
    double* d_os = nullptr;
    double* h_os = nullptr;  // pinned mirror
    double* partials = nullptr;
    unsigned int* counters = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long graph_nodes = 0;
};

int run(Batch& bt, const Rec& r, const int4* tab) {
    BArgs a{};
    a.lev = bt.d_lev;
    a.tinfo = tab + r.off;
    a.nseg = r.nseg;
    a.active = bt.d_active;
    a.level = r.level;
    a.s_r = r.s_r;
    a.s_x = r.s_x;
    a.s_y = r.s_y;
    a.s_y2 = r.s_y2;
    a.s_d1 = r.s_d1;
    a.s_d2 = r.s_d2;
    a.s_e = r.s_e;
    a.res_os = r.res_os;
    a.res_row = r.res_row;
    a.outer = r.outer;
    a.partials = bt.partials;
    a.counters = bt.counters;
    const bool pdl = r.tiles <= 4 * bt.bh.num_sms;  // small launches overlap their start
    int st = (r.dbl || !bt.mixed)
                 ? launch_batch<double>(bt.bh.work, r.kind, r.mode, r.ndots, a, r.tiles, pdl)
                 : launch_batch<float>(bt.bh.work, r.kind, r.mode, r.ndots, a, r.tiles, pdl);
    if (st == UAAMG_OK) count_launch(&bt.bh);
    return st;
}

}  // namespace

int solve_batch(Handle* const* hs, int nsys, const int* R, const double* const* B,
                double* const* X, double tol, int* iters, double* relres, cudaStream_t user) {
    const int dev = hs[0]->device;
    const bool mixed = hs[0]->p.precision == UAAMG_MIXED;
    for (int s = 0; s < nsys; s++) {
        const Handle* h = hs[s];
        if (h->device != dev || (h->p.precision == UAAMG_MIXED) != mixed)
            return UAAMG_ERR_INVALID_ARG;
        if (R[s] < 1 || R[s] > kBMaxR || h->p.pre != 1 || h->p.post != 1)
            return UAAMG_ERR_UNSUPPORTED;
    }
    int st = UAAMG_OK;
    for (int s = 0; s < nsys && st == UAAMG_OK; s++) st = ensure_multi(hs[s], R[s]);
    if (st) return st;

    Batch bt;
    bt.mixed = mixed;
    bt.nsys = nsys;
    bt.bh.device = dev;
    bt.bh.num_sms = hs[0]->num_sms;
    if ((st = check_cuda(cudaStreamCreateWithFlags(&bt.bh.work, cudaStreamNonBlocking)))) return st;
    bt.bh.user = bt.bh.work;
    std::vector<cudaEvent_t> evs;
    auto order_after = [&](cudaStream_t from) {  // the batch stream waits for `from`
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        cudaEventRecord(e, from);
        cudaStreamWaitEvent(bt.bh.work, e, 0);
        evs.push_back(e);
    };
    order_after(user);
    for (int s = 0; s < nsys; s++) order_after(hs[s]->work);

    // descriptors
    std::vector<BLevel> lev((size_t)nsys * kMaxLevels);
    memset(lev.data(), 0, sizeof(BLevel) * lev.size());
    std::vector<long long> os_off(nsys + 1, 0);
    for (int s = 0; s < nsys; s++) os_off[s + 1] = os_off[s] + 8LL * R[s];
    Plan plan;
    plan.lev = &lev;
    plan.nlev.resize(nsys);
    for (int s = 0; s < nsys; s++) {
        const Handle* h = hs[s];
        plan.nlev[s] = h->nlev;
        for (int l = 0; l < h->nlev; l++) {
            const Level& Lv = h->lev[l];
            const MultiLevel& M = h->mlev[l];
            BLevel& D = lev[(size_t)s * kMaxLevels + l];
            D.n = Lv.n;
            D.R = R[s];
            D.nc = (l < h->nlev - 1) ? Lv.nc : 0;
            int inner = h->p.kcycle_inner;
            if (l >= 1 && inner == 2 && h->p.kcycle_ratio > 0.0 &&
                (double)h->lev[l - 1].n < h->p.kcycle_ratio * (double)Lv.n)
                inner = 1;  // a level reached by weak coarsening takes one step
            D.inner = inner;
            D.tau = h->p.kcycle_tau;
            D.rowptr = Lv.rowptr;
            D.col = Lv.col;
            D.val = mixed ? (const void*)Lv.val32 : (const void*)Lv.val64;
            D.val64 = Lv.val64;
            D.minv = mixed ? (const void*)Lv.minv32 : (const void*)Lv.minv64;
            D.agg = Lv.agg;
            D.aggptr = Lv.aggptr;
            D.members = Lv.members;
            D.inv = (l == h->nlev - 1) ? h->coarse_inv : nullptr;
            D.v[BS_RHS] = M.rhs;
            D.v[BS_OUT] = M.out;
            D.v[BS_W] = M.w;
            D.v[BS_S] = M.s;
            D.v[BS_C1] = M.c1;
            D.v[BS_V1] = M.v1;
            D.v[BS_RT] = M.rt;
            D.v[BS_C2] = M.c2;
            D.v[BS_V2] = M.v2;
            D.sc = M.sc;
            if (l == 0) {
                D.v[BS_B] = h->mb;
                D.v[BS_X] = h->mx;
                D.v[BS_R] = h->mr;
                D.v[BS_P] = h->mp;
                D.v[BS_Q] = h->mq;
            }
        }
    }
    std::vector<int> all(nsys);
    for (int s = 0; s < nsys; s++) all[s] = s;
    plan.outer(all, mixed);
    if (plan.too_big) return UAAMG_ERR_UNSUPPORTED;
    const size_t n_iter_recs = plan.recs.size();
    // launches outside the iteration graph, over every system
    plan.emit(rec(BK_INIT, 0), all);
    plan.emit(rec(BK_NORM, 0), all);
    plan.emit(resid_rec(), all);
    const Rec r_init = plan.recs[n_iter_recs], r_norm = plan.recs[n_iter_recs + 1];
    const Rec r_resid = plan.recs[n_iter_recs + 2];
    {
        long long need = (long long)r_resid.tiles * 3 * kBPartStride;
        if (need > plan.max_part) plan.max_part = need;
    }

    // device buffers of the batch (stream-ordered, released at the end)
    bt.d_lev = dalloc<BLevel>(&bt.bh, lev.size(), &st);
    bt.d_tab = dalloc<int4>(&bt.bh, plan.tab.size(), &st);
    bt.d_chk = dalloc<int4>(&bt.bh, (size_t)r_resid.tiles, &st);
    bt.d_active = dalloc<int>(&bt.bh, nsys, &st);
    bt.d_os = dalloc<double>(&bt.bh, (size_t)os_off[nsys], &st);
    bt.partials = dalloc<double>(&bt.bh, (size_t)plan.max_part, &st);
    bt.counters = dalloc<unsigned int>(&bt.bh, nsys, &st);
    if (st == UAAMG_OK &&
        !(bt.h_os = static_cast<double*>(pinned_get(sizeof(double) * os_off[nsys]))))
        st = UAAMG_ERR_OOM;
    std::vector<int> h_active(nsys, 1);
    std::vector<int4> h_chk;
    int status = UAAMG_OK;
    std::vector<std::vector<int>> colact(nsys);
    std::vector<double> bn((size_t)os_off[nsys] / 8), rn((size_t)os_off[nsys] / 8);
    std::vector<long long> col0(nsys + 1, 0);  // first flat column of each system
    for (int s = 0; s < nsys; s++) col0[s + 1] = col0[s] + R[s];
    cudaStream_t ws = bt.bh.work;
    auto fail = [&](int code) {
        cudaStreamSynchronize(ws);
        if (bt.graph) cudaGraphExecDestroy(bt.graph);
        dfree_all(&bt.bh);
        cudaStreamSynchronize(ws);
        pinned_put(bt.h_os);
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        cudaStreamDestroy(ws);
        cudaGetLastError();
        return code;
    };
    if (st) return fail(st);
    for (int s = 0; s < nsys; s++) lev[(size_t)s * kMaxLevels].os = bt.d_os + os_off[s];
    // outer scalars: rows 0-5 zero, 6 (active column) and 7 (first direction) one
    for (int s = 0; s < nsys; s++) {
        double* o = bt.h_os + os_off[s];
        for (int k = 0; k < 8 * R[s]; k++) o[k] = (k >= 6 * R[s]) ? 1.0 : 0.0;
    }
    cudaMemcpyAsync(bt.d_lev, lev.data(), sizeof(BLevel) * lev.size(), cudaMemcpyHostToDevice, ws);
    cudaMemcpyAsync(bt.d_tab, plan.tab.data(), sizeof(int4) * plan.tab.size(),
                    cudaMemcpyHostToDevice, ws);
    cudaMemcpyAsync(bt.d_active, h_active.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, ws);
    cudaMemcpyAsync(bt.d_os, bt.h_os, sizeof(double) * os_off[nsys], cudaMemcpyHostToDevice, ws);
    cudaMemsetAsync(bt.counters, 0, sizeof(unsigned int) * nsys, ws);
    for (int s = 0; s < nsys && st == UAAMG_OK; s++)
        st = check_cuda(cudaMemcpyAsync(hs[s]->mb, B[s], sizeof(double) * hs[s]->lev[0].n * R[s],
                                        cudaMemcpyDefault, ws));
    if (st == UAAMG_OK) st = run(bt, r_init, bt.d_tab);
    if (st == UAAMG_OK) st = run(bt, r_norm, bt.d_tab);
    if (st == UAAMG_OK) st = run(bt, r_resid, bt.d_tab);
    auto read_os = [&]() {
        int e = check_cuda(cudaMemcpyAsync(bt.h_os, bt.d_os, sizeof(double) * os_off[nsys],
                                           cudaMemcpyDeviceToHost, ws));
        if (e == UAAMG_OK) e = check_cuda(cudaStreamSynchronize(ws));
        return e;
    };
    if (st == UAAMG_OK) st = read_os();
    if (st) return fail(st);
    for (int s = 0; s < nsys; s++) {
        const double* o = bt.h_os + os_off[s];
        colact[s].assign(R[s], 1);
        int any = 0;
        for (int c = 0; c < R[s]; c++) {
            const size_t k = col0[s] + c;
            iters[k] = 0;
            bn[k] = sqrt(o[4 * R[s] + c]);
            rn[k] = sqrt(o[3 * R[s] + c]);
            if (bn[k] == 0.0) bn[k] = 1.0;
            if (rn[k] <= tol * bn[k]) colact[s][c] = 0;
            any |= colact[s][c];
        }
        h_active[s] = any;
    }
    // pushes the column flags (os row 6) of the systems in `which` and the system flags
    auto push_flags = [&](const std::vector<int>& which) {
        for (int s : which) {
            double* o = bt.h_os + os_off[s];
            for (int c = 0; c < R[s]; c++) o[6 * R[s] + c] = colact[s][c] ? 1.0 : 0.0;
            cudaMemcpyAsync(bt.d_os + os_off[s] + 6 * R[s], o + 6 * R[s], sizeof(double) * R[s],
                            cudaMemcpyHostToDevice, ws);
        }
        return check_cuda(cudaMemcpyAsync(bt.d_active, h_active.data(), sizeof(int) * nsys,
                                          cudaMemcpyHostToDevice, ws));
    };
    if ((st = push_flags(all))) return fail(st);

    // capture one outer iteration (and the read-back of the outer scalars) as a graph
    {
        cudaGraph_t g = nullptr;
        bt.bh.capturing = true;
        bt.bh.graph_nodes = 0;
        st = check_cuda(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
        if (st == UAAMG_OK) {
            int st2 = UAAMG_OK;
            for (size_t k = 0; k < n_iter_recs && st2 == UAAMG_OK; k++)
                st2 = run(bt, plan.recs[k], bt.d_tab);
            if (st2 == UAAMG_OK)
                st2 = check_cuda(cudaMemcpyAsync(bt.h_os, bt.d_os, sizeof(double) * os_off[nsys],
                                                 cudaMemcpyDeviceToHost, ws));
            st = check_cuda(cudaStreamEndCapture(ws, &g));
            if (st2) st = st2;
        }
        bt.bh.capturing = false;
        bt.graph_nodes = bt.bh.graph_nodes;
        if (st == UAAMG_OK) st = check_cuda(cudaGraphInstantiate(&bt.graph, g, 0));
        if (g) cudaGraphDestroy(g);
        if (st) return fail(st);
    }
    int max_iter = 0;
    for (int s = 0; s < nsys; s++) max_iter = std::max(max_iter, hs[s]->p.max_iter);
    auto n_active = [&]() {
        int a = 0;
        for (int s = 0; s < nsys; s++) a += h_active[s];
        return a;
    };
    for (int k = 1; k <= max_iter && n_active() > 0; k++) {
        st = check_cuda(cudaGraphLaunch(bt.graph, ws));
        if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(ws));
        if (st) return fail(st);
        count_launch(&bt.bh, bt.graph_nodes);
        std::vector<int> check;
        for (int s = 0; s < nsys; s++) {
            if (!h_active[s]) continue;
            const double* o = bt.h_os + os_off[s];
            bool c_any = false;
            for (int c = 0; c < R[s]; c++) {
                if (!colact[s][c]) continue;
                const size_t q = col0[s] + c;
                iters[q] = k;
                rn[q] = sqrt(o[3 * R[s] + c]);
                if (rn[q] <= tol * bn[q]) c_any = true;
            }
            if (c_any) check.push_back(s);
        }
        std::vector<int> changed;
        if (!check.empty()) {  // confirm with the recomputed FP64 residual of those systems
            h_chk.clear();
            Rec rc = plan.table(resid_rec(), check, &h_chk);
            cudaMemcpyAsync(bt.d_chk, h_chk.data(), sizeof(int4) * h_chk.size(),
                            cudaMemcpyHostToDevice, ws);
            st = run(bt, rc, bt.d_chk);
            if (st == UAAMG_OK) st = read_os();
            if (st) return fail(st);
            for (int s : check) {
                const double* o = bt.h_os + os_off[s];
                bool ch = false;
                int any = 0;
                for (int c = 0; c < R[s]; c++) {
                    if (colact[s][c]) {
                        const size_t q = col0[s] + c;
                        rn[q] = sqrt(o[3 * R[s] + c]);
                        if (rn[q] <= tol * bn[q]) {
                            colact[s][c] = 0;
                            ch = true;
                        }
                    }
                    any |= colact[s][c];
                }
                h_active[s] = any;
                if (ch) changed.push_back(s);
            }
        }
        for (int s = 0; s < nsys; s++) {  // systems at their own iteration limit stop
            if (h_active[s] && k >= hs[s]->p.max_iter) {
                h_active[s] = 0;
                if (std::find(changed.begin(), changed.end(), s) == changed.end())
                    changed.push_back(s);
            }
        }
        if (!changed.empty() && (st = push_flags(changed))) return fail(st);
    }
    // final residual of every column from b - A x, and the solutions
    std::fill(h_active.begin(), h_active.end(), 1);
    st = check_cuda(cudaMemcpyAsync(bt.d_active, h_active.data(), sizeof(int) * nsys,
                                    cudaMemcpyHostToDevice, ws));
    if (st == UAAMG_OK) st = run(bt, r_resid, bt.d_tab);
    if (st == UAAMG_OK) st = read_os();
    if (st) return fail(st);
    for (int s = 0; s < nsys; s++) {
        const double* o = bt.h_os + os_off[s];
        for (int c = 0; c < R[s]; c++) {
            const size_t q = col0[s] + c;
            relres[q] = sqrt(o[3 * R[s] + c]) / bn[q];
            if (!(relres[q] <= tol)) status = UAAMG_ERR_NO_CONVERGENCE;
        }
        st = check_cuda(cudaMemcpyAsync(X[s], hs[s]->mx, sizeof(double) * hs[s]->lev[0].n * R[s],
                                        cudaMemcpyDefault, ws));
        if (st) return fail(st);
    }
    // every handle's later work, and the caller's stream, come after the batch
    cudaEvent_t done;
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    cudaEventRecord(done, ws);
    for (int s = 0; s < nsys; s++) cudaStreamWaitEvent(hs[s]->work, done, 0);
    cudaStreamWaitEvent(user, done, 0);
    evs.push_back(done);
    st = fail(UAAMG_OK);  // releases the batch's buffers and stream
    return st ? st : status;
}

}  // namespace uaamg

using namespace uaamg;

extern "C" {

int uaamg_solve_batch(uaamg_handle* const* handles, int32_t nsys, const int32_t* nrhs,
                      const double* const* B, double* const* X, double tol, int32_t* iters,
                      double* relres, void* stream) {
    if (!handles || nsys < 1 || !nrhs || !B || !X || !iters || !relres || !(tol >= 0.0))
        return UAAMG_ERR_INVALID_ARG;
    std::vector<Handle*> hs(nsys);
    long long cols = 0;
    for (int s = 0; s < nsys; s++) {
        hs[s] = reinterpret_cast<Handle*>(handles[s]);
        if (!hs[s] || !B[s] || !X[s] || hs[s]->nlev < 1) return UAAMG_ERR_INVALID_ARG;
        for (int t = 0; t < s; t++)
            if (hs[t] == hs[s]) return UAAMG_ERR_INVALID_ARG;  // one workspace per handle
        cols += nrhs[s];
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return UAAMG_ERR_CUDA;
    if (prev != hs[0]->device && cudaSetDevice(hs[0]->device) != cudaSuccess)
        return UAAMG_ERR_CUDA;
    std::vector<int> it(cols, 0);
    std::vector<double> rr(cols, 0.0);
    std::vector<int> R(nrhs, nrhs + nsys);
    int st = solve_batch(hs.data(), nsys, R.data(), B, X, tol, it.data(), rr.data(),
                         (cudaStream_t)stream);
    for (long long k = 0; k < cols; k++) {
        iters[k] = it[k];
        relres[k] = rr[k];
    }
    if (prev != hs[0]->device) cudaSetDevice(prev);
    return st;
}

int uaamg_setup_batch(int32_t nsys, const uaamg_csr* A, const uaamg_params* p, int32_t threads,
                      void* stream, uaamg_handle** out) {
    if (nsys < 1 || !A || !out || threads < 1) return UAAMG_ERR_INVALID_ARG;
    for (int s = 0; s < nsys; s++) out[s] = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return UAAMG_ERR_CUDA;
    const int nt = std::min<int>(threads, nsys);
    std::vector<int> res(nsys, UAAMG_OK);
    std::vector<std::thread> pool;
    for (int w = 0; w < nt; w++) {
        pool.emplace_back([&, w]() {
            cudaSetDevice(dev);
            // every handle keeps `stream` as its caller's stream; its work runs on its own
            for (int s = w; s < nsys; s += nt)
                res[s] = uaamg_setup(&A[s], p ? &p[s] : nullptr, stream, &out[s]);
        });
    }
    for (auto& t : pool) t.join();
    for (int s = 0; s < nsys; s++) {
        if (res[s] == UAAMG_OK) continue;
        for (int q = 0; q < nsys; q++) {  // all or nothing
            uaamg_free(out[q]);
            out[q] = nullptr;
        }
        return res[s];
    }
    return UAAMG_OK;
}

}  // extern "C"
