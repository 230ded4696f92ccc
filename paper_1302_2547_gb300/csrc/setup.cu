// setup.cu -- host driver of the setup phase (Algorithm 1): builds levels 0 (finest) to
// L-1 (coarsest) while n_l > coarse_size and fewer than max_levels levels exist.  Every
// step runs in the kernels of kern_setup.cu / kern_scan.cu on the handle's stream; the host
// only reads back, per level, the pass count, n_c and nnz_c to size the next level.
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "pinned.cuh"
#include "kern_sra.cuh"
#include "kernels.cuh"

namespace uaamg {

static uint32_t level_salt(uint64_t seed, int level) {
    uint32_t s = (uint32_t)(seed ^ (seed >> 32));
    return s + 0x9E3779B9u * (uint32_t)level;
}

struct HostReadback {
    int nc, zupper, nnzc, pad;
    Ctrl ctrl;
};

static int read_back(Handle* h, const int* d_tot, HostReadback* hb) {
    cudaMemcpyAsync(&hb->nc, d_tot, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->work);
    cudaMemcpyAsync(&hb->ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->work);
    int st = check_cuda(cudaStreamSynchronize(h->work));
    if (st != UAAMG_OK) return st;
    if (hb->ctrl.err & kErrTimeout) return UAAMG_ERR_TIMEOUT;
    if (hb->ctrl.err & kErrSlots) return UAAMG_ERR_UNSUPPORTED;
    if (hb->ctrl.err & kErrBadCsr) return UAAMG_ERR_BAD_CSR;
    if (hb->ctrl.err & kErrNotSpd) return UAAMG_ERR_NOT_SPD;
    return UAAMG_OK;
}

struct Scratch {
    PaaBuffers pb;
    int *f, *g, *mo, *cnt, *scan_tmp, *d_tot, *tJ, *sJ;
    double *tV, *sV;
};

struct Csr {
    int n = 0;
    long long nnz = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
};

struct Agg {
    int nc = 0, passes = 0;
    int *agg = nullptr, *aggptr = nullptr, *members = nullptr;
};

// Algorithmic bytes of the profiled aggregation launch: every pass sweeps the adjacency of
// its vertices twice (the maximum of the candidates' priorities within distance 1, then
// the roots' test and their aggregates), and a sweep over V of the n vertices moves
// V/n (4z + 4(n+1) + 8n + n) bytes: columns, row pointers, the priorities once (gathers
// served by L2) and the state.  The first sweep of a pass covers every vertex (pull) or the
// previous pass's candidates (push), as the kernel chooses; the second the pass's own
// candidates (their counts are the kernel's per-pass slots).
static int paa_profile_bytes(Handle* h, const Csr& G, const int* d_slots, int passes) {
    std::vector<int> c(passes + 1, 0);
    int st = check_cuda(cudaMemcpyAsync(c.data(), d_slots, sizeof(int) * (passes + 1),
                                        cudaMemcpyDeviceToHost, h->work));
    if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
    if (st) return st;
    const double n = G.n, z = (double)G.nnz;
    const double full = 4.0 * z + 4.0 * (n + 1.0) + 9.0 * n;
    double bytes = 0.0;
    int prev = G.n;
    for (int p = 0; p <= passes; p++) {
        const bool pull = p == 0 || (long long)prev * 4 > G.n;  // the kernel's kPullDiv rule
        bytes += full * (pull ? 1.0 : (double)prev / n);
        if (p < passes) bytes += full * (double)c[p] / n;
        prev = c[p];
    }
    h->prof_bytes = bytes;
    return UAAMG_OK;
}

// One aggregation stage on graph G: priorities with the given salt, the passes of
// Algorithm 2, ascending coarse numbering.  Outputs are handle temporaries.
static int aggregate_stage(Handle* h, int prof_level, const Csr& G, uint32_t salt, Scratch& S,
                           uint64_t* prio, int* pass_of, HostReadback* hb, Agg* out) {
    int st;
    if ((st = launch_priority(h, G.n, G.rowptr, G.col, salt, prio))) return st;
    if ((st = launch_paa(h, prof_level, G.n, G.nnz, G.rowptr, G.col, prio, h->p.max_agg_size,
                         h->p.pass_mode, S.pb, pass_of)))
        return st;
    if ((st = launch_root_flags(h, G.n, S.pb.root_of, S.pb.agg_size, S.f, S.g))) return st;
    if ((st = scan_exclusive(h, S.f, S.f, G.n, S.d_tot + 0, S.scan_tmp))) return st;
    if ((st = scan_exclusive(h, S.g, S.g, G.n, nullptr, S.scan_tmp))) return st;
    if ((st = read_back(h, S.d_tot, hb))) return st;
    out->passes = hb->ctrl.npasses;
    out->nc = hb->nc;
    if (h->prof_class == UAAMG_KCLASS_PAA && prof_level == 0 &&
        (st = paa_profile_bytes(h, G, S.pb.slots, out->passes)))
        return st;
    if (out->nc >= G.n) return UAAMG_OK;  // no coarsening possible
    out->agg = dalloc<int>(h, G.n, &st, true);
    out->aggptr = dalloc<int>(h, out->nc + 1, &st, true);
    out->members = dalloc<int>(h, G.n, &st, true);
    if (st) return st;
    return launch_renumber(h, G.n, S.pb.root_of, S.f, S.g, G.rowptr, G.col, S.d_tot + 0,
                           out->agg, out->aggptr, out->members);
}

// Coarse operator of G under the aggregation `a` (Eq. 2.4) into C (handle temporaries).
static int assemble(Handle* h, int prof_level, const Csr& G, const Agg& a, Scratch& S,
                    HostReadback* hb, Csr* C) {
    int st;
    const int nc = a.nc;
    if ((st = launch_coarse_m(h, nc, a.aggptr, a.members, G.rowptr, S.mo))) return st;
    if ((st = scan_exclusive(h, S.mo, S.mo, nc, S.d_tot + 1, S.scan_tmp))) return st;
    if ((st = launch_coarse_build(h, prof_level, nc, a.aggptr, a.members, G.rowptr, G.col, G.val,
                                  a.agg, S.mo, S.tJ, S.tV, S.sJ, S.sV, S.cnt)))
        return st;
    C->n = nc;
    C->rowptr = dalloc<int>(h, nc + 1, &st, true);
    if (st) return st;
    if ((st = scan_exclusive(h, S.cnt, C->rowptr, nc, S.d_tot + 2, S.scan_tmp))) return st;
    cudaMemcpyAsync(C->rowptr + nc, S.d_tot + 2, sizeof(int), cudaMemcpyDeviceToDevice, h->work);
    if ((st = read_back(h, S.d_tot, hb))) return st;
    C->nnz = hb->nnzc;
    if (h->prof_class == UAAMG_KCLASS_COARSE && prof_level == 0) {
        // the assembly's minimum: the fine matrix and the aggregation once (agg, aggptr,
        // members), the coarse matrix written once
        const double n = G.n, z = (double)G.nnz, ncd = nc, zc = (double)C->nnz;
        h->prof_bytes = z * 12.0 + 12.0 * n + zc * 12.0 + 4.0 * ncd;
    }
    C->col = dalloc<int>(h, C->nnz, &st, true);
    C->val = dalloc<double>(h, C->nnz, &st, true);
    if (st) return st;
    return launch_coarse_compact(h, nc, S.mo, C->rowptr, S.cnt, S.tJ, S.tV, C->col, C->val);
}

template <typename T>
static T* keep(Handle* h, const T* src, size_t count, int* st) {
    T* dst = dalloc<T>(h, count, st);
    if (*st == UAAMG_OK)
        *st = check_cuda(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDeviceToDevice,
                                         h->work));
    return dst;
}

int build_hierarchy(Handle* h, const uaamg_csr* A) {
    int st = UAAMG_OK;
    const int n0 = A->n;
    const long long z0 = A->nnz;
    const bool mixed = (h->p.precision == UAAMG_MIXED);
    const bool twice = (h->p.agg_repeat == 2);
    HostReadback* hb = nullptr;
    hb = static_cast<HostReadback*>(pinned_get(sizeof(HostReadback)));
    if (!hb) return UAAMG_ERR_OOM;
    memset(hb, 0, sizeof(HostReadback));

    h->ctrl = dalloc<Ctrl>(h, 1, &st);
    if (st) goto done;
    cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->work);
    if (h->p.wait_limit_ns > 0)  // the source lives in the handle until it is freed
        cudaMemcpyAsync(&h->ctrl->wait_ns, &h->p.wait_limit_ns, sizeof(long long),
                        cudaMemcpyHostToDevice, h->work);

    {  // level 0: copy and validate
        Level& L = h->lev[0];
        L.n = n0;
        L.nnz = z0;
        L.rowptr = dalloc<int>(h, n0 + 1, &st);
        L.col = dalloc<int>(h, z0, &st);
        L.val64 = dalloc<double>(h, z0, &st);
        if (st) goto done;
        cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaMemcpyAsync(L.rowptr, A->rowptr, sizeof(int) * (n0 + 1), kind, h->work);
        cudaMemcpyAsync(L.col, A->col, sizeof(int) * z0, kind, h->work);
        cudaMemcpyAsync(L.val64, A->val, sizeof(double) * z0, kind, h->work);
        if ((st = launch_validate(h, n0, (int)z0, L.rowptr, L.col, L.val64))) goto done;
    }
    {
        // setup scratch, sized for level 0 (every coarser graph is smaller)
        Scratch S;
        S.pb.state = dalloc<uint8_t>(h, n0, &st, true);
        S.pb.b1 = dalloc<uint64_t>(h, 2 * (size_t)n0, &st, true);
        S.pb.blocked = dalloc<uint8_t>(h, n0, &st, true);
        S.pb.list = dalloc<int>(h, 2 * (size_t)n0, &st, true);
        S.pb.cprio = dalloc<uint64_t>(h, n0, &st, true);
        S.pb.root_of = dalloc<int>(h, n0, &st, true);
        S.pb.agg_size = dalloc<int>(h, n0, &st, true);
        S.pb.slots = dalloc<int>(h, kMaxRoundSlots, &st, true);
        S.f = dalloc<int>(h, n0, &st, true);
        S.g = dalloc<int>(h, n0, &st, true);
        S.mo = dalloc<int>(h, n0, &st, true);
        S.cnt = dalloc<int>(h, n0, &st, true);
        S.scan_tmp = dalloc<int>(h, scan_scratch_ints(n0), &st, true);
        S.d_tot = dalloc<int>(h, 4, &st, true);
        S.tJ = dalloc<int>(h, z0, &st, true);
        S.sJ = dalloc<int>(h, z0, &st, true);
        S.tV = dalloc<double>(h, z0, &st, true);
        S.sV = dalloc<double>(h, z0, &st, true);
        if (st) goto done;
        if ((st = read_back(h, S.d_tot, hb))) goto done;  // validation result

        int l = 0;
        while (h->lev[l].n > h->p.coarse_size && l + 1 < h->p.max_levels && l + 1 < kMaxLevels) {
            Level& F = h->lev[l];
            Csr G{F.n, F.nnz, F.rowptr, F.col, F.val64};
            F.prio = dalloc<uint64_t>(h, F.n, &st);
            F.pass_of = dalloc<int>(h, F.n, &st);
            if (st) goto done;
            // stage 1: priorities (Eq. 3.2) and aggregation passes (Algorithm 2) on the level
            Agg a1;
            if ((st = aggregate_stage(h, l, G, level_salt(h->p.seed, twice ? 2 * l : l), S, F.prio,
                                      F.pass_of, hb, &a1)))
                goto done;
            F.passes = a1.passes;
            if (a1.nc >= F.n) break;  // no coarsening possible: F is the coarsest level
            // subgraph reshaping of the aggregates (Section 3.2, Algorithm 3)
            if (h->p.sra_rounds > 0 &&
                (st = reshape_aggregation(h, l, G.n, G.rowptr, G.col, G.val, a1.nc, a1.agg,
                                          &a1.aggptr, &a1.members, S.scan_tmp)))
                goto done;
            Csr C1;
            if ((st = assemble(h, l, G, a1, S, hb, &C1))) goto done;
            Agg fin = a1;
            Csr Cfin = C1;
            // stage 2 (Section 3.3): aggregate the intermediate graph once more
            if (twice && C1.n > h->p.coarse_size) {
                uint64_t* prio2 = dalloc<uint64_t>(h, C1.n, &st, true);
                int* pass2 = dalloc<int>(h, C1.n, &st, true);
                if (st) goto done;
                Agg a2;
                if ((st = aggregate_stage(h, -1, C1, level_salt(h->p.seed, 2 * l + 1), S, prio2,
                                          pass2, hb, &a2)))
                    goto done;
                if (a2.nc < C1.n) {
                    Csr C2;
                    if ((st = assemble(h, -1, C1, a2, S, hb, &C2))) goto done;
                    Agg comp;
                    comp.nc = a2.nc;
                    comp.agg = dalloc<int>(h, F.n, &st, true);
                    comp.aggptr = dalloc<int>(h, a2.nc + 1, &st, true);
                    comp.members = dalloc<int>(h, F.n, &st, true);
                    int* ctmp = dalloc<int>(h, F.n, &st, true);
                    if (st) goto done;
                    if ((st = launch_compose(h, F.n, a2.nc, a1.agg, a1.aggptr, a1.members, a2.agg,
                                             a2.aggptr, a2.members, comp.agg, comp.aggptr,
                                             comp.members, ctmp, S.scan_tmp)))
                        goto done;
                    fin = comp;
                    Cfin = C2;
                }
            }
            // stagnating coarsening: a small level that barely shrinks becomes the coarsest
            if (h->p.min_coarsening > 0.0 && F.n <= kMaxCoarsest &&
                (double)F.n < h->p.min_coarsening * (double)fin.nc)
                break;
            // keep the level's aggregation and the next level's matrix
            F.nc = fin.nc;
            F.agg = keep<int>(h, fin.agg, F.n, &st);
            F.aggptr = keep<int>(h, fin.aggptr, fin.nc + 1, &st);
            F.members = keep<int>(h, fin.members, F.n, &st);
            Level& C = h->lev[l + 1];
            C.n = Cfin.n;
            C.nnz = Cfin.nnz;
            C.rowptr = keep<int>(h, Cfin.rowptr, Cfin.n + 1, &st);
            C.col = keep<int>(h, Cfin.col, Cfin.nnz, &st);
            C.val64 = keep<double>(h, Cfin.val, Cfin.nnz, &st);
            if (st) goto done;
            l++;
        }
        h->nlev = l + 1;
    }
    // l1-Jacobi data (Section 4.1) and FP32 copies on every level; rows per block of the
    // row-block kernels: as many as fit one shared-memory chunk at the level's mean row
    // length, but few enough for at least four blocks per SM
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        const double avg = (double)L.nnz / (double)L.n;
        int rb = kRowsPerBlock;
        while (rb > 32 && (rb * avg > 0.9 * kChunk || (double)L.n / rb < 4.0 * h->num_sms)) rb >>= 1;
        L.rb_rows = rb;
        L.minv64 = dalloc<double>(h, L.n, &st);
        if (mixed) {
            L.minv32 = dalloc<float>(h, L.n, &st);
            L.val32 = dalloc<float>(h, L.nnz, &st);
        }
        if (st) goto done;
        if ((st = launch_level_finish(h, L.n, L.nnz, L.rowptr, L.col, L.val64, L.minv64, L.minv32,
                                      L.val32)))
            goto done;
    }
    // sliced ELLPACK copies of the large levels (not the coarsest, which is solved densely)
    for (int l = 0; h->p.sell_rows > 0 && l < h->nlev - 1; l++)
        if (h->lev[l].n >= h->p.sell_rows && (st = build_sell(h, h->lev[l], mixed))) goto done;
    {  // coarsest level: its dense FP64 inverse
        Level& Lc = h->lev[h->nlev - 1];
        h->nco = Lc.n;
        if (Lc.n > kMaxCoarsest) {
            st = UAAMG_ERR_UNSUPPORTED;
            goto done;
        }
        double* work = dalloc<double>(h, (size_t)Lc.n * Lc.n, &st, true);
        h->coarse_inv = dalloc<double>(h, (size_t)Lc.n * Lc.n, &st);
        if (st) goto done;
        if ((st = launch_dense_coarsest(h, Lc.n, Lc.rowptr, Lc.col, Lc.val64, work, h->coarse_inv)))
            goto done;
        int* d_dummy = dalloc<int>(h, 4, &st, true);
        if (st) goto done;
        cudaMemsetAsync(d_dummy, 0, 4 * sizeof(int), h->work);
        if ((st = read_back(h, d_dummy, hb))) goto done;
    }
    {  // solve workspace
        const size_t es = mixed ? sizeof(float) : sizeof(double);
        h->b = dalloc<double>(h, n0, &st);
        h->x = dalloc<double>(h, n0, &st);
        h->r = dalloc<double>(h, n0, &st);
        h->p_ = dalloc<double>(h, n0, &st);
        h->q = dalloc<double>(h, n0, &st);
        h->osc = dalloc<OuterScalars>(h, 1, &st);
        LevelScalars* sc = dalloc<LevelScalars>(h, h->nlev, &st);
        // partial sums of the widest reduction: three dots over blocks of at least 32 rows
        long long pcap = (long long)grid_for(n0, 32) * 3;
        if (pcap < 16LL * h->num_sms) pcap = 16LL * h->num_sms;
        h->partials = dalloc<double>(h, pcap, &st);
        h->partials_cap = pcap;
        if (st) goto done;
        cudaMemsetAsync(sc, 0, sizeof(LevelScalars) * h->nlev, h->work);
        cudaMemsetAsync(h->p_, 0, sizeof(double) * n0, h->work);
        cudaMemsetAsync(h->q, 0, sizeof(double) * n0, h->work);
        for (int l = 0; l < h->nlev; l++) {
            Level& L = h->lev[l];
            L.sc = sc + l;
            const bool coarsest = (l == h->nlev - 1);
            if (l == 0 && !mixed) L.rhs = h->r;
            else L.rhs = dalloc_bytes(h, es * L.n, &st);
            L.out = dalloc_bytes(h, es * L.n, &st);
            if (!coarsest) {
                L.w = dalloc_bytes(h, es * L.n, &st);
                L.s = dalloc_bytes(h, es * L.n, &st);
            }
            if (l >= 1 && !coarsest) {
                L.c1 = dalloc_bytes(h, es * L.n, &st);
                L.v1 = dalloc_bytes(h, es * L.n, &st);
                L.rt = dalloc_bytes(h, es * L.n, &st);
                L.c2 = dalloc_bytes(h, es * L.n, &st);
                L.v2 = dalloc_bytes(h, es * L.n, &st);
            }
            if (st) goto done;
        }
        h->osc_host = static_cast<OuterScalars*>(pinned_get(sizeof(OuterScalars)));
        if (!h->osc_host) st = UAAMG_ERR_OOM;
    }
    {  // levels small enough for a fused K-cycle kernel (one pre- and post-sweep only): the
        // cluster kernel where its levels fit in the cluster's shared memory, else one block
        auto first_below = [&](int below) {
            if (h->p.pre == 1 && h->p.post == 1)
                for (int l = 1; l < h->nlev - 1; l++)
                    if (h->lev[l].n <= below) return l;
            return 0;
        };
        if (st == UAAMG_OK && h->p.cluster_below > 0) {
            const int m = first_below(h->p.cluster_below);
            if (m > 0) st = tail_cluster_prepare(h, m);
        }
        if (st == UAAMG_OK && h->tail_level == 0) {
            const int m0 = first_below(h->p.fuse_below);
            h->tail_cluster = false;
            if (m0 > 0) {
                std::vector<TailLevel> tl(h->nlev);
                for (int l = 0; l < h->nlev; l++) {
                    const Level& L = h->lev[l];
                    TailLevel& t = tl[l];
                    memset(&t, 0, sizeof(t));
                    t.n = L.n;
                    int inner = h->p.kcycle_inner;
                    if (l >= 1 && inner == 2 && h->p.kcycle_ratio > 0.0 &&
                        (double)h->lev[l - 1].n < h->p.kcycle_ratio * (double)L.n)
                        inner = 1;
                    t.inner = inner;
                    t.rowptr = L.rowptr;
                    t.col = L.col;
                    t.agg = L.agg;
                    t.aggptr = L.aggptr;
                    t.members = L.members;
                    t.val = mixed ? (const void*)L.val32 : (const void*)L.val64;
                    t.minv = mixed ? (const void*)L.minv32 : (const void*)L.minv64;
                    t.rhs = L.rhs;
                    t.out = L.out;
                    t.w = L.w;
                    t.s = L.s;
                    t.c1 = L.c1;
                    t.v1 = L.v1;
                    t.rt = L.rt;
                    t.c2 = L.c2;
                    t.v2 = L.v2;
                }
                h->tail_dev = dalloc<TailLevel>(h, h->nlev, &st);
                if (st == UAAMG_OK) {
                    st = check_cuda(cudaMemcpyAsync(h->tail_dev, tl.data(), sizeof(TailLevel) * h->nlev,
                                                    cudaMemcpyHostToDevice, h->work));
                    if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
                    h->tail_level = m0;
                }
            }
        }
    }
    // per-level kernel choice by timing (after the workspace exists)
    if (st == UAAMG_OK && h->p.autotune) st = autotune_levels(h);
done:
    dfree_temps(h);
    cudaStreamSynchronize(h->work);  // no readback into hb is still in flight
    pinned_put(hb);
    return st;
}

}  // namespace uaamg
