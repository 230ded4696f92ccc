// setup.cu -- host driver of the setup phase (Algorithm 1): builds levels 0 (finest) to
// L-1 (coarsest) while n_l > coarse_size and fewer than max_levels levels exist.  Every
// step runs in the kernels of kern_setup.cu / kern_scan.cu on the handle's stream; the host
// only reads back, per level, the pass count, n_c and nnz_c to size the next level.
#include <string.h>

#include "common.cuh"
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

int build_hierarchy(Handle* h, const uaamg_csr* A) {
    int st = UAAMG_OK;
    const int n0 = A->n;
    const long long z0 = A->nnz;
    const bool mixed = (h->p.precision == UAAMG_MIXED);
    HostReadback* hb = nullptr;
    if (cudaMallocHost(&hb, sizeof(HostReadback)) != cudaSuccess) return UAAMG_ERR_OOM;
    memset(hb, 0, sizeof(HostReadback));

    h->ctrl = dalloc<Ctrl>(h, 1, &st);
    if (st) goto done;
    cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->work);

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
        // setup scratch, sized for level 0 (every coarser level is smaller)
        PaaBuffers pb;
        pb.state = dalloc<uint8_t>(h, n0, &st, true);
        pb.b1 = dalloc<uint64_t>(h, n0, &st, true);
        pb.blocked = dalloc<uint8_t>(h, n0, &st, true);
        pb.root_of = dalloc<int>(h, n0, &st, true);
        pb.agg_size = dalloc<int>(h, n0, &st, true);
        pb.slots = dalloc<int>(h, kMaxRoundSlots, &st, true);
        int* f = dalloc<int>(h, n0, &st, true);
        int* g = dalloc<int>(h, n0, &st, true);
        int* mo = dalloc<int>(h, n0, &st, true);
        int* cnt = dalloc<int>(h, n0, &st, true);
        int* scan_tmp = dalloc<int>(h, scan_scratch_ints(n0), &st, true);
        int* d_tot = dalloc<int>(h, 4, &st, true);
        int* tJ = dalloc<int>(h, z0, &st, true);
        int* sJ = dalloc<int>(h, z0, &st, true);
        double* tV = dalloc<double>(h, z0, &st, true);
        double* sV = dalloc<double>(h, z0, &st, true);
        if (st) goto done;
        if ((st = read_back(h, d_tot, hb))) goto done;  // validation result

        int l = 0;
        while (h->lev[l].n > h->p.coarse_size && l + 1 < h->p.max_levels && l + 1 < kMaxLevels) {
            Level& F = h->lev[l];
            F.prio = dalloc<uint64_t>(h, F.n, &st);
            F.pass_of = dalloc<int>(h, F.n, &st);
            if (st) goto done;
            // priorities (Eq. 3.2) and aggregation passes (Algorithm 2)
            if ((st = launch_priority(h, F.n, F.rowptr, F.col, level_salt(h->p.seed, l), F.prio)))
                goto done;
            if ((st = launch_paa(h, l, F.n, F.rowptr, F.col, F.prio, h->p.max_agg_size,
                                 h->p.pass_mode, pb, F.pass_of)))
                goto done;
            // coarse numbering by ascending root (Section 5.1)
            if ((st = launch_root_flags(h, F.n, pb.root_of, pb.agg_size, f, g))) goto done;
            if ((st = scan_exclusive(h, f, f, F.n, d_tot + 0, scan_tmp))) goto done;
            if ((st = scan_exclusive(h, g, g, F.n, nullptr, scan_tmp))) goto done;
            if ((st = read_back(h, d_tot, hb))) goto done;
            F.passes = hb->ctrl.npasses;
            const int nc = hb->nc;
            if (nc >= F.n) break;  // no coarsening possible: F is the coarsest level
            F.nc = nc;
            F.agg = dalloc<int>(h, F.n, &st);
            F.aggptr = dalloc<int>(h, nc + 1, &st);
            F.members = dalloc<int>(h, F.n, &st);
            if (st) goto done;
            if ((st = launch_renumber(h, F.n, pb.root_of, f, g, F.rowptr, F.col, d_tot + 0, F.agg,
                                      F.aggptr, F.members)))
                goto done;
            // coarse operator by aggregate sums (Eq. 2.4)
            if ((st = launch_coarse_m(h, nc, F.aggptr, F.members, F.rowptr, mo))) goto done;
            if ((st = scan_exclusive(h, mo, mo, nc, d_tot + 1, scan_tmp))) goto done;
            if ((st = launch_coarse_build(h, l, nc, F.aggptr, F.members, F.rowptr, F.col, F.val64,
                                          F.agg, mo, tJ, tV, sJ, sV, cnt)))
                goto done;
            Level& C = h->lev[l + 1];
            C.n = nc;
            C.rowptr = dalloc<int>(h, nc + 1, &st);
            if (st) goto done;
            if ((st = scan_exclusive(h, cnt, C.rowptr, nc, d_tot + 2, scan_tmp))) goto done;
            cudaMemcpyAsync(C.rowptr + nc, d_tot + 2, sizeof(int), cudaMemcpyDeviceToDevice, h->work);
            if ((st = read_back(h, d_tot, hb))) goto done;
            C.nnz = hb->nnzc;
            C.col = dalloc<int>(h, C.nnz, &st);
            C.val64 = dalloc<double>(h, C.nnz, &st);
            if (st) goto done;
            if ((st = launch_coarse_compact(h, nc, mo, C.rowptr, cnt, tJ, tV, C.col, C.val64)))
                goto done;
            l++;
        }
        h->nlev = l + 1;
    }
    // l1-Jacobi data (Section 4.1) and FP32 copies on every level
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
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
    {  // coarsest level: dense inverse through the Cholesky factor
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
        long long pcap = (long long)grid_for(n0, kRowsPerBlock) * 3;
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
        if (cudaMallocHost(&h->osc_host, sizeof(OuterScalars)) != cudaSuccess) st = UAAMG_ERR_OOM;
    }
done:
    dfree_temps(h);
    if (hb) cudaFreeHost(hb);
    return st;
}

}  // namespace uaamg
