// kernels.cuh -- host-side launchers of the CUDA kernels (one place for the signatures
// used by setup.cu and solve.cu).
#pragma once
#include "common.cuh"

namespace uaamg {

// ---- scan (kern_scan.cu) ----------------------------------------------------------------
size_t scan_scratch_ints(long long n);
int scan_exclusive(Handle* h, const int* in, int* out, int n, int* d_total, int* scratch);

// ---- setup (kern_setup.cu) --------------------------------------------------------------
int launch_validate(Handle* h, int n, int nnz, const int* rowptr, const int* col,
                    const double* val);
int launch_priority(Handle* h, int n, const int* rowptr, const int* col, uint32_t salt,
                    uint64_t* prio);
struct PaaBuffers {
    uint8_t* state;
    uint64_t* b1;  // 2 n entries
    uint8_t* blocked;
    int* list;     // 2 n entries
    uint64_t* cprio;  // n entries
    int* root_of;
    int* agg_size;
    int* slots;
};
int launch_paa(Handle* h, int level, int n, long long nnz, const int* rowptr, const int* col,
               const uint64_t* prio, int t, int mode, const PaaBuffers& b, int* pass_of);
int launch_root_flags(Handle* h, int n, const int* root_of, const int* agg_size, int* f, int* g);
int launch_renumber(Handle* h, int n, const int* root_of, const int* cid, const int* start,
                    const int* rowptr, const int* col, const int* d_nc, int* agg, int* aggptr,
                    int* members);
int launch_coarse_m(Handle* h, int nc, const int* aggptr, const int* members,
                    const int* rowptr, int* m);
int launch_coarse_build(Handle* h, int level, int nc, const int* aggptr, const int* members,
                        const int* rowptr, const int* col, const double* val, const int* agg,
                        const int* off, int* tJ, double* tV, int* sJ, double* sV, int* cnt);
int launch_coarse_compact(Handle* h, int nc, const int* off, const int* rowptr_c,
                          const int* cnt, const int* tJ, const double* tV, int* col_c,
                          double* val_c);
int launch_compose(Handle* h, int n, int nc, const int* agg1, const int* aggptr1,
                   const int* members1, const int* agg2, const int* aggptr2,
                   const int* members2, int* agg, int* aggptr, int* members, int* tmp,
                   int* scan_tmp);
int launch_level_finish(Handle* h, int n, long long nnz, const int* rowptr, const int* col,
                        const double* val64, double* minv64, float* minv32, float* val32);
int launch_dense_coarsest(Handle* h, int n, const int* rowptr, const int* col,
                          const double* val, double* work, double* inv);

// ---- solve (kern_solve.cu) --------------------------------------------------------------
// Row-block CSR kernels (Section 4.4 SpMV fused with the Section 4.1 smoother).
enum RBMode {
    RB_PRE1 = 0,        // x = Minv r (first sweep from zero); s = r - A x
    RB_SMOOTH = 1,      // y = x + Minv (r - A x)
    RB_RESID = 2,       // y = r - A x          (optional dot (y, y))
    RB_PROSMOOTH = 3,   // xp = x + P e; y = xp + Minv (r - A xp)
    RB_SPMV = 4,        // y = A x              (dots (x, y), (x, d1), (x, d2))
    RB_PRE1_RT = 5,     // RB_PRE1 with r = rho~ = rho - a1 v1 formed on the fly; writes rho~
    RB_PROSMOOTH_E = 6, // RB_PROSMOOTH with e = w1 c1 + w2 c2 formed on the fly
};
// Arguments of the row-block kernels.  The two fused modes take over the element-wise K-cycle
// steps (Section 4.3) with the same arithmetic per entry:
//   RB_PRE1_RT reads r = rho (the coarse right-hand side), d1 = v1 and rsc (a1 = alpha1/rho1)
//     and writes rho~ to y3;
//   RB_PROSMOOTH_E reads e = c1, e2 = c2 and esc (w1, w2) of coarse level elevel, and clears
//     that level's skip value (elevel + 1) in skip_rw.
// ksc != null on the first SpMV of a K-cycle step: its last block, once rho1 is summed,
// decides whether level klevel takes a second step (kinner = steps allowed).
template <typename T>
struct RBArgs {
    int n;
    int rows;  // rows per block: 256, 128, 64 or 32 (256 / rows threads share a row)
    long long nnz;  // stored entries (0 if not given)
    const int* rowptr;
    const int* col;
    const T* val;
    const T* minv;
    const T* r;
    const T* x;
    const int* agg;
    const T* e;
    T* y;
    T* y2;
    const T* d1;
    const T* d2;
    double* partials;
    unsigned int* counter;
    double* result;
    const int* skip;
    const T* e2;
    const LevelScalars* esc;
    int elevel;
    T* y3;
    const LevelScalars* rsc;
    LevelScalars* ksc;
    int klevel, kinner;
    int* skip_rw;
    LevelScalars* wsc;   // second SpMV of a K-cycle step: w1, w2 from its three dots
    OuterScalars* aosc;  // the outer SpMV: alpha from (p, A p) and (p, r)
    // sliced ELLPACK copy of the level (sptr != null: the SELL kernels run)
    const int* sptr;
    const int* scol;
    const T* sval;
    const uint16_t* slen;
    int nslices;
    int path;  // kernel family chosen for the level (-1: by the size thresholds)
};

// Scalars of the fused modes, read once per thread at kernel start.
template <typename T>
struct KScal {
    T a1, w1, w2;
    bool two;
};
template <typename T, int MODE>
__device__ __forceinline__ KScal<T> kscal(const RBArgs<T>& a) {
    KScal<T> k{T(0), T(0), T(0), false};
    if constexpr (sizeof(T) == 4) {  // FP32 copies rounded once by the reduction hooks
        if constexpr (MODE == RB_PRE1_RT) k.a1 = a.rsc->a1f;
        if constexpr (MODE == RB_PROSMOOTH_E) {
            k.w1 = a.esc->w1f;
            k.w2 = a.esc->w2f;
            k.two = a.esc->w2 != 0.0;
        }
    } else {
        if constexpr (MODE == RB_PRE1_RT) k.a1 = a.rsc->a1;
        if constexpr (MODE == RB_PROSMOOTH_E) {
            k.w1 = a.esc->w1;
            k.w2 = a.esc->w2;
            k.two = a.esc->w2 != 0.0;
        }
    }
    return k;
}
// rho~_j = rho_j - a1 v1_j and e_I = w1 c1_I (+ w2 c2_I), as the unfused steps compute them.
template <typename T>
__device__ __forceinline__ T kc_rt_at(const RBArgs<T>& a, const KScal<T>& k, int j) {
    return sub_rn(a.r[j], mul_rn(k.a1, a.d1[j]));
}
template <typename T>
__device__ __forceinline__ T kc_e_at(const RBArgs<T>& a, const KScal<T>& k, int I) {
    T v = mul_rn(k.w1, a.e[I]);
    if (k.two) v = add_rn(v, mul_rn(k.w2, a.e2[I]));
    return v;
}

// The vector entry a row-block kernel multiplies with column j in each mode.
template <typename T, int MODE>
__device__ __forceinline__ T rb_gather(const RBArgs<T>& a, const KScal<T>& k, int j) {
    if constexpr (MODE == RB_PRE1) return mul_rn(a.minv[j], a.r[j]);
    else if constexpr (MODE == RB_PRE1_RT) return mul_rn(a.minv[j], kc_rt_at(a, k, j));
    else if constexpr (MODE == RB_PROSMOOTH) return add_rn(a.x[j], a.e[a.agg[j]]);
    else if constexpr (MODE == RB_PROSMOOTH_E) return add_rn(a.x[j], kc_e_at(a, k, a.agg[j]));
    else return a.x[j];
}

// The operands a one-thread-per-row kernel loads for row i before its sum, by mode.
template <typename T>
struct RowOps {
    T ri, mi, xi, d1i, d2i;
    int gi;
};
template <typename T, int MODE, int ND>
__device__ __forceinline__ RowOps<T> rb_row_ops(const RBArgs<T>& a, const KScal<T>& ks, int i) {
    RowOps<T> o{T(0), T(0), T(0), T(0), T(0), 0};
    constexpr bool pro = MODE == RB_PROSMOOTH || MODE == RB_PROSMOOTH_E;
    if constexpr (MODE == RB_PRE1_RT) o.ri = kc_rt_at(a, ks, i);
    else if constexpr (MODE == RB_PRE1 || MODE == RB_SMOOTH || pro || MODE == RB_RESID)
        o.ri = a.r[i];
    if constexpr (MODE == RB_PRE1 || MODE == RB_PRE1_RT || MODE == RB_SMOOTH || pro)
        o.mi = a.minv[i];
    if constexpr (MODE == RB_SMOOTH || pro || MODE == RB_SPMV) o.xi = a.x[i];
    if constexpr (MODE == RB_SPMV && ND >= 2) o.d1i = a.d1[i];
    if constexpr (MODE == RB_SPMV && ND >= 3) o.d2i = a.d2[i];
    if constexpr (pro) o.gi = a.agg[i];
    return o;
}
// Row i's outputs from its sum acc = (A v)_i, by mode (the same arithmetic as k_rowblock).
template <typename T, int MODE, int ND>
__device__ __forceinline__ void rb_row_out(const RBArgs<T>& a, const KScal<T>& ks, int i, T acc,
                                           const RowOps<T>& o, double (&dv)[ND > 0 ? ND : 1]) {
    if constexpr (MODE == RB_PRE1) {
        a.y[i] = mul_rn(o.mi, o.ri);
        a.y2[i] = sub_rn(o.ri, acc);
    } else if constexpr (MODE == RB_PRE1_RT) {
        a.y[i] = mul_rn(o.mi, o.ri);
        a.y2[i] = sub_rn(o.ri, acc);
        a.y3[i] = o.ri;
    } else if constexpr (MODE == RB_SMOOTH) {
        a.y[i] = add_rn(o.xi, mul_rn(o.mi, sub_rn(o.ri, acc)));
    } else if constexpr (MODE == RB_RESID) {
        const T yi = sub_rn(o.ri, acc);
        a.y[i] = yi;
        if constexpr (ND >= 1) dv[0] = fma((double)yi, (double)yi, dv[0]);
    } else if constexpr (MODE == RB_PROSMOOTH) {
        const T xp = add_rn(o.xi, a.e[o.gi]);
        a.y[i] = add_rn(xp, mul_rn(o.mi, sub_rn(o.ri, acc)));
    } else if constexpr (MODE == RB_PROSMOOTH_E) {
        const T xp = add_rn(o.xi, kc_e_at(a, ks, o.gi));
        a.y[i] = add_rn(xp, mul_rn(o.mi, sub_rn(o.ri, acc)));
    } else {  // RB_SPMV
        a.y[i] = acc;
        const double xd = (double)o.xi;
        if constexpr (ND >= 1) dv[0] = fma(xd, (double)acc, dv[0]);
        if constexpr (ND >= 2) dv[1] = fma(xd, (double)o.d1i, dv[1]);
        if constexpr (ND >= 3) dv[2] = fma(xd, (double)o.d2i, dv[2]);
    }
}

// Kernel entry: false when the kernel lies inside a skipped second K-cycle step.  A fused
// prolongation of level elevel-1 runs when the skip value is its own child's (elevel + 1),
// which means the child skipped its second step, and clears it (block 0; a block that reads
// the cleared value runs as well).
template <typename T, int MODE>
__device__ __forceinline__ bool rb_enter(const RBArgs<T>& a) {
    if (!a.skip) return true;
    const int sk = *(volatile const int*)a.skip;
    if constexpr (MODE == RB_PROSMOOTH_E) {
        if (sk != 0 && sk != a.elevel + 1) return false;
        if (sk != 0 && blockIdx.x == 0 && threadIdx.x == 0) *a.skip_rw = 0;
        return true;
    } else {
        return sk == 0;
    }
}

// After the last block has summed rho1 = result[0] of a K-cycle's first SpMV: the second
// step is skipped when rho1 <= 0 or the level takes one step (Section 4.3 guards).
// It also sets a1 and the one-step weights (w1 = a1, w2 = 0), which a second step replaces.
template <typename T>
__device__ __forceinline__ void rb_kc_decide(const RBArgs<T>& a) {
    const double rho1 = a.result[0], alpha1 = a.result[1];
    const int skip2 = (!(rho1 > 0.0) || a.kinner < 2) ? 1 : 0;
    const double a1 = rho1 > 0.0 ? alpha1 / rho1 : 0.0;
    a.ksc->a1 = a1;
    a.ksc->w1 = a1;
    a.ksc->w2 = 0.0;
    a.ksc->a1f = (float)a1;
    a.ksc->w1f = (float)a1;
    a.ksc->w2f = 0.0f;
    a.ksc->skip2 = skip2;
    if (skip2 && a.kinner >= 2) *a.skip_rw = a.klevel + 1;
}

// After the last block has summed beta, gamma, alpha2 of a K-cycle's second step:
// rho2 = beta - gamma^2 / rho1; when rho2 > 0, w1 = a1 - gamma alpha2 / (rho1 rho2) and
// w2 = alpha2 / rho2 (Section 4.3 guards), else the one-step weights stand.
template <typename T>
__device__ __forceinline__ void rb_kc_weights(const RBArgs<T>& a) {
    LevelScalars* sc = a.wsc;
    const double rho1 = sc->rho1;
    const double beta = a.result[0], gamma = a.result[1], alpha2 = a.result[2];
    const double rho2 = beta - gamma * gamma / rho1;
    if (rho1 > 0.0 && rho2 > 0.0) {
        sc->w1 = sc->a1 - gamma * alpha2 / (rho1 * rho2);
        sc->w2 = alpha2 / rho2;
        sc->w1f = (float)sc->w1;
        sc->w2f = (float)sc->w2;
    }
}

// After the last block has summed (p, A p) and (p, r) of the outer iteration.
template <typename T>
__device__ __forceinline__ void rb_outer_alpha(const RBArgs<T>& a) {
    const double pq = a.result[0], pr = a.result[1];
    a.aosc->alpha_cur = pq > 0.0 ? pr / pq : 0.0;
}

// The hooks a row-block kernel runs in thread 0 of its last block.
template <typename T>
__device__ __forceinline__ void rb_last_block(const RBArgs<T>& a) {
    if (a.ksc) rb_kc_decide(a);
    if (a.wsc) rb_kc_weights(a);
    if (a.aosc) rb_outer_alpha(a);
}

template <typename T>
int launch_rowblock(Handle* h, int mode, int ndots, const RBArgs<T>& a);
template <typename T>
int launch_rowblock_tma(Handle* h, int mode, int ndots, const RBArgs<T>& a);
template <typename T>
int launch_sell(Handle* h, int mode, int ndots, const RBArgs<T>& a);
int build_sell(Handle* h, Level& L, bool mixed);
void drop_sell(Handle* h, Level& L);
// per-level choice of the SpMV kernel family by timing the first sweep (tune.cu)
int autotune_levels(Handle* h);

template <typename T>
int launch_restrict(Handle* h, int nc, const int* aggptr, const int* members, const T* s,
                    T* rc, const int* skip);
// RB_PRE1 / RB_PRE1_RT fused with the restriction of s = r - A x (s is not stored)
template <typename T>
int launch_pre1_restrict(Handle* h, int mode, const RBArgs<T>& a, int nc, const int* aggptr,
                         const int* members, T* rc);
template <typename T>
int launch_dense_apply(Handle* h, int n, const double* inv, const T* in, T* out,
                       const int* skip);
template <typename T>
int launch_kc_rt(Handle* h, int level, int n, const T* rho, const T* v1, T* rt,
                 LevelScalars* sc, int inner, double tau, Ctrl* ctrl);
template <typename T>
int launch_kc_combine(Handle* h, int level, int n, const T* c1, const T* c2, T* e,
                      const LevelScalars* sc, Ctrl* ctrl);
template <typename T>
int launch_copy(Handle* h, int n, const T* in, T* out, const int* skip);
template <typename T>
int launch_prolong(Handle* h, int n, const T* x, const int* agg, const T* e, T* y,
                   const int* skip);

// fused K-cycle of the levels m0 .. L-1 (kern_tail.cu)
template <typename T>
int launch_tail(Handle* h, int m0);
// Packs the cluster tail's per-block regions, starting at level m_first or, where those
// levels do not fit in shared memory, lower; sets h->tail_level (left 0 when none fits).
int tail_cluster_prepare(Handle* h, int m_first);

// R right-hand sides at once (kern_multi.cu)
template <typename T>
struct MArgs {
    int n, R;
    const int* rowptr;
    const int* col;
    const T* val;
    const T* minv;
    const T* r;
    const T* x;
    const int* agg;
    const T* e;
    T* y;
    T* y2;
    const T* d1;
    const T* d2;
    double* partials;
    unsigned int* counter;
    double* result;
};
template <typename T>
int launch_mrow(Handle* h, int mode, int ndots, const MArgs<T>& a);
template <typename T>
int launch_mrestrict(Handle* h, int nc, int R, const int* aggptr, const int* members,
                     const T* s, T* rc);
template <typename T>
int launch_mdense(Handle* h, int n, int R, const double* inv, const T* in, T* out);
template <typename T>
int launch_mkc_rt(Handle* h, int n, int R, const T* rho, const T* v1, T* rt, double* sc,
                  bool tau);
template <typename T>
int launch_mkc_combine(Handle* h, int n, int R, const T* c1, const T* c2, T* e,
                       const double* sc, int second, double tau);
int launch_mcast(Handle* h, long long m, const double* in, float* out);
template <typename T>
int launch_mouter(Handle* h, int n, int R, const T* z, double* p, const double* q, double* os);
int launch_mxr(Handle* h, int n, int R, double* x, double* r, const double* p, const double* q,
               double* os);
int launch_mnorm(Handle* h, int n, int R, const double* b, double* out);

// outer flexible CG (FP64 with the preconditioner output in T)
int launch_cast_d2f(Handle* h, int n, const double* in, float* out);
template <typename T>
int launch_outer_zq(Handle* h, int n, const T* z, const double* q, OuterScalars* osc);
template <typename T>
int launch_outer_p(Handle* h, int n, const T* z, double* p, OuterScalars* osc);
int launch_outer_loop(Handle* h, cudaGraphConditionalHandle cond);
int launch_outer_xr(Handle* h, int n, double* x, double* r, const double* p, const double* q,
                    OuterScalars* osc);
int launch_dot(Handle* h, int n, const double* a, const double* b, double* result);
int launch_to_host_scalars(Handle* h);

}  // namespace uaamg
