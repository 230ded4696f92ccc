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
    RB_PRE1 = 0,      // x = Minv r (first sweep from zero); s = r - A x
    RB_SMOOTH = 1,    // y = x + Minv (r - A x)
    RB_RESID = 2,     // y = r - A x          (optional dot (y, y))
    RB_PROSMOOTH = 3, // xp = x + P e; y = xp + Minv (r - A xp)
    RB_SPMV = 4,      // y = A x              (dots (x, y), (x, d1), (x, d2))
};
template <typename T>
struct RBArgs {
    int n;
    int rows;  // rows per block: 256, 128, 64 or 32 (256 / rows threads share a row)
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
};
// The vector entry a row-block kernel multiplies with column j in each mode.
template <typename T, int MODE>
__device__ __forceinline__ T rb_gather(const RBArgs<T>& a, int j) {
    if constexpr (MODE == RB_PRE1) return mul_rn(a.minv[j], a.r[j]);
    else if constexpr (MODE == RB_PROSMOOTH) return add_rn(a.x[j], a.e[a.agg[j]]);
    else return a.x[j];
}

template <typename T>
int launch_rowblock(Handle* h, int mode, int ndots, const RBArgs<T>& a);
template <typename T>
int launch_rowblock_tma(Handle* h, int mode, int ndots, const RBArgs<T>& a);

template <typename T>
int launch_restrict(Handle* h, int nc, const int* aggptr, const int* members, const T* s,
                    T* rc, const int* skip);
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
int launch_outer_xr(Handle* h, int n, double* x, double* r, const double* p, const double* q,
                    OuterScalars* osc);
int launch_dot(Handle* h, int n, const double* a, const double* b, double* result);
int launch_to_host_scalars(Handle* h);

}  // namespace uaamg
