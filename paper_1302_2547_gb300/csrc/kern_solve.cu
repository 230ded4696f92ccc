// kern_solve.cu -- kernels of the solve phase: CSR SpMV fused with the l1-Jacobi smoother
// (Sections 4.1, 4.4), residual restriction and piecewise-constant prolongation
// (Section 4.2), the scalar steps of the K-cycle (Section 4.3) and of the outer flexible CG.
//
// Row-block SpMV: a block owns 256 consecutive rows.  Their entries form one contiguous
// range of col/val, which the block streams in chunks with coalesced 16-byte loads, storing
// each value and the gathered vector entry in shared memory; each thread then accumulates
// its own row in stored order with fused multiply-adds and applies the fused epilogue.
// Loads are therefore coalesced whatever the row lengths, and every row sum has a fixed
// order.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
    return __ldcs(p);
}


// Four consecutive matrix values with one 16-byte (FP32) or two 16-byte (FP64) loads.
__device__ __forceinline__ void ld_val4(const float* p, float (&v)[4]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void ld_val4(const double* p, double (&v)[4]) {
    const double2 q0 = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 q1 = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
}

constexpr int kGrp = 2;  // four-entry groups a thread loads per batch

template <typename T, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) k_rowblock(RBArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    if (!rb_enter<T, MODE>(a)) return;
    const KScal<T> ks = kscal<T, MODE>(a);
    __shared__ T sval[kChunk];
    __shared__ T sx[kChunk];
    const int lanes = kRowsPerBlock / a.rows;  // threads per row: 1, 2, 4 or 8
    const int sub = threadIdx.x & (lanes - 1);
    const int r0 = blockIdx.x * a.rows;
    const int r1 = min(a.n, r0 + a.rows);
    const int row = r0 + (int)threadIdx.x / lanes;
    const int k0 = a.rowptr[r0], k1 = a.rowptr[r1];
    const int ktot = a.rowptr[a.n];
    int rs = 0, re = 0;
    if (row < r1) {
        rs = a.rowptr[row];
        re = a.rowptr[row + 1];
    }
    T acc = T(0);
    for (int c0 = k0; c0 < k1; c0 += kChunk) {
        const int c1 = min(k1, c0 + kChunk);
        // groups of four entries at 16-byte aligned indices; entries outside [c0, c1) are
        // loaded (they lie inside the arrays) but not used.  Each thread loads kGrp groups,
        // then issues all their gathers before using any, so it waits for two memory round
        // trips per batch instead of one per group.
        for (int kb0 = (c0 & ~3) + 4 * (int)threadIdx.x; kb0 < c1; kb0 += 4 * kThreads * kGrp) {
            int j[kGrp][4];
            T v[kGrp][4];
#pragma unroll
            for (int g = 0; g < kGrp; g++) {
                const int kb = kb0 + g * 4 * kThreads;
                if (kb + 4 <= ktot && kb < c1) {
                    const int4 cj = __ldcs(reinterpret_cast<const int4*>(a.col + kb));
                    j[g][0] = cj.x;
                    j[g][1] = cj.y;
                    j[g][2] = cj.z;
                    j[g][3] = cj.w;
                    ld_val4(a.val + kb, v[g]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const bool in = kb < c1 && kb + e < ktot;
                        j[g][e] = in ? a.col[kb + e] : 0;
                        v[g][e] = in ? a.val[kb + e] : T(0);
                    }
                }
            }
            T xg[kGrp][4];
#pragma unroll
            for (int g = 0; g < kGrp; g++)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int k = kb0 + g * 4 * kThreads + e;
                    xg[g][e] = (k >= c0 && k < c1) ? rb_gather<T, MODE>(a, ks, j[g][e]) : T(0);
                }
#pragma unroll
            for (int g = 0; g < kGrp; g++)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int k = kb0 + g * 4 * kThreads + e;
                    if (k >= c0 && k < c1) {
                        sval[k - c0] = v[g][e];
                        sx[k - c0] = xg[g][e];
                    }
                }
        }
        __syncthreads();
        const int lo = max(rs, c0), hi = min(re, c1);
        for (int k = lo + sub; k < hi; k += lanes) acc = fma_rn(sval[k - c0], sx[k - c0], acc);
        __syncthreads();
    }
    // the lanes of a row combine their partial sums by a fixed shuffle tree
    for (int o = lanes >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lanes);
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    if (row < r1 && sub == 0) {
        const int i = row;
        if constexpr (MODE == RB_PRE1) {
            a.y[i] = mul_rn(a.minv[i], a.r[i]);
            a.y2[i] = sub_rn(a.r[i], acc);
        } else if constexpr (MODE == RB_PRE1_RT) {
            const T ri = kc_rt_at(a, ks, i);
            a.y[i] = mul_rn(a.minv[i], ri);
            a.y2[i] = sub_rn(ri, acc);
            a.y3[i] = ri;
        } else if constexpr (MODE == RB_SMOOTH) {
            a.y[i] = add_rn(a.x[i], mul_rn(a.minv[i], sub_rn(a.r[i], acc)));
        } else if constexpr (MODE == RB_RESID) {
            const T yi = sub_rn(a.r[i], acc);
            a.y[i] = yi;
            if constexpr (ND >= 1) dv[0] = (double)yi * (double)yi;
        } else if constexpr (MODE == RB_PROSMOOTH) {
            const T xi = add_rn(a.x[i], a.e[a.agg[i]]);
            a.y[i] = add_rn(xi, mul_rn(a.minv[i], sub_rn(a.r[i], acc)));
        } else if constexpr (MODE == RB_PROSMOOTH_E) {
            const T xi = add_rn(a.x[i], kc_e_at(a, ks, a.agg[i]));
            a.y[i] = add_rn(xi, mul_rn(a.minv[i], sub_rn(a.r[i], acc)));
        } else {  // RB_SPMV
            a.y[i] = acc;
            const double xi = (double)a.x[i];
            if constexpr (ND >= 1) dv[0] = xi * (double)acc;
            if constexpr (ND >= 2) dv[1] = xi * (double)a.d1[i];
            if constexpr (ND >= 3) dv[2] = xi * (double)a.d2[i];
        }
    }
    if constexpr (ND > 0) {
        if (grid_reduce<ND>(dv, a.partials, a.counter, a.result)) rb_last_block(a);
    }
}

template <typename T>
int launch_rowblock(Handle* h, int mode, int ndots, const RBArgs<T>& a) {
    // the level's kernel family: the tuner's choice, else the size thresholds
    if (a.sptr && (a.path == 2 || a.path < 0))
        return launch_sell<T>(h, mode, ndots, a);  // sliced ELLPACK copy
    if (a.path == 1 || (a.path < 0 && h->p.tma_rows > 0 && a.n >= h->p.tma_rows))
        return launch_rowblock_tma<T>(h, mode, ndots, a);  // matrix stream via bulk copies
    const int grid = grid_for(a.n, a.rows);
    cudaStream_t st = h->work;
#define RB_CASE(M, D)                                                 \
    if (mode == M && ndots == D) {                                    \
        cudaError_t e = launch_k(a.n <= kPdlMaxRows, k_rowblock<T, M, D>, dim3(grid), \
                                 dim3(kThreads), 0, st, a);                          \
        count_launch(h);                                              \
        return check_cuda(e);                                         \
    }
    RB_CASE(RB_PRE1, 0)
    RB_CASE(RB_PRE1_RT, 0)
    RB_CASE(RB_PROSMOOTH_E, 0)
    RB_CASE(RB_SMOOTH, 0)
    RB_CASE(RB_RESID, 0)
    RB_CASE(RB_RESID, 1)
    RB_CASE(RB_PROSMOOTH, 0)
    RB_CASE(RB_SPMV, 0)
    RB_CASE(RB_SPMV, 2)
    RB_CASE(RB_SPMV, 3)
#undef RB_CASE
    return UAAMG_ERR_INVALID_ARG;
}

template int launch_rowblock<float>(Handle*, int, int, const RBArgs<float>&);
template int launch_rowblock<double>(Handle*, int, int, const RBArgs<double>&);

// ---------------------------------------------------------------------------------------
// Restriction (Section 4.2): (P^T s)_I = sum of s over the members of aggregate I, one
// thread per coarse entry, members in ascending order.
constexpr int kRestrictBatch = 8;  // members whose loads a thread has in flight
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_restrict(int nc, const int* __restrict__ aggptr, const int* __restrict__ members,
           const T* __restrict__ s, T* __restrict__ rc, const int* skip) {
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    const int q1 = aggptr[I + 1];
    T sum = T(0);
    for (int q = aggptr[I]; q < q1; q += kRestrictBatch) {  // members' loads issued together
        int m[kRestrictBatch];
        T v[kRestrictBatch];
#pragma unroll
        for (int u = 0; u < kRestrictBatch; u++) m[u] = q + u < q1 ? members[q + u] : 0;
#pragma unroll
        for (int u = 0; u < kRestrictBatch; u++) v[u] = q + u < q1 ? s[m[u]] : T(0);
#pragma unroll
        for (int u = 0; u < kRestrictBatch; u++)
            if (q + u < q1) sum = add_rn(sum, v[u]);
    }
    rc[I] = sum;
}

template <typename T>
int launch_restrict(Handle* h, int nc, const int* aggptr, const int* members, const T* s,
                    T* rc, const int* skip) {
    cudaError_t e = launch_k(nc <= kPdlMaxRows, k_restrict<T>, dim3(grid_for(nc, kThreads)),
                             dim3(kThreads), 0, h->work, nc, aggptr, members, s, rc, skip);
    count_launch(h);
    return check_cuda(e);
}
template int launch_restrict<float>(Handle*, int, const int*, const int*, const float*, float*, const int*);
template int launch_restrict<double>(Handle*, int, const int*, const int*, const double*, double*, const int*);

// ---------------------------------------------------------------------------------------
// The first sweep fused with the restriction (Sections 4.1, 4.2): for every aggregate I,
// x_j = Minv_j r_j for its members j and r_c[I] = sum_j (r_j - (A x)_j), members in
// ascending order, so the residual s = r - A x is never stored.  One warp per aggregate,
// one lane per member (32 at a time); each lane adds its row in stored order with fused
// multiply-adds, eight entries' loads issued together, and lane 0 adds the members'
// residuals in order.  With RT, r = rho~ = rho - a1 v1 is formed on the fly and stored in
// `y3` (as RB_PRE1_RT).
// ---------------------------------------------------------------------------------------
template <typename T, bool RT>
__global__ void __launch_bounds__(kThreads) k_pre1_restrict(RBArgs<T> a, int nc,
                                                            const int* __restrict__ aggptr,
                                                            const int* __restrict__ members,
                                                            T* __restrict__ rc) {
    pdl_wait();
    pdl_trigger();
    if (a.skip && *(volatile const int*)a.skip) return;
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I >= nc) return;  // whole warps leave together
    T a1 = T(0);
    if constexpr (RT) a1 = sizeof(T) == 4 ? (T)a.rsc->a1f : (T)a.rsc->a1;
    auto rin = [&](int j) -> T {
        if constexpr (RT) return sub_rn(a.r[j], mul_rn(a1, a.d1[j]));
        else return a.r[j];
    };
    const int q0 = aggptr[I], q1 = aggptr[I + 1];
    T sum = T(0);
    for (int qb = q0; qb < q1; qb += 32) {
        const int q = qb + lane;
        T sj = T(0);
        if (q < q1) {
            const int j = members[q];
            const T rj = rin(j);
            const int k1 = a.rowptr[j + 1];
            T acc = T(0);
            for (int k = a.rowptr[j]; k < k1; k += 8) {
                int jj[8];
                T vv[8], xg[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const bool in = k + u < k1;
                    jj[u] = in ? a.col[k + u] : 0;
                    vv[u] = in ? a.val[k + u] : T(0);
                }
#pragma unroll
                for (int u = 0; u < 8; u++)
                    xg[u] = (k + u < k1) ? mul_rn(a.minv[jj[u]], rin(jj[u])) : T(0);
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (k + u < k1) acc = fma_rn(vv[u], xg[u], acc);
            }
            a.y[j] = mul_rn(a.minv[j], rj);
            if constexpr (RT) a.y3[j] = rj;
            sj = sub_rn(rj, acc);
        }
        const int cnt = min(32, q1 - qb);
        for (int u = 0; u < cnt; u++) {
            const T v = __shfl_sync(0xffffffffu, sj, u);
            if (lane == 0) sum = add_rn(sum, v);
        }
    }
    if (lane == 0) rc[I] = sum;
}

template <typename T>
int launch_pre1_restrict(Handle* h, int mode, const RBArgs<T>& a, int nc, const int* aggptr,
                         const int* members, T* rc) {
    const int grid = grid_for((long long)nc * 32, kThreads);
    cudaError_t e;
    if (mode == RB_PRE1_RT)
        e = launch_k(a.n <= kPdlMaxRows, k_pre1_restrict<T, true>, dim3(grid), dim3(kThreads), 0,
                     h->work, a, nc, aggptr, members, rc);
    else
        e = launch_k(a.n <= kPdlMaxRows, k_pre1_restrict<T, false>, dim3(grid), dim3(kThreads), 0,
                     h->work, a, nc, aggptr, members, rc);
    count_launch(h);
    return check_cuda(e);
}
template int launch_pre1_restrict<float>(Handle*, int, const RBArgs<float>&, int, const int*,
                                         const int*, float*);
template int launch_pre1_restrict<double>(Handle*, int, const RBArgs<double>&, int, const int*,
                                          const int*, double*);

// ---------------------------------------------------------------------------------------
// Coarsest solve: out = A_c^{-1} in with the precomputed dense inverse (warp per row, FP64).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_dense_apply(int n, const double* __restrict__ inv, const T* __restrict__ in,
              T* __restrict__ out, const int* skip) {
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += inv[(size_t)i * n + j] * (double)in[j];
    s = warp_sum(s);
    if (lane == 0) out[i] = (T)s;
}

template <typename T>
int launch_dense_apply(Handle* h, int n, const double* inv, const T* in, T* out,
                       const int* skip) {
    cudaError_t e = launch_k(true, k_dense_apply<T>, dim3(grid_for((long long)n * 32, kThreads)),
                             dim3(kThreads), 0, h->work, n, inv, in, out, skip);
    count_launch(h);
    return check_cuda(e);
}
template int launch_dense_apply<float>(Handle*, int, const double*, const float*, float*, const int*);
template int launch_dense_apply<double>(Handle*, int, const double*, const double*, double*, const int*);

// ---------------------------------------------------------------------------------------
// K-cycle scalar steps (Section 4.3, two flexible-CG steps):
//   step 1: rho~ = rho - (alpha1 / rho1) v1; the second step is skipped when rho1 <= 0,
//           when only one step is configured, or when |rho~| <= tau |rho| (tau > 0).
//   combine: e = (alpha1/rho1 - gamma alpha2 / (rho1 rho2)) c1 + (alpha2 / rho2) c2 with
//           rho2 = beta - gamma^2 / rho1, falling back to (alpha1/rho1) c1 when the second
//           step was skipped or rho2 <= 0, and to 0 when rho1 <= 0.
// Ctrl::skip = level+1 while the kernels of a skipped second step must return at once.
// ---------------------------------------------------------------------------------------
template <typename T, bool TAU>
__global__ void __launch_bounds__(kThreads)
k_kc_rt(int level, int n, const T* __restrict__ rho, const T* __restrict__ v1, T* __restrict__ rt,
        LevelScalars* sc, int inner, double tau, Ctrl* ctrl, double* partials) {
    pdl_wait();
    pdl_trigger();
    if (*(volatile const int*)&ctrl->skip) return;
    const bool ok = sc->rho1 > 0.0;
    const T a1t = (T)sc->a1;  // alpha1 / rho1, set by the first SpMV's last block
    double dv[2] = {0.0, 0.0};
    const int gs = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        const T v = sub_rn(rho[i], mul_rn(a1t, v1[i]));
        rt[i] = v;
        if constexpr (TAU) {
            dv[0] += (double)v * (double)v;
            dv[1] += (double)rho[i] * (double)rho[i];
        }
    }
    if constexpr (TAU) grid_reduce<2>(dv, partials, &ctrl->red_count, &sc->rtrt);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int skip2 = (!ok || inner < 2) ? 1 : 0;
        sc->skip2 = skip2;
        if (skip2) ctrl->skip = level + 1;
    }
}

// The tau test needs the complete norms, so it runs as its own one-block step.
__global__ void k_kc_tau(int level, LevelScalars* sc, double tau, Ctrl* ctrl) {
    if (*(volatile const int*)&ctrl->skip) return;
    if (threadIdx.x == 0 && !sc->skip2) {
        if (sqrt(sc->rtrt) <= tau * sqrt(sc->rhorho)) {
            sc->skip2 = 1;
            ctrl->skip = level + 1;
        }
    }
}

template <typename T>
int launch_kc_rt(Handle* h, int level, int n, const T* rho, const T* v1, T* rt,
                 LevelScalars* sc, int inner, double tau, Ctrl* ctrl) {
    int grid = grid_for(n, kThreads);
    if (grid > 4 * h->num_sms) grid = 4 * h->num_sms;
    if (tau > 0.0 && inner >= 2) {
        k_kc_rt<T, true><<<grid, kThreads, 0, h->work>>>(level, n, rho, v1, rt, sc, inner, tau, ctrl, h->partials);
        k_kc_tau<<<1, 32, 0, h->work>>>(level, sc, tau, ctrl);
        count_launch(h, 2);
    } else {
        cudaError_t e = launch_k(n <= kPdlMaxRows, k_kc_rt<T, false>, dim3(grid), dim3(kThreads),
                                 0, h->work, level, n, rho, v1, rt, sc, inner, tau, ctrl,
                                 h->partials);
        count_launch(h);
        if (e != cudaSuccess) return check_cuda(e);
    }
    return check_cuda(cudaGetLastError());
}
template int launch_kc_rt<float>(Handle*, int, int, const float*, const float*, float*, LevelScalars*, int, double, Ctrl*);
template int launch_kc_rt<double>(Handle*, int, int, const double*, const double*, double*, LevelScalars*, int, double, Ctrl*);

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_kc_combine(int level, int n, const T* __restrict__ c1, const T* __restrict__ c2,
             T* __restrict__ e, const LevelScalars* sc, Ctrl* ctrl) {
    pdl_wait();
    pdl_trigger();
    const int sk = *(volatile const int*)&ctrl->skip;
    if (sk != 0 && sk != level + 1) return;  // inside an ancestor's skipped step
    const double w1 = sc->w1, w2 = sc->w2;    // set by the step SpMVs' last blocks
    const T w1t = (T)w1, w2t = (T)w2;
    const bool two = (w2 != 0.0);
    const int gs = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        T v = mul_rn(w1t, c1[i]);
        if (two) v = add_rn(v, mul_rn(w2t, c2[i]));
        e[i] = v;
    }
    if (sk == level + 1 && blockIdx.x == 0 && threadIdx.x == 0) ctrl->skip = 0;
}

template <typename T>
int launch_kc_combine(Handle* h, int level, int n, const T* c1, const T* c2, T* e,
                      const LevelScalars* sc, Ctrl* ctrl) {
    int grid = grid_for(n, kThreads);
    if (grid > 8 * h->num_sms) grid = 8 * h->num_sms;
    cudaError_t err = launch_k(n <= kPdlMaxRows, k_kc_combine<T>, dim3(grid), dim3(kThreads), 0,
                               h->work, level, n, c1, c2, e, sc, ctrl);
    count_launch(h);
    return check_cuda(err);
}
template int launch_kc_combine<float>(Handle*, int, int, const float*, const float*, float*, const LevelScalars*, Ctrl*);
template int launch_kc_combine<double>(Handle*, int, int, const double*, const double*, double*, const LevelScalars*, Ctrl*);

// Prolongation alone (Section 4.2): y_i = x_i + e_{agg[i]} (x = null: zero).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_prolong(int n, const T* __restrict__ x, const int* __restrict__ agg, const T* __restrict__ e,
          T* __restrict__ y, const int* skip) {
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x ? add_rn(x[i], e[agg[i]]) : e[agg[i]];
}

template <typename T>
int launch_prolong(Handle* h, int n, const T* x, const int* agg, const T* e, T* y,
                   const int* skip) {
    cudaError_t err = launch_k(n <= kPdlMaxRows, k_prolong<T>, dim3(grid_for(n, kThreads)),
                               dim3(kThreads), 0, h->work, n, x, agg, e, y, skip);
    count_launch(h);
    return check_cuda(err);
}
template int launch_prolong<float>(Handle*, int, const float*, const int*, const float*, float*, const int*);
template int launch_prolong<double>(Handle*, int, const double*, const int*, const double*, double*, const int*);

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_copy(int n, const T* __restrict__ in, T* __restrict__ out, const int* skip) {
    if (skip && *(volatile const int*)skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in ? in[i] : T(0);
}

template <typename T>
int launch_copy(Handle* h, int n, const T* in, T* out, const int* skip) {
    k_copy<T><<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, in, out, skip);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template int launch_copy<float>(Handle*, int, const float*, float*, const int*);
template int launch_copy<double>(Handle*, int, const double*, double*, const int*);

// ---------------------------------------------------------------------------------------
// Outer flexible CG (FP64): p = z - ((z, q_prev) / (p_prev, q_prev)) p_prev, q = A p,
// alpha = (p, r) / (p, q), x += alpha p, r -= alpha q.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_cast_d2f(int n, const double* __restrict__ in, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __double2float_rn(in[i]);
}

int launch_cast_d2f(Handle* h, int n, const double* in, float* out) {
    k_cast_d2f<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, in, out);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// result = (a, b).  With osc: result is (z, q) of the outer iteration, and the last block
// also derives beta = (z, q) / (p, q)_prev once for the direction update.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kThreads)
k_dot(int n, const TA* __restrict__ a, const TB* __restrict__ b, double* partials,
      unsigned int* counter, double* result, OuterScalars* osc) {
    double dv[1] = {0.0};
    const int gs = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs)
        dv[0] = fma((double)a[i], (double)b[i], dv[0]);
    if (grid_reduce<1>(dv, partials, counter, result) && osc)
        osc->beta_cur = osc->first ? 0.0 : result[0] / osc->pq_prev;
}

static int dot_grid(Handle* h, int n) {
    int g = grid_for(n, kThreads);
    return g > 4 * h->num_sms ? 4 * h->num_sms : g;
}

int launch_dot(Handle* h, int n, const double* a, const double* b, double* result) {
    k_dot<double, double><<<dot_grid(h, n), kThreads, 0, h->work>>>(n, a, b, h->partials, &h->ctrl->red_count, result, nullptr);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

template <typename T>
int launch_outer_zq(Handle* h, int n, const T* z, const double* q, OuterScalars* osc) {
    k_dot<T, double><<<dot_grid(h, n), kThreads, 0, h->work>>>(n, z, q, h->partials, &h->ctrl->red_count, &osc->zq, osc);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template int launch_outer_zq<float>(Handle*, int, const float*, const double*, OuterScalars*);
template int launch_outer_zq<double>(Handle*, int, const double*, const double*, OuterScalars*);

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_outer_p(int n, const T* __restrict__ z, double* __restrict__ p, const OuterScalars* osc) {
    const double beta = osc->beta_cur;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = fma(-beta, p[i], (double)z[i]);
}

template <typename T>
int launch_outer_p(Handle* h, int n, const T* z, double* p, OuterScalars* osc) {
    k_outer_p<T><<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, z, p, osc);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template int launch_outer_p<float>(Handle*, int, const float*, double*, OuterScalars*);
template int launch_outer_p<double>(Handle*, int, const double*, double*, OuterScalars*);

__global__ void __launch_bounds__(kThreads)
k_outer_xr(int n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
           const double* __restrict__ q, OuterScalars* osc, double* partials,
           unsigned int* counter) {
    const double pq = osc->pq;
    const bool ok = pq > 0.0;
    const double alpha = osc->alpha_cur;  // set by the outer SpMV's last block
    double dv[1] = {0.0};
    const int gs = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        dv[0] = fma(ri, ri, dv[0]);
    }
    grid_reduce<1>(dv, partials, counter, &osc->rr);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // fields read only by the next iteration's kernels
        osc->alpha = alpha;
        osc->pq_prev = pq;
        osc->first = 0;
        if (!ok) osc->breakdown = 1;
    }
}

int launch_outer_xr(Handle* h, int n, double* x, double* r, const double* p, const double* q,
                    OuterScalars* osc) {
    k_outer_xr<<<dot_grid(h, n), kThreads, 0, h->work>>>(n, x, r, p, q, osc, h->partials, &h->ctrl->red_count);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// End of one iteration of the device-side loop (one thread): count it, record the relative
// residual, and decide whether the loop's body runs again.
__global__ void k_outer_loop(OuterScalars* osc, double* hist, int hist_cap,
                             cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = ++osc->it;
    if (k < hist_cap) hist[k] = sqrt(osc->rr / osc->bb);
    const bool more = !osc->breakdown && osc->rr > osc->stop_rr && k < osc->it_limit;
    cudaGraphSetConditional(cond, more ? 1u : 0u);
}

int launch_outer_loop(Handle* h, cudaGraphConditionalHandle cond) {
    k_outer_loop<<<1, 32, 0, h->work>>>(h->osc, h->d_hist, h->hist_cap, cond);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

int launch_to_host_scalars(Handle* h) {
    return check_cuda(cudaMemcpyAsync(h->osc_host, h->osc, sizeof(OuterScalars),
                                      cudaMemcpyDeviceToHost, h->work));
}

}  // namespace uaamg
