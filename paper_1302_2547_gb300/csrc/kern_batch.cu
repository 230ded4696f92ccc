// kern_batch.cu -- kernels of uaamg_solve_batch: one launch per K-cycle step for every
// participating system (batch.cuh describes the tiling and the descriptors).
//
// Inside a tile the arithmetic is that of the R-column kernels of uaamg_solve_many: thread
// (row, column) walks its row once in stored order with fused multiply-adds, the R threads
// of a row read each matrix entry once for all columns, and every column has its own
// K-cycle and outer scalars.  The smoother (Section 4.1) is fused into the SpMV (Section
// 4.4), restriction sums the members of each aggregate in ascending order and
// prolongation adds the coarse value of the row's aggregate (Section 4.2).
#include "batch.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kBGather = 8;  // row entries whose loads a thread issues together

// The tile of this block (one 16-byte load of the launch's table): its system, the tile's
// index within the system and the system's tile count at this launch.
struct BTile {
    int sys, tile, ntiles, part0;
    const BLevel* L;
};

__device__ __forceinline__ bool b_enter(const BArgs& a, BTile& t) {
    const int4 ti = __ldg(a.tinfo + blockIdx.x);
    t.sys = ti.x;
    t.tile = ti.y;
    t.ntiles = ti.z;
    t.part0 = ti.w;
    t.L = a.lev + (size_t)t.sys * kMaxLevels + a.level;
    return a.active[t.sys] != 0;
}

// Per-system, per-column reduction of ND values of every thread: a fixed tree over the
// tile's rows, the tile's partial stored, and the last of the system's tiles to arrive adds
// the tiles' partials in tile order (slices of tiles, then the slices in order) and writes
// result[k * R + c].  Returns true in every thread of that last block, after the result is
// written.  All threads of the block must call it.
template <int ND>
__device__ __forceinline__ bool b_reduce(const double (&v)[ND], int lg, int R, const BTile& t,
                                         double* part, unsigned int* counter, double* result) {
    __shared__ double sh[ND][kThreads];
    __shared__ double sl[kThreads];
    __shared__ bool is_last;
    const int th = threadIdx.x;
#pragma unroll
    for (int k = 0; k < ND; k++) sh[k][th] = v[k];
    __syncthreads();
    for (int s = (kThreads >> lg) >> 1; s > 0; s >>= 1) {
        if ((th >> lg) < s) {
#pragma unroll
            for (int k = 0; k < ND; k++) sh[k][th] += sh[k][th + (s << lg)];
        }
        __syncthreads();
    }
    if (th < R) {
#pragma unroll
        for (int k = 0; k < ND; k++)
            part[((size_t)t.tile * ND + k) * kBPartStride + th] = sh[k][th];
    }
    __threadfence();
    __syncthreads();
    if (th == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)t.ntiles - 1u);
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    const int np = ND * R;
    const int slices = kThreads / np;
    double acc = 0.0;
    if (th < slices * np) {
        const int pair = th % np, slice = th / np;
        const int k = pair / R, c = pair % R;
        for (int b = slice; b < t.ntiles; b += slices)
            acc += __ldcg(&part[((size_t)b * ND + k) * kBPartStride + c]);
    }
    sl[th] = acc;
    __syncthreads();
    if (th < np) {
        double s = 0.0;
        for (int q = 0; q < slices; q++) s += sl[q * np + th];
        result[th] = s;
    }
    if (th == 0) *counter = 0u;
    __syncthreads();
    return true;
}

template <int ND>
__device__ __forceinline__ double* b_part(const BArgs& a, const BTile& t) {
    return a.partials + (size_t)t.part0 * ND * kBPartStride;
}
__device__ __forceinline__ double* b_os(const BArgs& a, const BTile& t) {
    return a.lev[(size_t)t.sys * kMaxLevels].os;
}

template <typename T>
__device__ __forceinline__ T* b_vec(const BLevel& L, int slot) {
    return slot >= 0 ? static_cast<T*>(L.v[slot]) : nullptr;
}

// Row range of this tile over `rows` rows, and this thread's column.
struct BRows {
    int lg, R, rpb, lr, r0, r1;
};
__device__ __forceinline__ BRows b_rows(const BTile& t, int rows, int R) {
    BRows g;
    g.lg = b_lg(R);
    g.R = R;
    g.rpb = kThreads >> g.lg;
    g.lr = threadIdx.x & ((1 << g.lg) - 1);
    const int tr = b_tile_rows(rows, R);
    g.r0 = t.tile * tr;
    g.r1 = min(rows, g.r0 + tr);
    return g;
}

// SpMV-based row kernels (modes of kernels.cuh): RB_PRE1, RB_PROSMOOTH, RB_SPMV with 2 or 3
// inner products, RB_RESID with (y, y).
template <typename T, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) kb_row(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const int R = g.R, lr = g.lr;
    const T* __restrict__ val = a.outer ? reinterpret_cast<const T*>(L.val64)
                                        : static_cast<const T*>(L.val);
    const T* __restrict__ minv = static_cast<const T*>(L.minv);
    const int* __restrict__ rowptr = L.rowptr;
    const int* __restrict__ col = L.col;
    const T* r = b_vec<T>(L, a.s_r);
    const T* x = b_vec<T>(L, a.s_x);
    T* y = b_vec<T>(L, a.s_y);
    T* y2 = b_vec<T>(L, a.s_y2);
    const T* d1 = b_vec<T>(L, a.s_d1);
    const T* d2 = b_vec<T>(L, a.s_d2);
    const int* agg = L.agg;
    const T* e = nullptr;
    if constexpr (MODE == RB_PROSMOOTH) e = b_vec<T>(t.L[1], a.s_e);
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        T acc = T(0);
        const int k1 = rowptr[i + 1];
        // kBGather entries at a time: their columns and values, then their vector entries,
        // are loaded before the first is used; the sum keeps the stored order
        for (int k = rowptr[i]; k < k1; k += kBGather) {
            int jj[kBGather];
            T vv[kBGather], xg[kBGather];
#pragma unroll
            for (int u = 0; u < kBGather; u++) {
                const bool in = k + u < k1;
                jj[u] = in ? col[k + u] : 0;
                vv[u] = in ? val[k + u] : T(0);
            }
#pragma unroll
            for (int u = 0; u < kBGather; u++) {
                const size_t oj = (size_t)jj[u] * R + lr;
                T xj = T(0);
                if (k + u < k1) {
                    if constexpr (MODE == RB_PRE1) xj = mul_rn(minv[jj[u]], r[oj]);
                    else if constexpr (MODE == RB_PROSMOOTH)
                        xj = add_rn(x[oj], e[(size_t)agg[jj[u]] * R + lr]);
                    else xj = x[oj];
                }
                xg[u] = xj;
            }
#pragma unroll
            for (int u = 0; u < kBGather; u++)
                if (k + u < k1) acc = fma_rn(vv[u], xg[u], acc);
        }
        if constexpr (MODE == RB_PRE1) {
            y[o] = mul_rn(minv[i], r[o]);
            y2[o] = sub_rn(r[o], acc);
        } else if constexpr (MODE == RB_RESID) {
            const T yi = sub_rn(r[o], acc);
            y[o] = yi;
            if constexpr (ND >= 1) dv[0] = fma((double)yi, (double)yi, dv[0]);
        } else if constexpr (MODE == RB_PROSMOOTH) {
            const T xi = add_rn(x[o], e[(size_t)agg[i] * R + lr]);
            y[o] = add_rn(xi, mul_rn(minv[i], sub_rn(r[o], acc)));
        } else {  // RB_SPMV
            y[o] = acc;
            const double xi = (double)x[o];
            if constexpr (ND >= 1) dv[0] = fma(xi, (double)acc, dv[0]);
            if constexpr (ND >= 2) dv[1] = fma(xi, (double)d1[o], dv[1]);
            if constexpr (ND >= 3) dv[2] = fma(xi, (double)d2[o], dv[2]);
        }
    }
    if constexpr (ND > 0) {
        double* res = (a.res_os ? b_os(a, t) : L.sc) + (size_t)a.res_row * R;
        b_reduce<ND>(dv, g.lg, R, t, b_part<ND>(a, t), a.counters + t.sys, res);
    }
}

// r_c = P^T s: thread (aggregate, column) adds the members' entries in ascending order, the
// loads of eight members issued before the first add.
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_restrict(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.nc, L.R);
    const int R = g.R, lr = g.lr;
    const T* __restrict__ s = static_cast<const T*>(L.v[BS_S]);
    T* __restrict__ rc = static_cast<T*>(t.L[1].v[BS_RHS]);
    const int* __restrict__ aggptr = L.aggptr;
    const int* __restrict__ members = L.members;
    for (int I = g.r0 + (int)(threadIdx.x >> g.lg); I < g.r1; I += g.rpb) {
        if (lr >= R) continue;
        const int q1 = aggptr[I + 1];
        T sum = T(0);
        for (int q = aggptr[I]; q < q1; q += 8) {
            int m[8];
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) m[u] = q + u < q1 ? members[q + u] : 0;
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = q + u < q1 ? s[(size_t)m[u] * R + lr] : T(0);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (q + u < q1) sum = add_rn(sum, v[u]);
        }
        rc[(size_t)I * R + lr] = sum;
    }
}

// Exact solve on the system's coarsest level with its dense FP64 inverse: one block per row
// i; the block's threads split the columns j into chunks for each right-hand side, and the
// chunks' sums are added in chunk order.
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_dense(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    __shared__ double part[kThreads];
    const BLevel& L = *t.L;
    const int n = L.n, R = L.R, lg = b_lg(R);
    const int i = t.tile;
    const int r = threadIdx.x & ((1 << lg) - 1);
    const int jc = threadIdx.x >> lg;
    const int nch = kThreads >> lg;
    const T* __restrict__ in = b_vec<T>(L, a.s_r);
    T* __restrict__ out = b_vec<T>(L, a.s_y);
    const double* __restrict__ inv = L.inv;
    double s = 0.0;
    if (r < R)
        for (int j = jc; j < n; j += nch) s = fma(inv[(size_t)i * n + j], (double)in[(size_t)j * R + r], s);
    part[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < R) {
        double acc = 0.0;
        for (int c = 0; c < nch; c++) acc += part[(c << lg) + threadIdx.x];
        out[(size_t)i * R + threadIdx.x] = (T)acc;
    }
}

// rho~ = rho - (alpha1 / rho1) v1 per column (Section 4.3), with |rho~|^2 and |rho|^2 when
// the system's tau > 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_kc_rt(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const int R = g.R, lr = g.lr;
    __shared__ double sa1[kBMaxR];
    if ((int)threadIdx.x < R) {
        const double rho1 = L.sc[threadIdx.x], alpha1 = L.sc[R + threadIdx.x];
        sa1[threadIdx.x] = rho1 > 0.0 ? alpha1 / rho1 : 0.0;
    }
    __syncthreads();
    const T a1 = (T)(lr < R ? sa1[lr] : 0.0);
    const T* __restrict__ rho = b_vec<T>(L, a.s_r);
    const T* __restrict__ v1 = static_cast<const T*>(L.v[BS_V1]);
    T* __restrict__ rt = static_cast<T*>(L.v[BS_RT]);
    const bool tau = L.tau > 0.0;
    double dv[2] = {0.0, 0.0};
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        const T v = sub_rn(rho[o], mul_rn(a1, v1[o]));
        rt[o] = v;
        if (tau) {
            dv[0] = fma((double)v, (double)v, dv[0]);
            dv[1] = fma((double)rho[o], (double)rho[o], dv[1]);
        }
    }
    if (tau) b_reduce<2>(dv, g.lg, R, t, b_part<2>(a, t), a.counters + t.sys, L.sc + 5 * R);
}

// e = w1 c1 + w2 c2 per column with the Section 4.3 guards: w = 0 when rho1 <= 0; the
// second step counts only when the level takes it (and, with tau, when |rho~| > tau |rho|)
// and rho2 = beta - gamma^2 / rho1 > 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_combine(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const int R = g.R, lr = g.lr;
    __shared__ double sw[2][kBMaxR];
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        const double* sc = L.sc;
        const double rho1 = sc[c], alpha1 = sc[R + c];
        double w1 = 0.0, w2 = 0.0;
        if (rho1 > 0.0) {
            w1 = alpha1 / rho1;
            bool two = L.inner >= 2;
            if (two && L.tau > 0.0 && sqrt(sc[5 * R + c]) <= L.tau * sqrt(sc[6 * R + c]))
                two = false;
            if (two) {
                const double beta = sc[2 * R + c], gamma = sc[3 * R + c], alpha2 = sc[4 * R + c];
                const double rho2 = beta - gamma * gamma / rho1;
                if (rho2 > 0.0) {
                    w1 = w1 - gamma * alpha2 / (rho1 * rho2);
                    w2 = alpha2 / rho2;
                }
            }
        }
        sw[0][c] = w1;
        sw[1][c] = w2;
    }
    __syncthreads();
    const T* __restrict__ c1 = static_cast<const T*>(L.v[BS_C1]);
    const T* __restrict__ c2 = static_cast<const T*>(L.v[BS_C2]);
    T* __restrict__ e = b_vec<T>(L, a.s_y);
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (lr >= R) continue;
        const double w1 = sw[0][lr], w2 = sw[1][lr];
        const size_t o = (size_t)i * R + lr;
        T v = mul_rn((T)w1, c1[o]);
        if (w2 != 0.0) v = add_rn(v, mul_rn((T)w2, c2[o]));
        e[o] = v;
    }
}

// ---- outer flexible CG per column (FP64; Sections 1 and 4.4) ----------------------------
// os rows (as uaamg_solve_many): 0 pq, 1 pr, 2 zq, 3 rr, 4 bb, 5 pq_prev, 6 active column,
// 7 first direction.

// The FP64 residual rounded to the cycle's precision (the cycle's right-hand side).
__global__ void __launch_bounds__(kThreads) kb_cast(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const double* __restrict__ r = static_cast<const double*>(L.v[BS_R]);
    float* __restrict__ f = static_cast<float*>(L.v[BS_RHS]);
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= g.R) continue;
        const size_t o = (size_t)i * g.R + g.lr;
        f[o] = __double2float_rn(r[o]);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb_zq(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const T* __restrict__ z = static_cast<const T*>(L.v[BS_OUT]);
    const double* __restrict__ q = static_cast<const double*>(L.v[BS_Q]);
    double dv[1] = {0.0};
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= g.R) continue;
        const size_t o = (size_t)i * g.R + g.lr;
        dv[0] = fma((double)z[o], q[o], dv[0]);
    }
    b_reduce<1>(dv, g.lg, g.R, t, b_part<1>(a, t), a.counters + t.sys, L.os + 2 * g.R);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb_p(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const int R = g.R;
    __shared__ double sb[kBMaxR];
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        const double* os = L.os;
        sb[c] = (os[7 * R + c] != 0.0) ? 0.0 : os[2 * R + c] / os[5 * R + c];
    }
    __syncthreads();
    const T* __restrict__ z = static_cast<const T*>(L.v[BS_OUT]);
    double* __restrict__ p = static_cast<double*>(L.v[BS_P]);
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= R) continue;
        const size_t o = (size_t)i * R + g.lr;
        p[o] = fma(-sb[g.lr], p[o], (double)z[o]);
    }
}

// x += alpha p, r -= alpha q and (r, r); the last tile of the system then advances the
// recurrence of its active columns (pq_prev = pq, first = 0).
__global__ void __launch_bounds__(kThreads) kb_xr(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const int R = g.R;
    double* os = L.os;
    __shared__ double sal[kBMaxR];
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        const double pq = os[c], active = os[6 * R + c];
        sal[c] = (active != 0.0 && pq > 0.0) ? os[R + c] / pq : 0.0;
    }
    __syncthreads();
    double* __restrict__ x = static_cast<double*>(L.v[BS_X]);
    double* __restrict__ r = static_cast<double*>(L.v[BS_R]);
    const double* __restrict__ p = static_cast<const double*>(L.v[BS_P]);
    const double* __restrict__ q = static_cast<const double*>(L.v[BS_Q]);
    double dv[1] = {0.0};
    const double alpha = g.lr < R ? sal[g.lr] : 0.0;
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= R) continue;
        const size_t o = (size_t)i * R + g.lr;
        x[o] = fma(alpha, p[o], x[o]);
        const double ri = fma(-alpha, q[o], r[o]);
        r[o] = ri;
        dv[0] = fma(ri, ri, dv[0]);
    }
    if (b_reduce<1>(dv, g.lg, R, t, b_part<1>(a, t), a.counters + t.sys, os + 3 * R)) {
        if ((int)threadIdx.x < R && os[6 * R + threadIdx.x] != 0.0) {
            os[5 * R + threadIdx.x] = os[threadIdx.x];
            os[7 * R + threadIdx.x] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) kb_norm(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    const double* __restrict__ b = static_cast<const double*>(L.v[BS_B]);
    double dv[1] = {0.0};
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= g.R) continue;
        const double v = b[(size_t)i * g.R + g.lr];
        dv[0] = fma(v, v, dv[0]);
    }
    b_reduce<1>(dv, g.lg, g.R, t, b_part<1>(a, t), a.counters + t.sys, L.os + 4 * g.R);
}

__global__ void __launch_bounds__(kThreads) kb_init(BArgs a) {
    pdl_wait();
    pdl_trigger();
    BTile t;
    if (!b_enter(a, t)) return;
    const BLevel& L = *t.L;
    const BRows g = b_rows(t, L.n, L.R);
    double* x = static_cast<double*>(L.v[BS_X]);
    double* p = static_cast<double*>(L.v[BS_P]);
    double* q = static_cast<double*>(L.v[BS_Q]);
    for (int i = g.r0 + (int)(threadIdx.x >> g.lg); i < g.r1; i += g.rpb) {
        if (g.lr >= g.R) continue;
        const size_t o = (size_t)i * g.R + g.lr;
        x[o] = 0.0;
        p[o] = 0.0;
        q[o] = 0.0;
    }
}

template <typename T>
int launch_batch(cudaStream_t st, int kind, int mode, int ndots, const BArgs& a, int tiles,
                 bool pdl) {
    if (tiles <= 0 || a.nseg <= 0) return UAAMG_OK;
    const dim3 grid(tiles), block(kThreads);
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
        case BK_ROW:
#define KB_ROW(M, D) \
    if (mode == M && ndots == D) e = launch_k(pdl, kb_row<T, M, D>, grid, block, 0, st, a);
            KB_ROW(RB_PRE1, 0)
            KB_ROW(RB_PROSMOOTH, 0)
            KB_ROW(RB_SPMV, 2)
            KB_ROW(RB_SPMV, 3)
            KB_ROW(RB_RESID, 1)
#undef KB_ROW
            break;
        case BK_RESTRICT: e = launch_k(pdl, kb_restrict<T>, grid, block, 0, st, a); break;
        case BK_DENSE: e = launch_k(pdl, kb_dense<T>, grid, block, 0, st, a); break;
        case BK_KC_RT: e = launch_k(pdl, kb_kc_rt<T>, grid, block, 0, st, a); break;
        case BK_COMBINE: e = launch_k(pdl, kb_combine<T>, grid, block, 0, st, a); break;
        case BK_CAST:
            if constexpr (sizeof(T) == 4) e = launch_k(pdl, kb_cast, grid, block, 0, st, a);
            break;
        case BK_ZQ: e = launch_k(pdl, kb_zq<T>, grid, block, 0, st, a); break;
        case BK_P: e = launch_k(pdl, kb_p<T>, grid, block, 0, st, a); break;
        case BK_XR: e = launch_k(pdl, kb_xr, grid, block, 0, st, a); break;
        case BK_NORM: e = launch_k(pdl, kb_norm, grid, block, 0, st, a); break;
        case BK_INIT: e = launch_k(pdl, kb_init, grid, block, 0, st, a); break;
        default: break;
    }
    return check_cuda(e);
}
template int launch_batch<float>(cudaStream_t, int, int, int, const BArgs&, int, bool);
template int launch_batch<double>(cudaStream_t, int, int, int, const BArgs&, int, bool);

}  // namespace uaamg
