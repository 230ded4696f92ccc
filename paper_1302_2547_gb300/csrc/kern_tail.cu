// kern_tail.cu -- the K-cycle of the small coarse levels in one kernel launch.
//
// Level m of the K-cycle (Section 4.3) is visited 2^(m-1) times per outer iteration (fewer
// with one-step levels), and on small levels every step is a sub-microsecond kernel, so the
// cycle becomes launch-bound.  From the first level with at most kTailMaxN unknowns down
// to the coarsest, this kernel runs the whole recursion K_m -> B_m -> K_{m+1} ... in one
// thread block of 512 threads: each step of the launched path (fused SpMV + l1-Jacobi
// sweeps, residual restriction, prolongation, the two flexible-CG steps and the exact
// coarsest solve) becomes a block-wide phase separated by __syncthreads, with the same
// arithmetic per entry and block-level fixed-order reductions for the inner products.
// Vectors stay in the levels' global buffers (L2-resident at these sizes).
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kTailThreads = 512;

// Block-wide fixed-order sum of ND values; every thread receives the totals.
template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND]) {
    __shared__ double sh[ND][kTailThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ND; k++) {
        double s = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; k++) {
        double s = 0.0;
        for (int w = 0; w < kTailThreads / 32; w++) s += sh[k][w];
        v[k] = s;
    }
    __syncthreads();
}

// The recursion K_m -> B_m -> K_{m+1} runs as an explicit stack of frames in shared memory
// (at most two frames per level), so the kernel needs no call stack.  Every thread reads
// the top frame, the block executes one phase of it, and thread 0 pushes or pops.
struct TailFrame {
    int kind;   // 0: K_m, 1: B_m
    int level;
    int phase;
    const void* in;
    void* out;
    double rho1, w1, w2;
};
constexpr int kTailMaxFrames = 2 * kMaxLevels;

constexpr int kTailBatch = 8;  // entries whose gathers a thread has in flight

// Row i's sum of val[k] g(col[k]) over its entries, in stored order, with the gathers of
// kTailBatch entries issued before the first is used.
template <typename T, typename G>
__device__ __forceinline__ T tail_row(const TailLevel& L, int i, G g) {
    const T* val = (const T*)L.val;
    const int k1 = L.rowptr[i + 1];
    T acc = T(0);
    for (int k = L.rowptr[i]; k < k1; k += kTailBatch) {
        T xg[kTailBatch], vv[kTailBatch];
#pragma unroll
        for (int u = 0; u < kTailBatch; u++) {
            const bool in = k + u < k1;
            xg[u] = in ? g(L.col[k + u]) : T(0);
            vv[u] = in ? val[k + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kTailBatch; u++)
            if (k + u < k1) acc = fma_rn(vv[u], xg[u], acc);
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void spmv_rows(const TailLevel& L, const T* x, T* y, int nd,
                                          const T* da, const T* db, double* d) {
    for (int i = threadIdx.x; i < L.n; i += kTailThreads) {
        const T acc = tail_row<T>(L, i, [&](int j) { return x[j]; });
        y[i] = acc;
        const double xi = (double)x[i];
        d[0] += xi * (double)acc;
        if (nd >= 2) d[1] += xi * (double)da[i];
        if (nd >= 3) d[2] += xi * (double)db[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
k_tail(const TailLevel* lv, int m0, int nlev, const double* inv, double tau, const int* skip) {
    if (skip && *(volatile const int*)skip) return;
    __shared__ TailFrame st[kTailMaxFrames];
    __shared__ int sp;
    __shared__ double s_w;  // a step scalar computed by thread 0
    __shared__ int s_flag;  // a step decision taken by thread 0
    if (threadIdx.x == 0) {
        st[0] = TailFrame{0, m0, 0, lv[m0].rhs, lv[m0].out, 0.0, 0.0, 0.0};
        sp = 1;
    }
    __syncthreads();
    while (true) {
        const int top = sp;
        if (top == 0) break;
        const TailFrame f = st[top - 1];
        __syncthreads();
        // the level's descriptor by value: its pointers stay in registers (through a
        // reference every store to a vector could alias them, so each use reloads them)
        const TailLevel L = lv[f.level];
        const T* in = (const T*)f.in;
        T* out = (T*)f.out;
        int push = 0, pop = 0, next_phase = f.phase;
        TailFrame child{};
        double rho1 = f.rho1, w1 = f.w1, w2 = f.w2;
        if (f.kind == 0) {  // ---- K_m: two flexible-CG steps preconditioned by B_m ----
            T *c1 = (T*)L.c1, *v1 = (T*)L.v1, *rt = (T*)L.rt, *c2 = (T*)L.c2, *v2 = (T*)L.v2;
            if (f.level == nlev - 1) {  // exact solve with the dense inverse, a warp per row
                const int lane = threadIdx.x & 31;
                for (int i = threadIdx.x >> 5; i < L.n; i += kTailThreads / 32) {
                    double sum = 0.0;
                    for (int j = lane; j < L.n; j += 32)
                        sum = fma(inv[(size_t)i * L.n + j], (double)in[j], sum);
                    sum = warp_sum(sum);
                    if (lane == 0) out[i] = (T)sum;
                }
                pop = 1;
            } else if (f.phase == 0) {  // c1 = B_m(rho)
                child = TailFrame{1, f.level, 0, in, c1, 0.0, 0.0, 0.0};
                push = 1;
                next_phase = 1;
            } else if (f.phase == 1) {  // v1 = A c1; rho1, alpha1; rho~
                double d[3] = {0.0, 0.0, 0.0};
                spmv_rows<T>(L, c1, v1, 2, in, nullptr, d);
                block_sum<3>(d);
                // the step's scalars in one thread, broadcast through shared memory
                if (threadIdx.x == 0) {
                    rho1 = d[0];
                    w1 = rho1 > 0.0 ? d[1] / rho1 : 0.0;
                    w2 = 0.0;
                    s_w = w1;
                    s_flag = (rho1 > 0.0 && L.inner >= 2) ? 1 : 0;
                }
                __syncthreads();
                bool second = s_flag != 0;
                if (second) {
                    const T a1t = (T)s_w;
                    double nr[2] = {0.0, 0.0};
                    for (int i = threadIdx.x; i < L.n; i += kTailThreads) {
                        const T v = sub_rn(in[i], mul_rn(a1t, v1[i]));
                        rt[i] = v;
                        nr[0] += (double)v * (double)v;
                        nr[1] += (double)in[i] * (double)in[i];
                    }
                    block_sum<2>(nr);
                    if (threadIdx.x == 0)
                        s_flag = (tau > 0.0 && sqrt(nr[0]) <= tau * sqrt(nr[1])) ? 0 : 1;
                    __syncthreads();
                    second = s_flag != 0;
                }
                if (second) {  // c2 = B_m(rho~)
                    child = TailFrame{1, f.level, 0, rt, c2, 0.0, 0.0, 0.0};
                    push = 1;
                    next_phase = 2;
                } else {
                    next_phase = 3;
                }
            } else if (f.phase == 2) {  // v2 = A c2; beta, gamma, alpha2
                double d[3] = {0.0, 0.0, 0.0};
                spmv_rows<T>(L, c2, v2, 3, v1, rt, d);
                block_sum<3>(d);
                if (threadIdx.x == 0) {  // only thread 0 keeps the frame's scalars
                    const double beta = d[0], gamma = d[1], alpha2 = d[2];
                    const double rho2 = beta - gamma * gamma / rho1;
                    if (rho2 > 0.0) {
                        w1 = w1 - gamma * alpha2 / (rho1 * rho2);
                        w2 = alpha2 / rho2;
                    }
                }
                next_phase = 3;
            } else {  // e = w1 c1 + w2 c2
                const T w1t = (T)w1, w2t = (T)w2;
                for (int i = threadIdx.x; i < L.n; i += kTailThreads) {
                    T v = mul_rn(w1t, c1[i]);
                    if (w2 != 0.0) v = add_rn(v, mul_rn(w2t, c2[i]));
                    out[i] = v;
                }
                pop = 1;
            }
        } else {  // ---- B_l: pre-sweep, restriction, K_{l+1}, prolongation + post-sweep ----
            const TailLevel C = lv[f.level + 1];
            const T* minv = (const T*)L.minv;
            T* x = (T*)L.w;
            T* s = (T*)L.s;
            T* rc = (T*)C.rhs;
            T* ec = (T*)C.out;
            if (f.phase == 0) {
                for (int i = threadIdx.x; i < L.n; i += kTailThreads) {
                    const T acc = tail_row<T>(L, i, [&](int j) { return mul_rn(minv[j], in[j]); });
                    x[i] = mul_rn(minv[i], in[i]);
                    s[i] = sub_rn(in[i], acc);
                }
                __syncthreads();
                for (int I = threadIdx.x; I < C.n; I += kTailThreads) {
                    const int q1 = L.aggptr[I + 1];
                    T sum = T(0);
                    for (int q = L.aggptr[I]; q < q1; q += kTailBatch) {
                        T sv[kTailBatch];
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++)
                            sv[u] = q + u < q1 ? s[L.members[q + u]] : T(0);
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++)
                            if (q + u < q1) sum = add_rn(sum, sv[u]);
                    }
                    rc[I] = sum;
                }
                child = TailFrame{0, f.level + 1, 0, rc, ec, 0.0, 0.0, 0.0};
                push = 1;
                next_phase = 1;
            } else {
                for (int i = threadIdx.x; i < L.n; i += kTailThreads) {
                    const T acc = tail_row<T>(L, i, [&](int j) { return add_rn(x[j], ec[L.agg[j]]); });
                    const T xi = add_rn(x[i], ec[L.agg[i]]);
                    out[i] = add_rn(xi, mul_rn(minv[i], sub_rn(in[i], acc)));
                }
                pop = 1;
            }
        }
        __syncthreads();  // this phase's global writes are visible to the whole block
        if (threadIdx.x == 0) {
            if (pop) {
                sp = top - 1;
            } else {
                st[top - 1].phase = next_phase;
                st[top - 1].rho1 = rho1;
                st[top - 1].w1 = w1;
                st[top - 1].w2 = w2;
                if (push) {
                    st[top] = child;
                    sp = top + 1;
                }
            }
        }
        __syncthreads();
    }
}

// ---- the same recursion on one thread-block cluster -------------------------------------
// Levels up to cluster_below unknowns: the recursion runs on a cluster of kClusterCtas
// blocks (one GPC), every block executing the same phase sequence on its share of the rows
// (row i goes to thread i mod (blocks x threads)).  A phase ends with a cluster barrier
// (release / acquire at cluster scope), so the next phase sees every block's writes;
// vectors written inside the kernel are read through L2.  Inner products: each block sums
// its rows in a fixed tree, publishes the partials in its shared memory, and after a
// cluster barrier every block adds the blocks' partials in rank order from distributed
// shared memory, so all blocks hold the same totals and take the same branches (the frame
// stack is replicated per block).  The coarsest solve gives one warp per row across the
// cluster.
}  // namespace uaamg
#include <cooperative_groups.h>
namespace uaamg {
namespace cg = cooperative_groups;

constexpr int kClusterThreads = 512;

template <typename T>
__device__ __forceinline__ T ldg_cg(const T* p) {
    return __ldcg(p);
}

// Cluster-wide fixed-order sum of ND values; every thread of every block receives the
// totals.  `slot` alternates between two partial buffers, so a block that runs ahead cannot
// overwrite partials another block is still reading.  One warp per block fetches the
// blocks' partials from distributed shared memory (lane r reads block r's, all loads in
// flight together) and adds them in rank order.
template <int ND>
__device__ __forceinline__ void cluster_sum(double (&v)[ND], double (*part)[3], int slot) {
    __shared__ double sh[ND][kClusterThreads / 32];
    __shared__ double tot[ND];
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ND; k++) {
        double s = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
            double s = 0.0;
            for (int w = 0; w < kClusterThreads / 32; w++) s += sh[k][w];
            part[slot][k] = s;
        }
    }
    cl.sync();
    if (wid == 0) {
        const int nb = (int)cl.num_blocks();
        double pv[ND];
#pragma unroll
        for (int k = 0; k < ND; k++)
            pv[k] = lane < nb ? cl.map_shared_rank(&part[slot][0], lane)[k] : 0.0;
#pragma unroll
        for (int k = 0; k < ND; k++) {
            double s = 0.0;
            for (int r = 0; r < nb; r++) s += __shfl_sync(0xffffffffu, pv[k], r);
            if (lane == 0) tot[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; k++) v[k] = tot[k];
}

// Every row of level L, 1 to 8 lanes per row by its mean row length: the lanes of a row take
// its entries in turn
// (each lane's own entries in stored order, eight loads in flight), combine their sums by a
// fixed shuffle tree, and the row's first lane calls epi(i, sum).  The loop is uniform over
// each warp (whole warps of rows), so the shuffles see every lane.  gw / nw: this warp's
// index and the warps of the cluster.
template <typename T, typename G, typename E>
__device__ __forceinline__ void cl_rows(const TailLevel& L, int gw, int nw, G g, E epi) {
    // a few entries per lane, so that one batch of gathers covers a row
    const int avg = L.rowptr[L.n] / (L.n > 0 ? L.n : 1);
    const int lpr = avg < 6 ? 1 : avg < 12 ? 2 : avg < 24 ? 4 : 8;
    const int lane = threadIdx.x & 31, sub = lane & (lpr - 1);
    const int rpw = 32 / lpr;
    const T* val = (const T*)L.val;
    for (int base = gw * rpw; base < L.n; base += nw * rpw) {
        const int i = base + lane / lpr;
        T acc = T(0);
        if (i < L.n) {
            const int k1 = L.rowptr[i + 1];
            for (int k = L.rowptr[i] + sub; k < k1; k += kTailBatch * lpr) {
                T xg[kTailBatch], vv[kTailBatch];
#pragma unroll
                for (int u = 0; u < kTailBatch; u++) {
                    const int kk = k + u * lpr;
                    const bool in = kk < k1;
                    xg[u] = in ? g(L.col[kk]) : T(0);
                    vv[u] = in ? val[kk] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kTailBatch; u++)
                    if (k + u * lpr < k1) acc = fma_rn(vv[u], xg[u], acc);
            }
        }
        for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lpr);
        if (i < L.n && sub == 0) epi(i, acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads, 1)
k_tail_cluster(const TailLevel* lv, int m0, int nlev, const double* inv, double tau,
               const int* skip) {
    if (skip && *(volatile const int*)skip) return;  // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    __shared__ TailFrame st[kTailMaxFrames];
    __shared__ int sp;
    __shared__ double part[2][3];  // this block's inner-product partials (two slots)
    __shared__ double s_w;         // a step scalar computed by thread 0
    __shared__ int s_flag;         // a step decision taken by thread 0
    int slot = 0;
    const int G = (int)cl.num_blocks() * kClusterThreads;
    const int g0 = (int)cl.block_rank() * kClusterThreads + threadIdx.x;
    const int nw = G >> 5, gw = g0 >> 5;  // warps of the cluster, this warp's index
    if (threadIdx.x == 0) {
        st[0] = TailFrame{0, m0, 0, lv[m0].rhs, lv[m0].out, 0.0, 0.0, 0.0};
        sp = 1;
    }
    __syncthreads();
    while (true) {
        const int top = sp;
        if (top == 0) break;
        const TailFrame f = st[top - 1];
        __syncthreads();
        // the level's descriptor by value: its pointers stay in registers (through a
        // reference every store to a vector could alias them, so each use reloads them)
        const TailLevel L = lv[f.level];
        const T* in = (const T*)f.in;
        T* out = (T*)f.out;
        int push = 0, pop = 0, next_phase = f.phase;
        TailFrame child{};
        double rho1 = f.rho1, w1 = f.w1, w2 = f.w2;
        if (f.kind == 0) {  // ---- K_m: two flexible-CG steps preconditioned by B_m ----
            T *c1 = (T*)L.c1, *v1 = (T*)L.v1, *rt = (T*)L.rt, *c2 = (T*)L.c2, *v2 = (T*)L.v2;
            if (f.level == nlev - 1) {  // exact solve with the dense inverse, a warp per row
                const int lane = threadIdx.x & 31;
                for (int i = g0 >> 5; i < L.n; i += G >> 5) {
                    double sum = 0.0;
                    for (int j = lane; j < L.n; j += 32)
                        sum = fma(inv[(size_t)i * L.n + j], (double)ldg_cg(in + j), sum);
                    sum = warp_sum(sum);
                    if (lane == 0) out[i] = (T)sum;
                }
                pop = 1;
            } else if (f.phase == 0) {  // c1 = B_m(rho)
                child = TailFrame{1, f.level, 0, in, c1, 0.0, 0.0, 0.0};
                push = 1;
                next_phase = 1;
            } else if (f.phase == 1) {  // v1 = A c1; rho1, alpha1; rho~
                double d[3] = {0.0, 0.0, 0.0};
                cl_rows<T>(
                    L, gw, nw, [&](int j) { return ldg_cg(c1 + j); },
                    [&](int i, T acc) {
                        v1[i] = acc;
                        const double xi = (double)ldg_cg(c1 + i);
                        d[0] = fma(xi, (double)acc, d[0]);
                        d[1] = fma(xi, (double)ldg_cg(in + i), d[1]);
                    });
                cluster_sum<3>(d, part, slot);
                slot ^= 1;
                // the step's scalars in one thread (FP64 divisions are costly on GB300's
                // FP64 units when every thread repeats them), broadcast through shared memory
                if (threadIdx.x == 0) {
                    rho1 = d[0];
                    w1 = rho1 > 0.0 ? d[1] / rho1 : 0.0;
                    w2 = 0.0;
                    s_w = w1;
                    s_flag = (rho1 > 0.0 && L.inner >= 2) ? 1 : 0;
                }
                __syncthreads();
                bool second = s_flag != 0;
                if (second) {
                    const T a1t = (T)s_w;
                    double nr[2] = {0.0, 0.0};
                    for (int i = g0; i < L.n; i += G) {
                        const T v = sub_rn(ldg_cg(in + i), mul_rn(a1t, v1[i]));
                        rt[i] = v;
                        nr[0] += (double)v * (double)v;
                        nr[1] += (double)ldg_cg(in + i) * (double)ldg_cg(in + i);
                    }
                    if (tau > 0.0) {
                        cluster_sum<2>(nr, part, slot);
                        slot ^= 1;
                        if (threadIdx.x == 0) s_flag = (sqrt(nr[0]) <= tau * sqrt(nr[1])) ? 0 : 1;
                        __syncthreads();
                        second = s_flag != 0;
                    }
                }
                if (second) {  // c2 = B_m(rho~)
                    child = TailFrame{1, f.level, 0, rt, c2, 0.0, 0.0, 0.0};
                    push = 1;
                    next_phase = 2;
                } else {
                    next_phase = 3;
                }
            } else if (f.phase == 2) {  // v2 = A c2; beta, gamma, alpha2
                double d[3] = {0.0, 0.0, 0.0};
                cl_rows<T>(
                    L, gw, nw, [&](int j) { return ldg_cg(c2 + j); },
                    [&](int i, T acc) {
                        v2[i] = acc;
                        const double xi = (double)ldg_cg(c2 + i);
                        d[0] = fma(xi, (double)acc, d[0]);
                        d[1] = fma(xi, (double)ldg_cg(v1 + i), d[1]);
                        d[2] = fma(xi, (double)ldg_cg(rt + i), d[2]);
                    });
                cluster_sum<3>(d, part, slot);
                slot ^= 1;
                if (threadIdx.x == 0) {  // only thread 0 keeps the frame's scalars
                    const double beta = d[0], gamma = d[1], alpha2 = d[2];
                    const double rho2 = beta - gamma * gamma / rho1;
                    if (rho2 > 0.0) {
                        w1 = w1 - gamma * alpha2 / (rho1 * rho2);
                        w2 = alpha2 / rho2;
                    }
                }
                next_phase = 3;
            } else {  // e = w1 c1 + w2 c2
                const T w1t = (T)w1, w2t = (T)w2;
                for (int i = g0; i < L.n; i += G) {
                    T v = mul_rn(w1t, ldg_cg(c1 + i));
                    if (w2 != 0.0) v = add_rn(v, mul_rn(w2t, ldg_cg(c2 + i)));
                    out[i] = v;
                }
                pop = 1;
            }
        } else {  // ---- B_l: pre-sweep, restriction, K_{l+1}, prolongation + post-sweep ----
            const TailLevel C = lv[f.level + 1];
            const T* minv = (const T*)L.minv;
            T* x = (T*)L.w;
            T* s = (T*)L.s;
            T* rc = (T*)C.rhs;
            T* ec = (T*)C.out;
            if (f.phase == 0) {
                cl_rows<T>(
                    L, gw, nw, [&](int j) { return mul_rn(minv[j], ldg_cg(in + j)); },
                    [&](int i, T acc) {
                        x[i] = mul_rn(minv[i], ldg_cg(in + i));
                        s[i] = sub_rn(ldg_cg(in + i), acc);
                    });
                cl.sync();  // every block's s before the restriction
                for (int I = g0; I < C.n; I += G) {
                    const int q1 = L.aggptr[I + 1];
                    T sum = T(0);
                    for (int q = L.aggptr[I]; q < q1; q += kTailBatch) {
                        T sv[kTailBatch];
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++)
                            sv[u] = q + u < q1 ? ldg_cg(s + L.members[q + u]) : T(0);
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++)
                            if (q + u < q1) sum = add_rn(sum, sv[u]);
                    }
                    rc[I] = sum;
                }
                child = TailFrame{0, f.level + 1, 0, rc, ec, 0.0, 0.0, 0.0};
                push = 1;
                next_phase = 1;
            } else {
                cl_rows<T>(
                    L, gw, nw,
                    [&](int j) { return add_rn(ldg_cg(x + j), ldg_cg(ec + L.agg[j])); },
                    [&](int i, T acc) {
                        const T xi = add_rn(ldg_cg(x + i), ldg_cg(ec + L.agg[i]));
                        out[i] = add_rn(xi, mul_rn(minv[i], sub_rn(ldg_cg(in + i), acc)));
                    });
                pop = 1;
            }
        }
        cl.sync();  // this phase's writes are visible to every block of the cluster
        if (threadIdx.x == 0) {
            if (pop) {
                sp = top - 1;
            } else {
                st[top - 1].phase = next_phase;
                st[top - 1].rho1 = rho1;
                st[top - 1].w1 = w1;
                st[top - 1].w2 = w2;
                if (push) {
                    st[top] = child;
                    sp = top + 1;
                }
            }
        }
        __syncthreads();
    }
}

// Blocks of the cluster: 16 where the device allows that size for this kernel, else 8.
template <typename T>
static int cluster_blocks(Handle* h) {
    static DevCache cache;
    int c = cache.get(h->device);
    if (c) return c;
    c = 8;
    if (cudaFuncSetAttribute(k_tail_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) == cudaSuccess) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kClusterThreads);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_tail_cluster<T>, &cfg) == cudaSuccess &&
            nclusters >= 1)
            c = 16;
    }
    cudaGetLastError();
    cache.set(h->device, c);
    return c;
}

template <typename T>
int launch_tail(Handle* h, int m0) {
    if (!h->tail_cluster) {
        k_tail<T><<<1, kTailThreads, 0, h->work>>>(h->tail_dev, m0, h->nlev, h->coarse_inv,
                                                   h->p.kcycle_tau, &h->ctrl->skip);
        count_launch(h);
        return check_cuda(cudaGetLastError());
    }
    const int nb = cluster_blocks<T>(h);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.stream = h->work;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nb;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tail_cluster<T>, (const TailLevel*)h->tail_dev,
                                       m0, h->nlev, (const double*)h->coarse_inv,
                                       h->p.kcycle_tau, (const int*)&h->ctrl->skip);
    count_launch(h);
    return check_cuda(e);
}
template int launch_tail<float>(Handle*, int);
template int launch_tail<double>(Handle*, int);

}  // namespace uaamg
