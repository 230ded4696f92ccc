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


// ---- the same recursion on one thread-block cluster, its data in shared memory ----------
//
// From level m0 down to the coarsest, the recursion runs on one cluster of C blocks (16
// where the device allows that size, else 8) of 1024 threads.  Every level's rows are split
// into C contiguous ranges of chunk = ceil(n / C) rows, and block c owns range c: it
// computes those rows in every phase.
//  - Vectors that other rows gather (x, s and e, c1, c2; on the coarsest level its
//    right-hand side and solution) are replicated: each block keeps the whole vector in its
//    shared memory, and a block writes its rows into every block's copy (coalesced stores
//    to distributed shared memory), so every gather is a local shared-memory load.  A phase
//    whose rows other blocks read ends with a cluster barrier (release / acquire at
//    cluster scope).  The rest (rho, v1, rho~) are kept for the block's own rows only.
//  - Setup packs each block's rows of the level matrices (row offsets, columns, values,
//    the aggregate of every column), its rows of the l1-Jacobi diagonal, its aggregates'
//    member lists and its rows of the coarsest inverse into one region per block; every
//    launch stages the region into shared memory with asynchronous 16-byte copies.  Where a
//    tail does not fit, the per-entry arrays of its largest levels stay in global memory
//    (L2) and the row loops read them there.
// Inner products: each block reduces its rows in a fixed tree, and every block adds the C
// block partials in rank order, so all blocks hold the same totals, take the same branches
// and keep identical frame stacks.  The arithmetic of every vector entry is that of the
// launch-by-launch kernels: rows summed in stored order by their lanes with a fixed shuffle
// tree, aggregates' members in ascending order, rounded adds and multiplies where those
// round.
}  // namespace uaamg
#include <cooperative_groups.h>

#include <type_traits>
namespace uaamg {
namespace cg = cooperative_groups;

constexpr int kDsmThreads = 1024;
constexpr int kDsmMaxRows = 1 << 16;    // rows of a tail level, at most (16-bit indices)
constexpr int kDsmInvStaged = 96 * 1024;  // coarsest inverse rows staged up to this size
constexpr int kDsmMaxLev = 16;            // levels of the tail, at most

// Vectors of a level: RHS (rho), V1 and RT are the block's own rows; X, SE (s, and later
// e), C1 and C2 are replicated.  On the coarsest level RHS and SE (the solution) are
// replicated and the others absent.
enum DsmVec { DV_RHS = 0, DV_X, DV_SE, DV_C1, DV_V1, DV_RT, DV_C2, kDsmVecs };
__host__ __device__ inline bool dsm_replicated(int v, bool coarsest) {
    return coarsest ? (v == DV_RHS || v == DV_SE) : (v == DV_X || v == DV_SE || v == DV_C1 || v == DV_C2);
}

// One level as a block of the cluster sees it.  `vec` are byte offsets in the block's
// shared memory (the same in every block); the arrays are byte offsets in the block's
// region (staged at byte `vb` of shared memory, or read from global memory when `streamed`).
struct DsmLev {
    int n, chunk, rows, row0;  // rows of the level, rows per block, this block's rows, first
    int inner, lpr;            // flexible-CG steps as a coarse level; lanes per row
    int chunkc, rowsc, row0c;  // next level: rows per block, this block's aggregates, first
    int streamed;              // col, agg and val read from global memory
    int vec[kDsmVecs];
    int rp, col, agg, val, minv, aggo, ap, mem;  // coarsest: val = this block's inverse rows
    int inv_global;  // coarsest: 1 when the inverse rows are read from the handle's inverse
};
// Head of a block's region (a 16-byte multiple).
struct DsmHead {
    int bytes;   // bytes of the region, this head included
    int staged;  // bytes of its staged part (the head first)
    int pad[2];
    DsmLev lv[kDsmMaxLev];  // level m0 + i at i
};
static_assert(sizeof(DsmHead) % 16 == 0, "region head size");

// Per-block entry counts of a level (from the pack kernel's first pass).
struct DsmCount {
    int E, M;  // matrix entries of the block's rows; members of its aggregates
};

// Offsets of one block's region: the head, the staged arrays of every level, then the
// streamed per-entry arrays.  The same function runs on the host (to choose m0 and what
// is streamed) and in the pack kernel (to write the region).
__host__ __device__ inline void dsm_layout(DsmHead& H, int nl, int tsize, const DsmCount* cnt,
                                           unsigned streamed_mask) {
    long long off = sizeof(DsmHead);
    auto take = [&](long long bytes) {
        const long long o = off;
        off += (bytes + 15) & ~15LL;
        return (int)o;
    };
    for (int i = 0; i < nl; i++) {
        DsmLev& D = H.lv[i];
        D.streamed = (streamed_mask >> i) & 1;
        if (i == nl - 1) {
            if (!D.inv_global && !D.streamed) D.val = take(8LL * D.rows * D.n);
            continue;
        }
        D.rp = take(4LL * (D.chunk + 1));
        if (!D.streamed) {
            D.col = take(2LL * cnt[i].E);
            D.agg = take(2LL * cnt[i].E);
            D.val = take((long long)tsize * cnt[i].E);
        }
        D.minv = take((long long)tsize * D.chunk);
        D.aggo = take(2LL * D.chunk);
        D.ap = take(4LL * (D.chunkc + 1));
        D.mem = take(2LL * cnt[i].M);
    }
    H.staged = off > (1LL << 30) ? (1 << 30) : (int)off;
    for (int i = 0; i < nl; i++) {
        DsmLev& D = H.lv[i];
        if (!D.streamed) continue;
        if (i == nl - 1) {  // the coarsest inverse rows, read through L2
            if (!D.inv_global) D.val = take(8LL * D.rows * D.n);
            continue;
        }
        D.col = take(2LL * cnt[i].E);
        D.agg = take(2LL * cnt[i].E);
        D.val = take((long long)tsize * cnt[i].E);
    }
    H.bytes = off > (1LL << 30) ? (1 << 30) : (int)off;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t dsm_map(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsm_st(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void dsm_st(uint32_t a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ float dsm_ldr(uint32_t a, float) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double dsm_ldr(uint32_t a, double) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
// Entry `p` (shared address in this block) of every block's copy of a replicated vector.
template <typename T>
__device__ __forceinline__ void bcast(const T* p, T v, int C) {
    const uint32_t a = smem_u32(p);
    for (int r = 0; r < C; r++) dsm_st(dsm_map(a, r), v);
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Inner-product accumulators.  FP64 cycles add FP64 products.  FP32 cycles accumulate in
// FP32 pairs (hi + lo): each product is split exactly by an FMA (Dekker's two-product) and
// added with Knuth's two-sum, which keeps about 48 significant bits at these lengths.
// GB300 runs FP32 at many times its FP64 rate, and one FP64 instruction of a warp occupies
// an SM's FP64 units for many cycles, which made FP64 block reductions the longest part of
// these small-level phases.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& a, float b) {  // two-sum of a.hi and b
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ void acc_prod(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_prod(FF& a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);  // x y - p, exactly
    ff_add(a, p);
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void acc_merge(double& a, double b) { a += b; }
__device__ __forceinline__ void acc_merge(FF& a, FF b) {
    ff_add(a, b.hi);
    a.lo = __fadd_rn(a.lo, b.lo);
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_down(double a, int o) {
    return __shfl_down_sync(0xffffffffu, a, o);
}
__device__ __forceinline__ FF acc_down(FF a, int o) {
    return FF{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}
// Fixed tree over the warp; lane 0 holds the total.
template <typename A>
__device__ __forceinline__ A acc_warp(A a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_merge(a, acc_down(a, o));
    return a;
}
// Block `rank`'s copy of the partial at shared address `pa`.
__device__ __forceinline__ double acc_remote(uint32_t pa, int rank, double) {
    return dsm_ldr(dsm_map(pa, rank), 0.0);
}
__device__ __forceinline__ FF acc_remote(uint32_t pa, int rank, FF) {
    const uint32_t r = dsm_map(pa, rank);
    return FF{dsm_ldr(r, 0.f), dsm_ldr(r + 4u, 0.f)};
}
template <typename T>
using DotAcc = typename std::conditional<sizeof(T) == 4, FF, double>::type;

// Cluster-wide fixed-order sum of ND accumulators: a tree over each warp, over the block's
// warps, then over the blocks in rank order; every thread of every block receives the same
// FP64 totals.  `slot` alternates between two partial buffers, so a block that runs ahead
// cannot overwrite partials another block is still reading.
template <typename A, int ND>
__device__ __forceinline__ void dsm_sum(const A (&v)[ND], double (&out)[ND], A (*part)[4], int slot,
                                        int C) {
    __shared__ A sh[ND][kDsmThreads / 32];
    __shared__ double tot[ND];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ND; k++) {
        const A s = acc_warp(v[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
            const A s = acc_warp(lane < kDsmThreads / 32 ? sh[k][lane] : A{});
            if (lane == 0) part[slot][k] = s;
        }
    }
    cluster_barrier();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
            A pv{};
            if (lane < C) pv = acc_remote(smem_u32(&part[slot][k]), lane, pv);
            const A s = acc_warp(pv);
            if (lane == 0) tot[k] = acc_value(s);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; k++) out[k] = tot[k];
}

// The block's view of one level: its arrays (staged or streamed) and vectors.
template <typename T>
struct DsmView {
    const int* rp;
    const uint16_t *col, *agg, *aggo, *mem;
    const T *val, *minv;
    const int* ap;
};
template <typename T>
__device__ __forceinline__ DsmView<T> dsm_view(const DsmLev& L, const unsigned char* staged,
                                               const unsigned char* region) {
    const unsigned char* pe = L.streamed ? region : staged;  // the per-entry arrays
    DsmView<T> v;
    v.rp = (const int*)(staged + L.rp);
    v.col = (const uint16_t*)(pe + L.col);
    v.agg = (const uint16_t*)(pe + L.agg);
    v.val = (const T*)(pe + L.val);
    v.minv = (const T*)(staged + L.minv);
    v.aggo = (const uint16_t*)(staged + L.aggo);
    v.ap = (const int*)(staged + L.ap);
    v.mem = (const uint16_t*)(staged + L.mem);
    return v;
}

// This block's rows of level L, L.lpr lanes per row: the lanes of a row take its entries
// in turn (each lane's own in stored order, kTailBatch operands in flight), combine their
// sums by a fixed shuffle tree, and the row's first lane calls epi(i, sum) (i counts the
// block's rows).  g(k) is the gathered operand of entry k.  The loop is uniform over each
// warp.
template <typename T, typename G, typename E>
__device__ __forceinline__ void dsm_rows(const DsmLev& L, const DsmView<T>& V, G g, E epi) {
    const int lpr = L.lpr, rows = L.rows;
    const int lane = threadIdx.x & 31, sub = lane & (lpr - 1), rpw = 32 / lpr;
    for (int base = (threadIdx.x >> 5) * rpw; base < rows; base += (kDsmThreads / 32) * rpw) {
        const int i = base + lane / lpr;
        T acc = T(0);
        if (i < rows) {
            const int k1 = V.rp[i + 1];
            for (int k = V.rp[i] + sub; k < k1; k += kTailBatch * lpr) {
                T xg[kTailBatch], vv[kTailBatch];
#pragma unroll
                for (int u = 0; u < kTailBatch; u++) {
                    const int kk = k + u * lpr;
                    const bool in = kk < k1;
                    xg[u] = in ? g(kk) : T(0);
                    vv[u] = in ? V.val[kk] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kTailBatch; u++)
                    if (k + u * lpr < k1) acc = fma_rn(vv[u], xg[u], acc);
            }
        }
        for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lpr);
        if (i < rows && sub == 0) epi(i, acc);
    }
}

// A frame of the recursion; `in` and `out` name vectors of the frame's level.
struct DsmFrame {
    int kind;  // 0: K_m, 1: B_m
    int level;
    int phase;
    int in, out;
    double rho1, w1, w2;
};

template <typename T>
__global__ void __launch_bounds__(kDsmThreads, 1)
k_tail_dsm(const unsigned char* __restrict__ blob, long long stride, int copy16, int vb, int m0,
           int nlev, const double* __restrict__ inv, double tau, const T* __restrict__ rhs_g,
           T* __restrict__ out_g, const int* skip) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ DsmFrame st[2 * kDsmMaxLev];
    __shared__ int sp;
    __shared__ DotAcc<T> part[2][4];  // this block's inner-product partials (two slots)
    __shared__ double s_w;            // a step scalar computed by thread 0
    __shared__ int s_flag;            // a step decision taken by thread 0
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int tid = threadIdx.x;
    const unsigned char* region = blob + (size_t)blockIdx.x * (size_t)stride;
    {  // stage the region's staged part
        const uint32_t dst = smem_u32(sm + vb);
        for (int i = tid; i < copy16; i += kDsmThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * i),
                         "l"(region + 16 * (size_t)i)
                         : "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    // the region is setup data; what the preceding kernels write is read from here on
    pdl_wait();
    if (skip && *(volatile const int*)skip) return;  // uniform over the cluster
    __syncthreads();
    const unsigned char* staged = sm + vb;
    const DsmHead& H = *(const DsmHead*)staged;
    {
        const DsmLev& L = H.lv[0];
        T* rho = (T*)(sm + L.vec[DV_RHS]);
        for (int i = tid; i < L.rows; i += kDsmThreads) rho[i] = rhs_g[L.row0 + i];
    }
    if (tid == 0) {  // K_m0, with its first step's B_m0 already pushed
        st[0] = DsmFrame{0, m0, 1, DV_RHS, DV_SE, 0.0, 0.0, 0.0};
        st[1] = DsmFrame{1, m0, 0, DV_RHS, DV_C1, 0.0, 0.0, 0.0};
        sp = 2;
    }
    int slot = 0;
    __syncthreads();
    while (true) {
        const int top = sp;
        if (top == 0) break;
        const DsmFrame f = st[top - 1];
        const DsmLev& L = H.lv[f.level - m0];
        const bool coarsest = f.level == nlev - 1;
        // a vector of this level: the block's rows (own), or the whole replicated vector
        auto full = [&](int v) { return (T*)(sm + L.vec[v]); };
        auto own = [&](int v) {
            return (T*)(sm + L.vec[v]) + (dsm_replicated(v, coarsest) ? L.row0 : 0);
        };
        int push = 0, pop = 0, next_phase = f.phase;
        DsmFrame child{}, child2{};  // push = 2: child2 goes on top of child
        double rho1 = f.rho1, w1 = f.w1, w2 = f.w2;
        bool cluster_end = false;  // the phase's rows are read by other blocks next
        if (coarsest) {  // exact solve with the dense inverse, a warp per row
            cluster_barrier();  // every block's rows of the right-hand side
            const T* b = full(DV_RHS);
            T* e = full(DV_SE);
            const int lane = tid & 31;
            for (int i = tid >> 5; i < L.rows; i += kDsmThreads / 32) {
                T v;
                bool done = false;
                if constexpr (sizeof(T) == 4) {
                    if (!L.inv_global) {  // FP32 pairs hi + lo of the inverse, FP32-pair sums
                        const float2* row =
                            (const float2*)((L.streamed ? region : staged) + L.val) + (size_t)i * L.n;
                        FF a{0.f, 0.f};
                        for (int j = lane; j < L.n; j += 32) {
                            const float2 w = row[j];
                            acc_prod(a, w.x, b[j]);
                            a.lo = __fmaf_rn(w.y, b[j], a.lo);
                        }
                        a = acc_warp(a);
                        v = __fadd_rn(a.hi, a.lo);
                        done = true;
                    }
                }
                if (!done) {
                    const double* row = L.inv_global ? inv + (size_t)(L.row0 + i) * L.n
                                                     : (const double*)((L.streamed ? region : staged) + L.val) +
                                                           (size_t)i * L.n;
                    double sum = 0.0;
                    for (int j = lane; j < L.n; j += 32) sum = fma(row[j], (double)b[j], sum);
                    sum = warp_sum(sum);
                    v = (T)sum;
                }
                if (lane == 0) bcast(e + L.row0 + i, v, C);
            }
            pop = 1;
            cluster_end = true;
        } else if (f.kind == 0) {  // ---- K_m: flexible-CG steps preconditioned by B_m ----
            const DsmView<T> V = dsm_view<T>(L, staged, region);
            const T* in = own(DV_RHS);
            const T *c1 = full(DV_C1), *c2 = full(DV_C2);
            T *v1 = own(DV_V1), *rt = own(DV_RT);
            if (f.phase == 0) {  // c1 = B_m(rho)
                child = DsmFrame{1, f.level, 0, DV_RHS, DV_C1, 0.0, 0.0, 0.0};
                push = 1;
                next_phase = 1;
            } else if (f.phase == 1) {  // v1 = A c1; rho1, alpha1; rho~
                DotAcc<T> a[2] = {};
                const T* c1o = c1 + L.row0;
                dsm_rows<T>(
                    L, V, [&](int k) { return c1[V.col[k]]; },
                    [&](int i, T acc) {
                        v1[i] = acc;
                        acc_prod(a[0], c1o[i], acc);
                        acc_prod(a[1], c1o[i], in[i]);
                    });
                double d[2];
                dsm_sum(a, d, part, slot, C);
                slot ^= 1;
                // the step's scalars in one thread, broadcast through shared memory
                if (tid == 0) {
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
                    DotAcc<T> an[2] = {};
                    for (int i = tid; i < L.rows; i += kDsmThreads) {
                        const T v = sub_rn(in[i], mul_rn(a1t, v1[i]));
                        rt[i] = v;
                        acc_prod(an[0], v, v);
                        acc_prod(an[1], in[i], in[i]);
                    }
                    if (tau > 0.0) {
                        double nr[2];
                        dsm_sum(an, nr, part, slot, C);
                        slot ^= 1;
                        if (tid == 0) s_flag = (sqrt(nr[0]) <= tau * sqrt(nr[1])) ? 0 : 1;
                        __syncthreads();
                        second = s_flag != 0;
                    }
                }
                if (second) {  // c2 = B_m(rho~)
                    child = DsmFrame{1, f.level, 0, DV_RT, DV_C2, 0.0, 0.0, 0.0};
                    push = 1;
                    next_phase = 2;
                } else {
                    next_phase = 3;
                }
            } else if (f.phase == 2) {  // v2 = A c2; beta, gamma, alpha2
                DotAcc<T> a[3] = {};
                const T* c2o = c2 + L.row0;
                dsm_rows<T>(
                    L, V, [&](int k) { return c2[V.col[k]]; },
                    [&](int i, T acc) {
                        acc_prod(a[0], c2o[i], acc);
                        acc_prod(a[1], c2o[i], v1[i]);
                        acc_prod(a[2], c2o[i], rt[i]);
                    });
                double d[3];
                dsm_sum(a, d, part, slot, C);
                slot ^= 1;
                if (tid == 0) {  // only thread 0 keeps the frame's scalars
                    const double beta = d[0], gamma = d[1], alpha2 = d[2];
                    const double rho2 = beta - gamma * gamma / rho1;
                    if (rho2 > 0.0) {
                        w1 = w1 - gamma * alpha2 / (rho1 * rho2);
                        w2 = alpha2 / rho2;
                    }
                }
                next_phase = 3;
            } else {  // e = w1 c1 + w2 c2, every row in every block (c1, c2 are replicated)
                const T w1t = (T)w1, w2t = (T)w2;
                T* e = full(DV_SE);
                for (int j = tid; j < L.n; j += kDsmThreads) {
                    T v = mul_rn(w1t, c1[j]);
                    if (w2 != 0.0) v = add_rn(v, mul_rn(w2t, c2[j]));
                    e[j] = v;
                }
                pop = 1;
            }
        } else {  // ---- B_l: pre-sweep, restriction, K_{l+1}, prolongation + post-sweep ----
            const DsmView<T> V = dsm_view<T>(L, staged, region);
            const DsmLev& Lc = H.lv[f.level + 1 - m0];
            const bool child_coarsest = f.level + 1 == nlev - 1;
            const T* in = own(f.in);
            T* x = full(DV_X);
            if (f.phase == 0) {
                T* s = full(DV_SE);
                for (int i = tid; i < L.rows; i += kDsmThreads)
                    bcast(x + L.row0 + i, mul_rn(V.minv[i], in[i]), C);
                cluster_barrier();  // every block's rows of x
                dsm_rows<T>(
                    L, V, [&](int k) { return x[V.col[k]]; },
                    [&](int i, T acc) { bcast(s + L.row0 + i, sub_rn(in[i], acc), C); });
                cluster_barrier();  // every block's rows of s
                // r_c = P^T s for this block's aggregates
                T* rc = (T*)(sm + Lc.vec[DV_RHS]) + (child_coarsest ? Lc.row0 : 0);
                for (int I = tid; I < L.rowsc; I += kDsmThreads) {
                    const int q1 = V.ap[I + 1];
                    T sum = T(0);
                    for (int q = V.ap[I]; q < q1; q += kTailBatch) {
                        T sv[kTailBatch];
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++) sv[u] = q + u < q1 ? s[V.mem[q + u]] : T(0);
#pragma unroll
                        for (int u = 0; u < kTailBatch; u++)
                            if (q + u < q1) sum = add_rn(sum, sv[u]);
                    }
                    if (child_coarsest) bcast(rc + I, sum, C);  // the dense solve reads it all
                    else rc[I] = sum;
                }
                if (child_coarsest) {
                    child = DsmFrame{0, f.level + 1, 0, DV_RHS, DV_SE, 0.0, 0.0, 0.0};
                    push = 1;
                } else {  // K_{l+1} at its first step, with that step's B_{l+1} on top
                    child = DsmFrame{0, f.level + 1, 1, DV_RHS, DV_SE, 0.0, 0.0, 0.0};
                    child2 = DsmFrame{1, f.level + 1, 0, DV_RHS, DV_C1, 0.0, 0.0, 0.0};
                    push = 2;
                }
                next_phase = 1;
            } else {  // out = x' + Minv (in - A x'), x' = x + P e_c
                const T* ec = (const T*)(sm + Lc.vec[DV_SE]);
                T* out = full(f.out);
                dsm_rows<T>(
                    L, V, [&](int k) { return add_rn(x[V.col[k]], ec[V.agg[k]]); },
                    [&](int i, T acc) {
                        const T xi = add_rn(x[L.row0 + i], ec[V.aggo[i]]);
                        bcast(out + L.row0 + i, add_rn(xi, mul_rn(V.minv[i], sub_rn(in[i], acc))), C);
                    });
                pop = 1;
                cluster_end = true;  // K_l's SpMV gathers its c1 or c2
            }
        }
        if (cluster_end) cluster_barrier();
        else __syncthreads();
        if (tid == 0) {
            if (pop) {
                sp = top - 1;
            } else {
                st[top - 1].phase = next_phase;
                st[top - 1].rho1 = rho1;
                st[top - 1].w1 = w1;
                st[top - 1].w2 = w2;
                if (push) st[top] = child;
                if (push == 2) st[top + 1] = child2;
                sp = top + push;
            }
        }
        __syncthreads();
    }
    // K_m0's output rows; the last barrier keeps every block's shared memory alive until no
    // block reads another's partials any more
    const DsmLev& L = H.lv[0];
    const T* e = (const T*)(sm + L.vec[DV_SE]) + L.row0;
    for (int i = tid; i < L.rows; i += kDsmThreads) out_g[L.row0 + i] = e[i];
    cluster_barrier();
}

// ---- setup: one region per block -------------------------------------------------------
struct DsmPackLevel {
    int n, nc;
    const int *rowptr, *col, *agg, *aggptr, *members;
    const void *val, *minv;
};
struct DsmPackArgs {
    int m0, nl, write;   // tail levels m0 .. m0 + nl - 1; 0: count only, 1: write regions
    unsigned streamed;   // levels (bit i: level m0 + i) whose per-entry arrays are streamed
    long long stride;    // bytes between two blocks' regions
    DsmHead H;           // the fields every block shares (sizes, vector offsets, lpr, inner)
    DsmPackLevel lv[kDsmMaxLev];
    const double* inv;
    unsigned char* blob;
    DsmCount* counts;  // block c's count of level m0 + i at counts[c * cstride + coff + i]
    int cstride, coff;
};

// Block c counts (write = 0) or writes (write = 1) region c.
template <typename T>
__global__ void k_tail_pack(const DsmPackArgs a) {
    __shared__ DsmHead H;
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        H = a.H;
        for (int i = 0; i < a.nl; i++) {
            const DsmPackLevel& P = a.lv[i];
            DsmLev& D = H.lv[i];
            D.row0 = min(c * D.chunk, D.n);
            D.rows = min(D.row0 + D.chunk, D.n) - D.row0;
            if (i < a.nl - 1) {
                D.row0c = min(c * D.chunkc, P.nc);
                D.rowsc = min(D.row0c + D.chunkc, P.nc) - D.row0c;
                if (!a.write) {
                    DsmCount& k = a.counts[c * a.cstride + a.coff + i];
                    k.E = P.rowptr[D.row0 + D.rows] - P.rowptr[D.row0];
                    k.M = P.aggptr[D.row0c + D.rowsc] - P.aggptr[D.row0c];
                }
            } else {
                D.row0c = D.rowsc = 0;
            }
        }
        if (a.write) dsm_layout(H, a.nl, (int)sizeof(T), a.counts + c * a.cstride + a.coff, a.streamed);
    }
    __syncthreads();
    if (!a.write || H.bytes > a.stride) return;
    unsigned char* reg = a.blob + (size_t)c * a.stride;
    {
        const int* hp = (const int*)&H;
        int* rp = (int*)reg;
        for (int i = threadIdx.x; i < (int)(sizeof(DsmHead) / 4); i += blockDim.x) rp[i] = hp[i];
    }
    for (int i = 0; i < a.nl; i++) {
        const DsmPackLevel& P = a.lv[i];
        const DsmLev& D = H.lv[i];
        const int r0 = D.row0;
        if (i == a.nl - 1) {
            if (!D.inv_global) {  // FP32 cycles: each entry as an FP32 pair hi + lo
                const long long cnt = (long long)D.rows * D.n;
                for (long long k = threadIdx.x; k < cnt; k += blockDim.x) {
                    const double v = a.inv[(size_t)r0 * D.n + k];
                    if (sizeof(T) == 4) {
                        const float hi = (float)v;
                        ((float2*)(reg + D.val))[k] = make_float2(hi, (float)(v - (double)hi));
                    } else {
                        ((double*)(reg + D.val))[k] = v;
                    }
                }
            }
            continue;
        }
        const int e0 = P.rowptr[r0], E = P.rowptr[r0 + D.rows] - e0;
        const int q0 = P.aggptr[D.row0c], M = P.aggptr[D.row0c + D.rowsc] - q0;
        int* rpo = (int*)(reg + D.rp);
        for (int k = threadIdx.x; k <= D.chunk; k += blockDim.x)
            rpo[k] = P.rowptr[r0 + min(k, D.rows)] - e0;
        uint16_t* col = (uint16_t*)(reg + D.col);
        uint16_t* agg = (uint16_t*)(reg + D.agg);
        T* val = (T*)(reg + D.val);
        const T* sval = (const T*)P.val;
        for (int k = threadIdx.x; k < E; k += blockDim.x) {
            const int j = P.col[e0 + k];
            col[k] = (uint16_t)j;
            agg[k] = (uint16_t)P.agg[j];
            val[k] = sval[e0 + k];
        }
        T* mv = (T*)(reg + D.minv);
        uint16_t* ao = (uint16_t*)(reg + D.aggo);
        const T* smv = (const T*)P.minv;
        for (int k = threadIdx.x; k < D.chunk; k += blockDim.x) {
            mv[k] = k < D.rows ? smv[r0 + k] : T(0);
            ao[k] = k < D.rows ? (uint16_t)P.agg[r0 + k] : (uint16_t)0;
        }
        int* apo = (int*)(reg + D.ap);
        for (int I = threadIdx.x; I <= D.chunkc; I += blockDim.x)
            apo[I] = P.aggptr[D.row0c + min(I, D.rowsc)] - q0;
        uint16_t* mem = (uint16_t*)(reg + D.mem);
        for (int q = threadIdx.x; q < M; q += blockDim.x) mem[q] = (uint16_t)P.members[q0 + q];
    }
}

static int round16(long long b) { return (int)((b + 15) & ~15LL); }

// Blocks per cluster for k_tail_dsm<T> with `smem` bytes of dynamic shared memory: 16
// where the device runs such a cluster, else 8, else 0.
template <typename T>
static int dsm_cluster_blocks(int smem) {
    for (int c : {16, 8}) {
        if (c > 8 && cudaFuncSetAttribute(k_tail_dsm<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                          1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kDsmThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_tail_dsm<T>, &cfg) == cudaSuccess &&
            nclusters >= 1)
            return c;
        cudaGetLastError();
    }
    return 0;
}

// Chooses the tail (its first level m0 >= m_first, and which of its levels stream their
// per-entry arrays) so that every block's vectors and staged region fit in `dyn` bytes,
// packs the regions and sets the handle's tail fields; leaves the tail off when none fits.
// Dynamic shared memory per block and blocks per cluster of k_tail_dsm<T> on this device
// (attributes set once per device); C = 0 where the device runs no such cluster.
template <typename T>
static void dsm_device(int device, int* dyn, int* C) {
    static DevCache cache;  // (dyn << 5) | C, plus one so that 0 means "not computed"
    int v = cache.get(device);
    if (!v) {
        int optin = 0, d = 0, c = 0;
        cudaFuncAttributes fa{};
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) ==
                cudaSuccess &&
            cudaFuncGetAttributes(&fa, k_tail_dsm<T>) == cudaSuccess) {
            d = (optin - (int)fa.sharedSizeBytes - 1024) & ~15;
            if (d > 0 && cudaFuncSetAttribute(k_tail_dsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              d) == cudaSuccess)
                c = dsm_cluster_blocks<T>(d);
        }
        cudaGetLastError();
        v = ((c ? d : 0) << 5 | c) + 1;
        cache.set(device, v);
    }
    *dyn = (v - 1) >> 5;
    *C = (v - 1) & 31;
}

template <typename T>
static int tail_prepare_t(Handle* h, int m_first) {
    const bool mixed = sizeof(T) == 4;
    int dyn = 0, C = 0;
    dsm_device<T>(h->device, &dyn, &C);
    if (C == 0) return UAAMG_OK;  // no cluster tail on this device
    int st = UAAMG_OK;
    const int L = h->nlev - 1;
    int m = m_first;
    while (m < L && (h->lev[m].n > kDsmMaxRows || (h->lev[m].n + C - 1) / C > kDsmMaxRows ||
                     L - m + 1 > kDsmMaxLev))
        m++;
    if (m >= L) return UAAMG_OK;
    // the shared fields, for the deepest tail m .. L
    const int nl_max = L - m + 1;
    DsmPackArgs a{};
    a.m0 = m;
    a.nl = nl_max;
    a.inv = h->coarse_inv;
    for (int i = 0; i < nl_max; i++) {
        const int l = m + i;
        const Level& Lv = h->lev[l];
        DsmLev& D = a.H.lv[i];
        D.n = Lv.n;
        D.chunk = (Lv.n + C - 1) / C;
        int inner = h->p.kcycle_inner;
        if (inner == 2 && h->p.kcycle_ratio > 0.0 &&
            (double)h->lev[l - 1].n < h->p.kcycle_ratio * (double)Lv.n)
            inner = 1;
        D.inner = inner;
        const int avg = Lv.n > 0 ? (int)(Lv.nnz / Lv.n) : 1;
        int lpr = 1;
        while (lpr < 8 && D.chunk * lpr * 2 <= kDsmThreads && lpr * 2 <= std::max(1, avg / 2))
            lpr *= 2;
        D.lpr = lpr;
        DsmPackLevel& P = a.lv[i];
        P.n = Lv.n;
        P.rowptr = Lv.rowptr;
        P.col = Lv.col;
        P.val = mixed ? (const void*)Lv.val32 : (const void*)Lv.val64;
        P.minv = mixed ? (const void*)Lv.minv32 : (const void*)Lv.minv64;
        if (l < L) {
            P.nc = h->lev[l + 1].n;
            D.chunkc = (P.nc + C - 1) / C;
            P.agg = Lv.agg;
            P.aggptr = Lv.aggptr;
            P.members = Lv.members;
        } else {
            D.inv_global = 8LL * D.chunk * D.n > kDsmInvStaged ? 1 : 0;
        }
    }
    // first pass: every block's entry and member counts
    DsmCount* counts = dalloc<DsmCount>(h, (size_t)C * nl_max, &st, true);
    std::vector<DsmCount> counts_hv((size_t)C * nl_max);
    DsmCount* counts_h = counts_hv.data();
    if (st == UAAMG_OK) {
        a.counts = counts;
        a.cstride = nl_max;
        a.coff = 0;
        a.write = 0;
        k_tail_pack<T><<<C, 256, 0, h->work>>>(a);
        count_launch(h);
        st = check_cuda(cudaGetLastError());
    }
    if (st == UAAMG_OK)
        st = check_cuda(cudaMemcpyAsync(counts_h, counts, sizeof(DsmCount) * C * nl_max,
                                        cudaMemcpyDeviceToHost, h->work));
    if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
    // the deepest tail that fits: tails from m0 = m, m + 1, ..., each first with every level
    // staged, then streaming the per-entry arrays of its top levels one by one
    int best_m0 = 0, best_copy = 0, best_vb = 0;
    unsigned best_mask = 0;
    long long best_stride = 0;
    for (int m0 = m; m0 < L && st == UAAMG_OK && !best_m0; m0++) {
        const int off = m0 - m, nl = nl_max - off;
        long long vb = 0;
        DsmHead H{};
        for (int i = 0; i < nl; i++) {
            H.lv[i] = a.H.lv[off + i];
            const bool co = i == nl - 1;
            for (int v = 0; v < kDsmVecs; v++) {
                H.lv[i].vec[v] = (int)vb;
                if (co && !dsm_replicated(v, true)) continue;
                vb += round16((long long)sizeof(T) * (dsm_replicated(v, co) ? H.lv[i].n : H.lv[i].chunk));
            }
        }
        if (vb >= dyn) continue;
        // what streams, in order of preference: nothing; the coarsest inverse; that and the
        // per-entry arrays of the top levels, one more level at a time
        unsigned masks[kDsmMaxLev + 1];
        int nm = 0;
        masks[nm++] = 0u;
        for (int ns = 0; ns < nl - 1; ns++) masks[nm++] = (1u << (nl - 1)) | ((1u << ns) - 1u);
        for (int mi = 0; mi < nm && !best_m0; mi++) {
            const unsigned mask = masks[mi];
            int staged = 0;
            long long total = 0;
            for (int c = 0; c < C; c++) {
                DsmHead Hc = H;
                for (int i = 0; i < nl; i++) {
                    const DsmLev& D = a.H.lv[off + i];
                    Hc.lv[i].row0 = std::min(c * D.chunk, D.n);
                    Hc.lv[i].rows = std::min(Hc.lv[i].row0 + D.chunk, D.n) - Hc.lv[i].row0;
                }
                dsm_layout(Hc, nl, (int)sizeof(T), counts_h + (size_t)c * nl_max + off, mask);
                staged = std::max(staged, Hc.staged);
                total = std::max(total, (long long)Hc.bytes);
            }
            if (vb + staged <= dyn) {
                best_m0 = m0;
                best_mask = mask;
                best_copy = staged;
                best_vb = (int)vb;
                best_stride = (total + 255) & ~255LL;
                a.H = H;
            }
        }
    }
    if (best_m0 && st == UAAMG_OK) {
        const int off = best_m0 - m;
        a.m0 = best_m0;
        a.nl = nl_max - off;
        for (int i = 0; i < a.nl; i++) a.lv[i] = a.lv[off + i];
        a.coff = off;
        const size_t blob_bytes = (size_t)C * (size_t)best_stride;
        unsigned char* blob = st ? nullptr : (unsigned char*)dalloc_bytes(h, blob_bytes, &st);
        if (st == UAAMG_OK) {
            a.write = 1;
            a.streamed = best_mask;
            a.stride = best_stride;
            a.blob = blob;
            k_tail_pack<T><<<C, 256, 0, h->work>>>(a);
            count_launch(h);
            st = check_cuda(cudaGetLastError());
        }
        if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
        if (st == UAAMG_OK) {
            h->tail_blob = blob;
            h->tail_stride = best_stride;
            h->tail_copy = best_copy;
            h->tail_vb = best_vb;
            h->tail_cl = C;
            h->tail_smem = best_vb + best_copy;
            h->tail_level = best_m0;
            h->tail_cluster = true;
        }
    }
    return st;
}

int tail_cluster_prepare(Handle* h, int m_first) {
    return h->p.precision == UAAMG_MIXED ? tail_prepare_t<float>(h, m_first)
                                         : tail_prepare_t<double>(h, m_first);
}

template <typename T>
int launch_tail(Handle* h, int m0) {
    if (!h->tail_cluster) {
        k_tail<T><<<1, kTailThreads, 0, h->work>>>(h->tail_dev, m0, h->nlev, h->coarse_inv,
                                                   h->p.kcycle_tau, &h->ctrl->skip);
        count_launch(h);
        return check_cuda(cudaGetLastError());
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h->tail_cl);
    cfg.blockDim = dim3(kDsmThreads);
    cfg.dynamicSmemBytes = h->tail_smem;
    cfg.stream = h->work;
    // programmatic serialization: the launch and the staging of the region overlap the
    // preceding kernel, which the kernel waits for before it reads its input
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->tail_cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    const Level& L = h->lev[m0];
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tail_dsm<T>, (const unsigned char*)h->tail_blob,
                                       h->tail_stride, h->tail_copy / 16, h->tail_vb, m0, h->nlev,
                                       (const double*)h->coarse_inv, h->p.kcycle_tau,
                                       (const T*)L.rhs, (T*)L.out, (const int*)&h->ctrl->skip);
    count_launch(h);
    return check_cuda(e);
}
template int launch_tail<float>(Handle*, int);
template int launch_tail<double>(Handle*, int);

}  // namespace uaamg
