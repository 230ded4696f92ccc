// kern_tma.cu -- the row-block SpMV kernels of the large levels with their matrix stream
// staged by the Tensor Memory Accelerator.
//
// A persistent block walks row blocks rb = blockIdx.x, blockIdx.x + G, ...  The entries of
// a row block are one contiguous range of col/val; thread 0 copies the ranges of the next
// two row blocks into a two-stage shared-memory ring with 1D bulk copies
// (cp.async.bulk ... mbarrier::complete_tx), so the HBM stream of the matrix runs ahead
// of the computation instead of sitting on each block's critical path.  Each thread then
// walks its own row in the staged arrays, gathering the vector entries eight at a time,
// adds the row in stored order with fused multiply-adds and applies the same fused epilogue
// as k_rowblock: every vector entry is bit-identical to that kernel's with one thread per
// row (the fused inner products are summed in another fixed order, as each block covers
// several row blocks).  A row block whose entries do not fit a stage is read directly from
// global memory.  Every wait on a stage barrier is bounded; on timeout the block records
// kErrTimeout, waits (bounded) for its copies in flight and leaves.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kTmaRows = 256;
constexpr int kTmaCap = 2048;              // entries per stage (16-byte aligned range)
constexpr int kTmaBatch = 8;               // gathers a thread has in flight per row
constexpr long long kTmaSpin = 1LL << 31;  // clock cycles before a stage wait gives up

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

template <typename T>
struct TmaSmem {
    int col[2][kTmaCap];
    T val[2][kTmaCap];
    uint64_t bar[2];
};

// Issues the copies of the entry range [k0, k1) into stage s; false when it does not fit.
template <typename T>
__device__ __forceinline__ bool tma_issue(const RBArgs<T>& a, TmaSmem<T>& sm, int k0, int k1,
                                          int s) {
    const int a0 = k0 & ~3, a1 = (k1 + 3) & ~3;
    const int cnt = a1 - a0;
    if (cnt > kTmaCap || cnt <= 0) return false;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&sm.bar[s], (unsigned)cnt * (4u + (unsigned)sizeof(T)));
    bulk_g2s(sm.col[s], a.col + a0, (unsigned)cnt * 4u, &sm.bar[s]);
    bulk_g2s(sm.val[s], a.val + a0, (unsigned)cnt * (unsigned)sizeof(T), &sm.bar[s]);
    return true;
}

// One row's sum over entries [lo, hi) of col/val, in stored order; the vector entries of
// kTmaBatch entries are gathered before the first is used.
template <typename T, int MODE>
__device__ __forceinline__ T row_sum(const RBArgs<T>& a, const KScal<T>& ks, const int* col,
                                     const T* val, int lo, int hi) {
    T acc = T(0);
    for (int k = lo; k < hi; k += kTmaBatch) {
        T xg[kTmaBatch], vv[kTmaBatch];
#pragma unroll
        for (int u = 0; u < kTmaBatch; u++) {
            const bool in = k + u < hi;
            xg[u] = in ? rb_gather<T, MODE>(a, ks, col[k + u]) : T(0);
            vv[u] = in ? val[k + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kTmaBatch; u++)
            if (k + u < hi) acc = fma_rn(vv[u], xg[u], acc);
    }
    return acc;
}

template <typename T, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) k_rowblock_tma(RBArgs<T> a, Ctrl* ctrl) {
    if (!rb_enter<T, MODE>(a)) return;
    const KScal<T> ks = kscal<T, MODE>(a);
    extern __shared__ __align__(128) unsigned char dyn[];
    TmaSmem<T>& sm = *reinterpret_cast<TmaSmem<T>*>(dyn);
    __shared__ int staged[2];  // 1 when the stage holds its row block's entries
    const int nblk = (a.n + kTmaRows - 1) / kTmaRows;
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < 2; s++) {
            const int rb = blockIdx.x + s * G;
            staged[s] = 0;
            if (rb < nblk)
                staged[s] = tma_issue<T>(a, sm, a.rowptr[rb * kTmaRows],
                                         a.rowptr[min(a.n, (rb + 1) * kTmaRows)], s) ? 1 : 0;
        }
    }
    __syncthreads();
    unsigned phase = 0u;  // bit s: parity of the next completion of stage s
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    bool failed = false;
    for (int it = 0;; it++) {
        const int rb = blockIdx.x + it * G;
        if (rb >= nblk) break;
        const int s = it & 1;
        const int r0 = rb * kTmaRows, r1 = min(a.n, r0 + kTmaRows);
        const int row = r0 + threadIdx.x;
        // thread 0 loads the bounds of the row block it copies into this stage next, so the
        // copy is issued without a memory round trip on the block's path
        const int nrb = rb + 2 * G;
        int nk0 = 0, nk1 = 0;
        if (threadIdx.x == 0 && nrb < nblk) {
            nk0 = a.rowptr[nrb * kTmaRows];
            nk1 = a.rowptr[min(a.n, (nrb + 1) * kTmaRows)];
        }
        int rs = 0, re = 0;
        T ri = T(0), mi = T(0), xi = T(0);
        int gi = 0;
        if (row < r1) {  // per-row operands, loaded before waiting on the stage
            rs = a.rowptr[row];
            re = a.rowptr[row + 1];
            constexpr bool pro = MODE == RB_PROSMOOTH || MODE == RB_PROSMOOTH_E;
            if constexpr (MODE == RB_PRE1_RT) ri = kc_rt_at(a, ks, row);
            else if constexpr (MODE == RB_PRE1 || MODE == RB_SMOOTH || pro || MODE == RB_RESID)
                ri = a.r[row];
            if constexpr (MODE == RB_PRE1 || MODE == RB_PRE1_RT || MODE == RB_SMOOTH || pro)
                mi = a.minv[row];
            if constexpr (MODE == RB_SMOOTH || pro || MODE == RB_SPMV) xi = a.x[row];
            if constexpr (pro) gi = a.agg[row];
        }
        T acc = T(0);
        if (staged[s]) {
            const int a0 = a.rowptr[r0] & ~3;
            long long t0 = clock64();
            while (!mbar_try_wait(&sm.bar[s], (phase >> s) & 1u)) {
                if (clock64() - t0 > kTmaSpin) {
                    failed = true;
                    break;
                }
            }
            if (__syncthreads_or(failed)) {  // one decision for the whole block
                if (threadIdx.x == 0) {
                    atomicOr(&ctrl->err, kErrTimeout);
                    // let the copies still in flight land before the block releases its
                    // shared memory, again with a bound
                    for (int q = 0; q < 2; q++) {
                        if (!staged[q]) continue;
                        const long long t1 = clock64();
                        while (!mbar_try_wait(&sm.bar[q], (phase >> q) & 1u) &&
                               clock64() - t1 < kTmaSpin) {
                        }
                    }
                }
                return;
            }
            phase ^= 1u << s;
            if (row < r1) acc = row_sum<T, MODE>(a, ks, sm.col[s], sm.val[s], rs - a0, re - a0);
        } else if (row < r1) {  // entries beyond a stage: straight from global memory
            acc = row_sum<T, MODE>(a, ks, a.col, a.val, rs, re);
        }
        if (row < r1) {
            const int i = row;
            if constexpr (MODE == RB_PRE1) {
                a.y[i] = mul_rn(mi, ri);
                a.y2[i] = sub_rn(ri, acc);
            } else if constexpr (MODE == RB_PRE1_RT) {
                a.y[i] = mul_rn(mi, ri);
                a.y2[i] = sub_rn(ri, acc);
                a.y3[i] = ri;
            } else if constexpr (MODE == RB_SMOOTH) {
                a.y[i] = add_rn(xi, mul_rn(mi, sub_rn(ri, acc)));
            } else if constexpr (MODE == RB_RESID) {
                const T yi = sub_rn(ri, acc);
                a.y[i] = yi;
                if constexpr (ND >= 1) dv[0] = fma((double)yi, (double)yi, dv[0]);
            } else if constexpr (MODE == RB_PROSMOOTH) {
                const T xp = add_rn(xi, a.e[gi]);
                a.y[i] = add_rn(xp, mul_rn(mi, sub_rn(ri, acc)));
            } else if constexpr (MODE == RB_PROSMOOTH_E) {
                const T xp = add_rn(xi, kc_e_at(a, ks, gi));
                a.y[i] = add_rn(xp, mul_rn(mi, sub_rn(ri, acc)));
            } else {
                a.y[i] = acc;
                const double xd = (double)xi;
                if constexpr (ND >= 1) dv[0] = fma(xd, (double)acc, dv[0]);
                if constexpr (ND >= 2) dv[1] = fma(xd, (double)a.d1[i], dv[1]);
                if constexpr (ND >= 3) dv[2] = fma(xd, (double)a.d2[i], dv[2]);
            }
        }
        // Stage s is free once every thread is past this barrier.  staged[s] is read next
        // two iterations later, after at least one more barrier.
        __syncthreads();
        if (threadIdx.x == 0) staged[s] = (nrb < nblk) ? (tma_issue<T>(a, sm, nk0, nk1, s) ? 1 : 0) : 0;
    }
    if constexpr (ND > 0) {
        if (grid_reduce<ND>(dv, a.partials, a.counter, a.result)) rb_last_block(a);
    }
}

template <typename T, int MODE, int ND>
static int launch_one(Handle* h, const RBArgs<T>& a) {
    static int grid_cache[64] = {0};
    const size_t smem = sizeof(TmaSmem<T>);
    int dev = h->device < 64 ? h->device : 0;
    if (!grid_cache[dev]) {
        cudaFuncSetAttribute(k_rowblock_tma<T, MODE, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowblock_tma<T, MODE, ND>, kThreads,
                                                      smem);
        grid_cache[dev] = (per_sm > 0 ? per_sm : 1) * h->num_sms;
    }
    const int nblk = grid_for(a.n, kTmaRows);
    const int grid = nblk < grid_cache[dev] ? nblk : grid_cache[dev];
    k_rowblock_tma<T, MODE, ND><<<grid, kThreads, smem, h->work>>>(a, h->ctrl);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

template <typename T>
int launch_rowblock_tma(Handle* h, int mode, int ndots, const RBArgs<T>& a) {
#define TMA_CASE(M, D) \
    if (mode == M && ndots == D) return launch_one<T, M, D>(h, a);
    TMA_CASE(RB_PRE1, 0)
    TMA_CASE(RB_PRE1_RT, 0)
    TMA_CASE(RB_PROSMOOTH_E, 0)
    TMA_CASE(RB_SMOOTH, 0)
    TMA_CASE(RB_RESID, 0)
    TMA_CASE(RB_RESID, 1)
    TMA_CASE(RB_PROSMOOTH, 0)
    TMA_CASE(RB_SPMV, 0)
    TMA_CASE(RB_SPMV, 2)
    TMA_CASE(RB_SPMV, 3)
#undef TMA_CASE
    return UAAMG_ERR_INVALID_ARG;
}
template int launch_rowblock_tma<float>(Handle*, int, int, const RBArgs<float>&);
template int launch_rowblock_tma<double>(Handle*, int, int, const RBArgs<double>&);

}  // namespace uaamg
