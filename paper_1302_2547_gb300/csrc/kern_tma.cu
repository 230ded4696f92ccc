// kern_tma.cu -- the row-block SpMV kernels of the large levels with their matrix stream
// staged by the Tensor Memory Accelerator, one pipeline per warp.
//
// A persistent grid; every warp walks its own chunks of 32 rows, c = w, w + W, ... (W warps
// in the grid).  The entries of a chunk are one contiguous range of col/val.  Lane 0 of the
// warp copies the ranges of the warp's next kTmaStages chunks into the warp's own
// shared-memory ring with 1D bulk copies (cp.async.bulk ... mbarrier::complete_tx), so the
// HBM stream of the matrix runs ahead of the computation.  Each lane then walks its own row
// in the staged arrays, gathering the vector entries eight at a time, adds the row in stored
// order with fused multiply-adds and applies the same fused epilogue as k_rowblock: every
// vector entry is bit-identical to that kernel's with one thread per row (the fused inner
// products are summed in another fixed order).  Warps never wait for each other, so no
// block-wide barrier sits between a chunk's gathers and the next one's.  A chunk whose
// entries do not fit a stage is read directly from global memory.  Every wait on a stage
// is bounded; on timeout the warp records kErrTimeout, waits (bounded) for its copies in
// flight, stops its work and still joins the block's final reduction.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kTmaWarps = kThreads / 32;   // warps per block, each with its own pipeline
constexpr int kTmaBatch = 8;               // gathers a lane has in flight per row
constexpr long long kTmaSpin = 1LL << 31;  // clock cycles before a stage wait gives up (default)
// Chunks a warp has staged or in flight, and the stage entries for rows of about 7 entries.
// The kernel is bound by the latency of its vector gathers, so resident warps count more
// than ring depth: with two stages of 232 entries, seven FP32 blocks fit an SM (six with
// 256 entries, four or five with three stages).
constexpr int kTmaStages = 2;
constexpr int kTmaShortCap = 232;

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

// One warp's stages of CAP entries each (CAP a multiple of 4: every array starts on 16 bytes).
template <typename T, int CAP>
struct alignas(16) WarpStages {
    int col[kTmaStages][CAP];
    T val[kTmaStages][CAP];
    uint64_t bar[kTmaStages];
};
static_assert(kTmaShortCap % 4 == 0 && kTmaStages >= 2, "stages start on 16 bytes");
static_assert(sizeof(WarpStages<double, 512>) * kTmaWarps <= 227 * 1024, "ring fits a block");

// Lane 0: copies of the entry range [k0, k1) into stage s; false when it does not fit.
template <typename T, int CAP>
__device__ __forceinline__ bool tma_issue(const RBArgs<T>& a, WarpStages<T, CAP>& ws, int k0,
                                          int k1, int s) {
    const int a0 = k0 & ~3, a1 = (k1 + 3) & ~3;
    const int cnt = a1 - a0;
    if (cnt > CAP || cnt <= 0) return false;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&ws.bar[s], (unsigned)cnt * (4u + (unsigned)sizeof(T)));
    bulk_g2s(ws.col[s], a.col + a0, (unsigned)cnt * 4u, &ws.bar[s]);
    bulk_g2s(ws.val[s], a.val + a0, (unsigned)cnt * (unsigned)sizeof(T), &ws.bar[s]);
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

template <typename T, int MODE, int ND, int CAP>
__global__ void __launch_bounds__(kThreads) k_rowwarp_tma(RBArgs<T> a, Ctrl* ctrl) {
    if (!rb_enter<T, MODE>(a)) return;
    const KScal<T> ks = kscal<T, MODE>(a);
    // a stage wait gives up after the handle's wait limit (about 2 cycles per ns), else
    // kTmaSpin cycles; the wait for copies still in flight after that always takes kTmaSpin
    const long long wait_ns = ctrl->wait_ns;
    const long long spin = wait_ns > 0 ? 2 * wait_ns : kTmaSpin;
    extern __shared__ __align__(128) unsigned char dyn[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStages<T, CAP>& ws = reinterpret_cast<WarpStages<T, CAP>*>(dyn)[warp];
    const int nch = (a.n + 31) >> 5;
    const int W = gridDim.x * kTmaWarps;
    const int gw = blockIdx.x * kTmaWarps + warp;
    unsigned staged = 0;  // bit s: stage s holds its chunk (lane 0's copy, broadcast)
    if (lane == 0) {
        for (int s = 0; s < kTmaStages; s++) mbar_init(&ws.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < kTmaStages; s++) {
            const int c = gw + s * W;
            if (c < nch && tma_issue<T, CAP>(a, ws, a.rowptr[c << 5],
                                             a.rowptr[min(a.n, (c + 1) << 5)], s))
                staged |= 1u << s;
        }
    }
    staged = __shfl_sync(0xffffffffu, staged, 0);
    __syncwarp();
    unsigned phase = 0u;  // bit s: parity of the next completion of stage s
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    for (int it = 0;; it++) {
        const int c = gw + it * W;
        if (c >= nch) break;
        const int s = it % kTmaStages;
        const int r0 = c << 5, r1 = min(a.n, r0 + 32);
        const int row = r0 + lane;
        // lane 0 loads the bounds of the chunk it copies into this stage next
        const int nc = c + kTmaStages * W;
        int nk0 = 0, nk1 = 0;
        if (lane == 0 && nc < nch) {
            nk0 = a.rowptr[nc << 5];
            nk1 = a.rowptr[min(a.n, (nc + 1) << 5)];
        }
        int rs = 0, re = 0;
        RowOps<T> o{};
        if (row < r1) {  // per-row operands, loaded before waiting on the stage
            rs = a.rowptr[row];
            re = a.rowptr[row + 1];
            o = rb_row_ops<T, MODE, ND>(a, ks, row);
        }
        const int k0 = __shfl_sync(0xffffffffu, rs, 0);  // lane 0 holds row r0
        T acc = T(0);
        if ((staged >> s) & 1u) {
            bool failed = false;
            const long long t0 = clock64();
            while (!mbar_try_wait(&ws.bar[s], (phase >> s) & 1u)) {
                if (clock64() - t0 > spin) {
                    failed = true;
                    break;
                }
            }
            if (__any_sync(0xffffffffu, failed)) {
                if (lane == 0) {
                    atomicOr(&ctrl->err, kErrTimeout);
                    // let the copies still in flight land before this warp stops using them
                    for (int q = 0; q < kTmaStages; q++) {
                        if (!((staged >> q) & 1u)) continue;
                        const long long t1 = clock64();
                        while (!mbar_try_wait(&ws.bar[q], (phase >> q) & 1u) &&
                               clock64() - t1 < kTmaSpin) {
                        }
                    }
                }
                __syncwarp();
                break;  // no more work from this warp; it still joins the block reduction
            }
            phase ^= 1u << s;
            const int a0 = k0 & ~3;
            if (row < r1) acc = row_sum<T, MODE>(a, ks, ws.col[s], ws.val[s], rs - a0, re - a0);
        } else if (row < r1) {  // entries beyond a stage: straight from global memory
            acc = row_sum<T, MODE>(a, ks, a.col, a.val, rs, re);
        }
        if (row < r1) rb_row_out<T, MODE, ND>(a, ks, row, acc, o, dv);
        __syncwarp();  // every lane is done with stage s
        if (lane == 0) {
            staged &= ~(1u << s);
            if (nc < nch && tma_issue<T, CAP>(a, ws, nk0, nk1, s)) staged |= 1u << s;
        }
        staged = __shfl_sync(0xffffffffu, staged, 0);
    }
    if constexpr (ND > 0) {
        if (grid_reduce<ND>(dv, a.partials, a.counter, a.result)) rb_last_block(a);
    }
}

template <typename T, int MODE, int ND, int CAP>
static int launch_one(Handle* h, const RBArgs<T>& a) {
    static DevCache grid_cache;  // persistent grid per device (the attribute is set with it)
    const size_t smem = sizeof(WarpStages<T, CAP>) * kTmaWarps;
    int full = grid_cache.get(h->device);
    if (!full) {
        cudaFuncSetAttribute(k_rowwarp_tma<T, MODE, ND, CAP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowwarp_tma<T, MODE, ND, CAP>,
                                                      kThreads, smem);
        full = (per_sm > 0 ? per_sm : 1) * h->num_sms;
        grid_cache.set(h->device, full);
    }
    const int nblk = grid_for((a.n + 31) / 32, kTmaWarps);
    const int grid = nblk < full ? nblk : full;
    k_rowwarp_tma<T, MODE, ND, CAP><<<grid, kThreads, smem, h->work>>>(a, h->ctrl);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

template <typename T, int CAP>
static int launch_cap(Handle* h, int mode, int ndots, const RBArgs<T>& a) {
#define TMA_CASE(M, D) \
    if (mode == M && ndots == D) return launch_one<T, M, D, CAP>(h, a);
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

// Stage size from the average row length: a chunk of 32 rows of a 7-point stencil (224
// entries plus up to 6 of alignment) fits kTmaShortCap entries; longer rows take 512.
template <typename T>
int launch_rowblock_tma(Handle* h, int mode, int ndots, const RBArgs<T>& a) {
    const bool short_rows = a.n > 0 && a.nnz > 0 && a.nnz * 4 <= (long long)a.n * 29;
    return short_rows ? launch_cap<T, kTmaShortCap>(h, mode, ndots, a)
                      : launch_cap<T, 512>(h, mode, ndots, a);
}
template int launch_rowblock_tma<float>(Handle*, int, int, const RBArgs<float>&);
template int launch_rowblock_tma<double>(Handle*, int, int, const RBArgs<double>&);

}  // namespace uaamg
