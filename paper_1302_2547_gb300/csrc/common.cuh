// common.cuh -- types and device helpers shared by the CUDA sources of libuaamg.
#pragma once
#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "uaamg.h"

namespace uaamg {

constexpr int kMaxLevels = 64;
constexpr int kMaxCoarsest = 1024;        // dense inverse of the coarsest level
constexpr int kMaxRoundSlots = 1 << 16;   // aggregation rounds + passes per level
constexpr int kThreads = 256;             // block size of every row / element kernel
constexpr int kRowsPerBlock = 256;        // rows of one row-block SpMV block
constexpr int kChunk = 2048;              // matrix entries staged in shared memory per step
constexpr long long kBarrierTimeoutNs = 2000000000LL;  // bounded grid-barrier wait (default)
constexpr long long kFastPollNs = 100000;  // limits below this are checked on every poll

// error bits raised by device code into Ctrl::err
constexpr int kErrTimeout = 1;
constexpr int kErrNotSpd = 2;
constexpr int kErrBadCsr = 4;
constexpr int kErrSlots = 8;

// vertex states of the aggregation passes (Algorithm 2)
constexpr uint8_t ST_CAND = 0;  // unprocessed, still a candidate of this pass
constexpr uint8_t ST_EXCL = 1;  // unprocessed, within distance 2 of a root of this pass
constexpr uint8_t ST_ROOT = 2;  // coarse vertex chosen in this pass
constexpr uint8_t ST_DONE = 3;  // processed (in an aggregate)

// Device-resident control words of a handle.
struct Ctrl {
    int skip;                // level+1 of the K-cycle level skipping its second step, else 0
    int err;                 // kErr* bits
    unsigned int red_count;  // arrival counter of the last-block reductions
    unsigned int bar_count;  // grid barrier arrivals (zeroed before each cooperative launch)
    unsigned int pad0;
    int npasses;             // written by the aggregation kernel
    long long wait_ns;       // limit of every bounded device wait (0: the defaults)
};

// FP64 scalars of one K-cycle level (Section 4.3).  Step 1 writes (rho1, alpha1), step 2
// writes (beta, gamma, alpha2) contiguously, matching the dot order of the fused kernels.
struct LevelScalars {
    double rho1, alpha1, beta, gamma, alpha2, rtrt, rhorho;
    int skip2;  // 1 when this level's second step is skipped
    int pad;
    // derived once by the last block of the reduction that completes their inputs (per-thread
    // FP64 divisions would make the element-wise kernels FP64-bound):
    //   a1 = alpha1 / rho1 (0 when rho1 <= 0); e = w1 c1 + w2 c2
    double a1, w1, w2;
    float a1f, w1f, w2f, pad2;  // the same, rounded once for FP32 cycles
};

// FP64 scalars of the outer flexible CG.
struct OuterScalars {
    double pq, pr;  // written together by the fused SpMV + dots
    double zq;
    double rr;
    double bb;
    double pq_prev;
    double alpha;
    int first;      // 1 until the first direction update
    int breakdown;  // (p, A p) <= 0 seen
    // device-side iteration loop: stop once rr <= stop_rr, after it_limit iterations or on
    // breakdown; it counts the iterations of the current launch
    double stop_rr;
    int it;
    int it_limit;
    // this iteration's step sizes, derived once by the reductions that complete them
    double beta_cur;   // (z, q) / (p, q)_prev, 0 on the first iteration
    double alpha_cur;  // (p, r) / (p, A p), 0 when (p, A p) <= 0
};

struct Level {
    int n = 0;
    long long nnz = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val64 = nullptr;
    float* val32 = nullptr;
    double* minv64 = nullptr;
    float* minv32 = nullptr;
    uint64_t* prio = nullptr;
    int* pass_of = nullptr;
    int* agg = nullptr;      // fine -> coarse (absent on the coarsest)
    int nc = 0;
    int* aggptr = nullptr;   // [nc+1] members of each aggregate, ascending
    int* members = nullptr;  // [n]
    int passes = 0;
    int rb_rows = kRowsPerBlock;  // rows per block of this level's row-block kernels
    // SpMV kernel family of this level: -1 by the size thresholds (tma_rows, sell_rows),
    // else chosen by the tuner: 0 row-block (rb_rows rows per block), 1 per-warp TMA,
    // 2 sliced ELLPACK; tune_us holds the tuner's timings of its first sweep (row-block with
    // 256, 128, 64, 32 rows per block, TMA, ELLPACK; -1 where not timed)
    int path = -1;
    float tune_us[6] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f};
    // sliced ELLPACK copy (levels with n >= sell_rows): slice offsets, row lengths, columns
    // and values in slice layout; null when not built
    int* sl_ptr = nullptr;
    uint16_t* sl_len = nullptr;
    int* sl_col = nullptr;
    double* sl_val64 = nullptr;
    float* sl_val32 = nullptr;
    int sl_ns = 0;
    long long sl_padded = 0;  // entries of the slices, padding included
    // K-cycle workspace in the handle's precision
    void *rhs = nullptr, *out = nullptr, *w = nullptr, *s = nullptr;
    void *c1 = nullptr, *v1 = nullptr, *rt = nullptr, *c2 = nullptr, *v2 = nullptr;
    LevelScalars* sc = nullptr;
};

// Device descriptor of one level for the fused small-level K-cycle (kern_tail.cu).
struct TailLevel {
    int n, inner;
    const int *rowptr, *col, *agg, *aggptr, *members;
    const void *val, *minv;
    void *rhs, *out, *w, *s, *c1, *v1, *rt, *c2, *v2;
};

constexpr int kTailMaxN = 8192;  // levels at most this large may run fused in one block

// R-column workspace of one level for uaamg_solve_many (interleaved [n][R]).
struct MultiLevel {
    void *rhs, *out, *w, *s, *c1, *v1, *rt, *c2, *v2;
    double* sc;  // per-column K-cycle scalars, 7 rows of R
};

struct ProfSlot {
    cudaEvent_t a, b;
};

struct Handle {
    int device = 0;
    int num_sms = 0;
    cudaStream_t user = nullptr;  // caller's stream
    cudaStream_t work = nullptr;  // the handle's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    uaamg_params p{};
    int nlev = 0;
    Level lev[kMaxLevels];
    double* coarse_inv = nullptr;  // dense inverse of the coarsest matrix (FP64)
    int nco = 0;
    // outer iteration vectors (FP64)
    double *b = nullptr, *x = nullptr, *r = nullptr, *p_ = nullptr, *q = nullptr;
    OuterScalars* osc = nullptr;
    OuterScalars* osc_host = nullptr;  // pinned mirror
    Ctrl* ctrl = nullptr;
    double* partials = nullptr;
    size_t partials_cap = 0;
    // fused small-level K-cycle: first level handled by k_tail (0 = none)
    int tail_level = 0;
    bool tail_cluster = false;  // the tail runs on a thread-block cluster (else one block)
    TailLevel* tail_dev = nullptr;
    // cluster tail: per-block regions of packed level data (tail_stride bytes apart, the
    // first tail_copy bytes of each staged at byte tail_vb of the block's shared memory),
    // blocks per cluster and dynamic shared memory per block
    void* tail_blob = nullptr;
    long long tail_stride = 0;
    int tail_copy = 0, tail_vb = 0, tail_cl = 0, tail_smem = 0;
    // uaamg_solve_many workspace (sized for multi_R columns) and its iteration graph
    int multi_R = 0;
    MultiLevel mlev[kMaxLevels];
    double *mb = nullptr, *mx = nullptr, *mr = nullptr, *mp = nullptr, *mq = nullptr;
    double* mos = nullptr;       // per-column outer scalars, 8 rows of R
    double* mos_host = nullptr;  // pinned mirror
    cudaGraphExec_t mgraph = nullptr;
    int mgraph_R = 0;
    long long mgraph_nodes = 0;
    // graph of one outer iteration
    cudaGraphExec_t graph = nullptr;
    long long graph_nodes = 0;
    // graph of the whole iteration loop (a while node around one iteration; the condition is
    // set on the device), its kernel count per iteration and the relative residual per
    // iteration it writes
    cudaGraphExec_t loop_graph = nullptr;
    long long loop_nodes = 0;
    double* d_hist = nullptr;
    int hist_cap = 0;
    // stats
    double setup_ms = 0, solve_ms = 0;
    long long launches = 0;
    std::vector<double> hist;
    // profiling
    int prof_class = 0;
    std::vector<ProfSlot> prof_slots;
    long long prof_launches = 0;
    double prof_ms = 0, prof_bytes = 0;
    // allocations
    std::vector<void*> allocs;
    std::vector<std::pair<void*, size_t>> temps;  // setup scratch, released when setup ends
    size_t bytes = 0;
    bool capturing = false;
};

// ---- host helpers (defined in runtime.cu) ------------------------------------------------
int check_cuda(cudaError_t e);
void* dalloc_bytes(Handle* h, size_t bytes, int* status, bool temp = false);
template <typename T>
T* dalloc(Handle* h, size_t count, int* status, bool temp = false) {
    return static_cast<T*>(dalloc_bytes(h, sizeof(T) * (count ? count : 1), status, temp));
}
// Releases one allocation of the handle made with dalloc_bytes(h, bytes) (stream-ordered).
void dfree_one(Handle* h, void* ptr, size_t bytes);
void dfree_temps(Handle* h);
void dfree_all(Handle* h);
void count_launch(Handle* h, long long k = 1);
int grid_for(long long items, int per_block);

// ---- device helpers ---------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A launch property (occupancy, an attribute set) computed once per device and read from
// any host thread (the solve service runs setups and solves on several threads).
struct DevCache {
    std::atomic<int> v[64];
    int get(int dev) const {
        return (dev >= 0 && dev < 64) ? v[dev].load(std::memory_order_relaxed) : 0;
    }
    void set(int dev, int x) {
        if (dev >= 0 && dev < 64) v[dev].store(x, std::memory_order_relaxed);
    }
};

// Programmatic dependent launch (small-level kernels): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor on the stream still
// runs; pdl_wait() blocks until that predecessor has completed and its writes are visible,
// and must precede every read of them.  pdl_trigger() lets this kernel's own successor
// start launching.  Both are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
constexpr int kPdlMaxRows = 65536;  // levels up to this size launch with the attribute

// Launch, with the programmatic-serialization attribute when `pdl`.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  The arrival counter
// only grows (the launcher zeroes it): the k-th barrier is passed once it reaches
// (k+1) * gridDim.x, so an arrival costs one atomic and no block has to reset or flip
// anything.  The wait polls with an acquire load, first back to back, then with a short
// sleep, and gives up (kErrTimeout, returns false) after the handle's wait limit
// (c->wait_ns, default kBarrierTimeoutNs) or as soon as another block has given up.  Limits
// below kFastPollNs are checked on every poll.
__device__ __forceinline__ bool grid_barrier(Ctrl* c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const long long lim0 = *(volatile long long*)&c->wait_ns;
        const long long lim = lim0 > 0 ? lim0 : kBarrierTimeoutNs;
        const bool fast = lim < kFastPollNs;
        const unsigned int arrived = atomicAdd(&c->bar_count, 1u);
        const unsigned int target = (arrived / gridDim.x + 1u) * gridDim.x;
        long long t0 = fast ? global_ns() : 0;
        int spins = 0;
        while ((int)(ld_acquire(&c->bar_count) - target) < 0) {
            if (!fast && ++spins < 64) continue;
            const long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > lim || (*(volatile int*)&c->err & kErrTimeout)) {
                atomicOr(&c->err, kErrTimeout);
                break;
            }
            if (!fast) __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return (*(volatile int*)&c->err & kErrTimeout) == 0;
}

// Deterministic reduction of ND per-thread values over the whole grid: each block reduces
// with a fixed tree and stores its partials; the last block to arrive adds the partials in
// block order and writes result[0..ND).  Every thread of every block must call it.  Returns
// true only in thread 0 of the last block, once result is written.
template <int ND>
__device__ __forceinline__ bool grid_reduce(const double (&v)[ND], double* partials,
                                            unsigned int* counter, double* result) {
    __shared__ double sh[ND][kThreads / 32];
    __shared__ bool is_last;
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
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[k][w];
            partials[(size_t)blockIdx.x * ND + k] = s;
        }
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) acc[k] = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < ND; k++) acc[k] += __ldcg(&partials[(size_t)b * ND + k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; k++) {
        double s = warp_sum(acc[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[k][w];
            result[k] = s;
        }
        *counter = 0u;
    }
    return threadIdx.x == 0;  // thread 0 of the last block, after result is written
}

// Rounded arithmetic without contraction, so that FP64 epilogues round exactly like the
// plain C statement of the method.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
// a * b + c with one rounding (one FP64 instruction instead of two on GB300's FP64 units)
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace uaamg
