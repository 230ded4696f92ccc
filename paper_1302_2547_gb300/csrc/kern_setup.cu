// kern_setup.cu -- kernels of the setup phase (Algorithm 1): CSR validation, priority
// vector (Eq. 3.2), parallel aggregation (Algorithm 2), ascending coarse numbering
// (Section 5.1), coarse operator by aggregate sums (Eq. 2.4), l1-Jacobi data (Section 4.1)
// and the dense inverse of the coarsest matrix.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

// ---------------------------------------------------------------------------------------
// CSR validation: every access is guarded, so a malformed matrix raises kErrBadCsr and
// never reads out of bounds.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_validate(int n, int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
           const double* __restrict__ val, Ctrl* ctrl) {
    const int stride = gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz))
        atomicOr(&ctrl->err, kErrBadCsr);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int k0 = rowptr[i], k1 = rowptr[i + 1];
        bool bad = !(0 <= k0 && k0 <= k1 && k1 <= nnz);
        bool diag = false;
        int prev = -1;
        for (int k = k0; !bad && k < k1; k++) {
            int c = col[k];
            double v = val[k];
            if (c < 0 || c >= n || c <= prev || !isfinite(v)) {
                bad = true;
                break;
            }
            prev = c;
            if (c == i) {
                diag = true;
                if (!(v > 0.0)) bad = true;
                continue;
            }
            // symmetric pattern and values: find (c, i)
            int lo = rowptr[c], hi = rowptr[c + 1];
            if (!(0 <= lo && lo <= hi && hi <= nnz)) {
                bad = true;
                break;
            }
            int hi0 = hi - 1;
            bool found = false;
            while (lo <= hi0) {
                int mid = (lo + hi0) >> 1;
                int cm = col[mid];
                if (cm == i) {
                    found = (val[mid] == v);
                    break;
                }
                if (cm < i) lo = mid + 1;
                else hi0 = mid - 1;
            }
            if (!found) bad = true;
        }
        if (bad || !diag) atomicOr(&ctrl->err, kErrBadCsr);
    }
}

int launch_validate(Handle* h, int n, int nnz, const int* rowptr, const int* col,
                    const double* val) {
    int g = grid_for(n, kThreads);
    if (g > 8 * h->num_sms) g = 8 * h->num_sms;
    k_validate<<<g, kThreads, 0, h->work>>>(n, nnz, rowptr, col, val, h->ctrl);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Priority vector, Eq. (3.2): v_i = d_i + ((i mod 12) + rand()) / 12 with rand() replaced
// by the MurmurHash3 32-bit finalizer of (i + salt), a bijection on 32-bit words, encoded
// as the integer P_i = ((12 d_i + (i mod 12) + 1) << 32) | h_i (unique, same order).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void __launch_bounds__(kThreads)
k_priority(int n, const int* __restrict__ rowptr, const int* __restrict__ col, uint32_t salt,
           uint64_t* __restrict__ prio) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k0 = rowptr[i], k1 = rowptr[i + 1];
    long long d = 0;
    for (int k = k0; k < k1; k++) d += (col[k] != i);
    uint64_t band = (uint64_t)(12 * d + (i % 12) + 1);
    prio[i] = (band << 32) | (uint64_t)fmix32((uint32_t)i + salt);
}

int launch_priority(Handle* h, int n, const int* rowptr, const int* col, uint32_t salt,
                    uint64_t* prio) {
    k_priority<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, rowptr, col, salt, prio);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Parallel aggregation, Algorithm 2: one kernel runs every pass of an aggregation.  A pass
// is (A) rounds of coarse-vertex selection and (B) star aggregation.  Single-round mode
// (the default) runs k_paa_sr<G> (cooperative, candidate worklists) or k_paa_sr_block (a
// small level in one block's shared memory), below; maximal mode runs k_paa or k_paa_small.
//
// Round of maximal mode (two sweeps, separated by grid barriers; the state array is a
// snapshot per sweep, so the result does not depend on thread order):
//   sweep 1, every vertex v: b1[v] = max priority of the candidates in N[v] (closed
//     neighbourhood), blocked[v] = N[v] contains a root of this pass;
//   sweep 2, every candidate v: if some u in N[v] is blocked, v is within distance 2 of a
//     root and leaves the pass; else v becomes a root iff max_{u in N[v]} b1[u] = P_v,
//     i.e. v beats every candidate within distance 2 (paths through any vertex).
// One-round mode stops after the first round (Algorithm 2 as printed); maximal mode
// repeats until no candidate remains, which yields the greedy maximal set in descending
// priority.  Roots are pairwise at distance >= 3 (Eq. 3.1), so in (B) each root takes its
// unprocessed neighbours (ascending, at most t-1) with no write conflicts.
// Reads of arrays written inside the kernel bypass L1 (ld.global.cg).
// ---------------------------------------------------------------------------------------
struct PaaArgs {
    int n;
    const int* rowptr;
    const int* col;
    const uint64_t* prio;
    uint8_t* state;
    uint64_t* b1;
    uint8_t* blocked;
    int* list;        // two candidate lists of n entries (single-round mode)
    uint64_t* cprio;  // n entries: priority while a candidate, else 0 (single-round mode)
    int* root_of;
    int* pass_of;
    int* agg_size;
    int t;
    int mode;
    int* slots;
    int nslots;
    Ctrl* ctrl;
    int handoff;  // grid kernel: hand the passes to the cluster kernel once a pass has at most
                  // this many candidates (0: never)
};

__device__ __forceinline__ uint8_t ld_state(const uint8_t* p) {
    return (uint8_t)__ldcg(reinterpret_cast<const unsigned char*>(p));
}

__device__ __forceinline__ int block_sum_int(int v) {
    __shared__ int sh[kThreads / 32];
    __shared__ int out;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kThreads / 32; w++) s += sh[w];
        out = s;
    }
    __syncthreads();
    int r = out;
    __syncthreads();
    return r;
}

// Single-round passes (Algorithm 2 as printed) on candidate worklists, one cooperative
// kernel per aggregation.  Pass p needs b1 of every vertex next to a candidate; two b1
// buffers alternate between passes.
//   pull pass (pass 0, and while the candidates are many): every vertex w computes
//     b1[w] = max priority of the candidates in N[w] into the current buffer and clears
//     the other one;
//   push pass: each vertex w of the previous pass's list clears the old buffer at N[w]
//     (exactly the entries that pass made nonzero) and, if still a candidate, raises the
//     current buffer at N[w] to P_w with atomicMax.
// Both build the list of this pass's candidates (warp-aggregated appends; its order does
// not matter).  Then every listed candidate v becomes a root iff max_{u in N[v]} b1[u] = P_v
// and takes its neighbours at once.  Fusing selection and aggregation is safe: a neighbour
// w of a root v is never a root itself (P_v > P_w within distance 2) and no other root
// reaches it (roots are >= 3 apart), so w has a single writer.
// On small levels the sweeps are latency-bound chains (col -> state -> priority), so G
// lanes share a vertex, one neighbour each, and the grid holds about one vertex per group:
// a row of up to G entries costs one chain.  Large levels use G = 1.  Arrays written
// inside the kernel are read through L2.
constexpr int kPullDiv = 4;  // pull while more than n / kPullDiv candidates remain

// Maximum over the G lanes of a vertex's group; every lane of the warp takes part.
template <int G>
__device__ __forceinline__ uint64_t group_max(uint64_t x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o, G);
        x = y > x ? y : x;
    }
    return x;
}

constexpr int kPaaThreads = 1024;  // large blocks: fewer arrivals at each grid barrier

constexpr int kPaaBatch = 4;  // neighbour steps whose loads are issued together

// Once a pass has few candidates, a pass is a chain of dependent L2 round trips plus two
// barriers, and a barrier over the whole grid costs several times one over a cluster of
// 16 SMs.  So the cooperative grid kernel (CL = false) hands the remaining passes to the
// same kernel launched as one thread-block cluster (CL = true), which synchronises with
// cluster barriers (release / acquire at cluster scope order the global-memory state).
// The hand-off leaves ctrl->npasses = -(next pass + 1); the cluster kernel resumes there,
// or returns at once when the grid kernel finished (npasses >= 0) or failed.
__device__ __forceinline__ void paa_cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <bool CL>
__device__ __forceinline__ bool paa_barrier(Ctrl* ctrl) {
    if constexpr (CL) {
        paa_cluster_barrier();
        return true;
    } else {
        return grid_barrier(ctrl);
    }
}

template <int G, bool CL>
__global__ void __launch_bounds__(kPaaThreads, CL ? 1 : 2) k_paa_sr(PaaArgs a) {
    const int n = a.n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    // cp[v] = P_v while v is a candidate, 0 once aggregated: one load answers both "is it a
    // candidate" and "with what priority"
    unsigned long long* cp = reinterpret_cast<unsigned long long*>(a.cprio);
    int prev_cnt = n, pass = 0;
    if constexpr (CL) {  // resume where the grid kernel handed off (uniform over the cluster)
        const int np = *(volatile const int*)&a.ctrl->npasses;
        if (np >= 0 || *(volatile const int*)&a.ctrl->err) return;
        pass = -np - 1;
        prev_cnt = *(volatile const int*)&a.slots[pass - 1];
    } else {
        for (int v = tid; v < n; v += nthreads) {
            cp[v] = a.prio[v];
            a.root_of[v] = -1;
            a.pass_of[v] = -1;
        }
        if (!grid_barrier(a.ctrl)) return;
    }
    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);  // lane within the vertex's group
    const int gw = lane / G;         // group within the warp
    const unsigned gmask = (unsigned)((1ull << G) - 1ull) << (gw * G);
    const int wbase = (tid - lane) / G;  // this warp's first group
    const int gstride = nthreads / G;
    while (true) {
        uint64_t* bcur = a.b1 + (size_t)(pass & 1) * n;
        uint64_t* bold = a.b1 + (size_t)((pass + 1) & 1) * n;
        int* cur = a.list + (size_t)(pass & 1) * n;
        const int* prev = a.list + (size_t)((pass + 1) & 1) * n;
        const bool pull = pass == 0 || (long long)prev_cnt * kPullDiv > n;
        const int span = pull ? n : prev_cnt;
        for (int q0 = wbase; q0 < span; q0 += gstride) {  // uniform over the warp
            const int q = q0 + gw;
            const bool valid = q < span;
            const int w = valid ? (pull ? q : __ldcg(prev + q)) : 0;
            const int k0 = valid ? a.rowptr[w] : 0, k1 = valid ? a.rowptr[w + 1] : 0;
            const unsigned long long pw = valid ? __ldcg(cp + w) : 0ull;
            const bool cand = pw != 0ull;
            const unsigned m = __ballot_sync(0xffffffffu, cand && sub == 0);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&a.slots[pass], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (cand && sub == 0) cur[base + __popc(m & ((1u << lane) - 1u))] = w;
            const unsigned steps = __reduce_max_sync(0xffffffffu, (unsigned)(k1 - k0 + G - 1) / G);
            uint64_t best = 0;
            for (unsigned c0 = 0; c0 < steps; c0 += kPaaBatch) {
                int u[kPaaBatch];
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++) {
                    const int k = k0 + (int)(c0 + b) * G + sub;
                    u[b] = (c0 + b < steps && k < k1) ? a.col[k] : -1;
                }
                if (pull) {
                    unsigned long long pu[kPaaBatch];
#pragma unroll
                    for (int b = 0; b < kPaaBatch; b++) pu[b] = u[b] >= 0 ? __ldcg(cp + u[b]) : 0ull;
#pragma unroll
                    for (int b = 0; b < kPaaBatch; b++) best = pu[b] > best ? pu[b] : best;
                } else {
#pragma unroll
                    for (int b = 0; b < kPaaBatch; b++) {
                        if (u[b] < 0) continue;
                        bold[u[b]] = 0;
                        if (cand) atomicMax(reinterpret_cast<unsigned long long*>(bcur + u[b]), pw);
                    }
                }
            }
            if (pull) {
                best = group_max<G>(best);
                if (valid && sub == 0) {
                    bcur[w] = best;
                    bold[w] = 0;
                }
            }
        }
        if (!paa_barrier<CL>(a.ctrl)) return;
        const int cnt = *(volatile int*)&a.slots[pass];
        if (cnt == 0) break;
        for (int q0 = wbase; q0 < cnt; q0 += gstride) {
            const int q = q0 + gw;
            const bool valid = q < cnt;
            const int v = valid ? __ldcg(cur + q) : 0;
            const int k0 = valid ? a.rowptr[v] : 0, k1 = valid ? a.rowptr[v + 1] : 0;
            const unsigned steps = __reduce_max_sync(0xffffffffu, (unsigned)(k1 - k0 + G - 1) / G);
            uint64_t mx = 0;
            for (unsigned c0 = 0; c0 < steps; c0 += kPaaBatch) {
                int u[kPaaBatch];
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++) {
                    const int k = k0 + (int)(c0 + b) * G + sub;
                    u[b] = (c0 + b < steps && k < k1) ? a.col[k] : -1;
                }
                unsigned long long bu[kPaaBatch];
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++)
                    bu[b] = u[b] >= 0 ? __ldcg(reinterpret_cast<const unsigned long long*>(bcur + u[b])) : 0ull;
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++) mx = bu[b] > mx ? bu[b] : mx;
            }
            mx = group_max<G>(mx);
            const bool root = valid && mx == a.prio[v];
            if (!__any_sync(0xffffffffu, root)) continue;
            // v's star aggregate: its unprocessed neighbours in ascending order, at most t-1;
            // the group ranks each step's takers by lane, which keeps the stored order
            int taken = 1;
            for (unsigned c0 = 0; c0 < steps; c0 += kPaaBatch) {
                int u[kPaaBatch];
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++) {
                    const int k = k0 + (int)(c0 + b) * G + sub;
                    u[b] = (root && c0 + b < steps && k < k1) ? a.col[k] : -1;
                }
                bool take[kPaaBatch];
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++)
                    take[b] = u[b] >= 0 && u[b] != v && __ldcg(cp + u[b]) != 0ull;
#pragma unroll
                for (int b = 0; b < kPaaBatch; b++) {
                    const unsigned bm = __ballot_sync(0xffffffffu, take[b]) & gmask;
                    const int room = a.t > 0 ? a.t - taken : 0x7fffffff;
                    if (take[b] && __popc(bm & ((1u << lane) - 1u)) < room) {
                        a.root_of[u[b]] = v;
                        a.pass_of[u[b]] = pass;
                        cp[u[b]] = 0ull;
                    }
                    taken += min(__popc(bm), room);
                }
            }
            if (root && sub == 0) {
                a.root_of[v] = v;
                a.pass_of[v] = pass;
                a.agg_size[v] = taken;
                cp[v] = 0ull;
            }
        }
        if (!paa_barrier<CL>(a.ctrl)) return;
        prev_cnt = cnt;
        if (++pass >= a.nslots) {
            if (tid == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
        if (!CL && a.handoff > 0 && cnt <= a.handoff) {  // uniform: cnt is read after a barrier
            if (tid == 0) a.ctrl->npasses = -(pass + 1);
            return;
        }
    }
    if (tid == 0) a.ctrl->npasses = pass;
}

// The same single-round passes for a small level in one thread block, with the level's CSR
// (column indices as 16-bit when they fit), the candidate priorities cp and b1 staged in
// shared memory: a pass is two shared-memory sweeps over every vertex and two block
// barriers, where the grid version pays L2 round trips and grid barriers.  The sweeps
// read cp snapshots exactly as the grid version does: a vertex whose cp is cleared by a
// root during sweep 2 has that root within distance 1, so it is not a root either way.
// One SM's issue rate caps this version: it beats the grid kernel up to about a thousand
// vertices (measured: 225 vertices 1.7 vs 6.0 us per pass; 2817 vertices 18 vs 7.7 us).
constexpr int kPaaBlockThreads = 1024;
constexpr int kPaaBlockMaxN = 1024;
constexpr size_t kPaaBlockSmem = 200 * 1024;

template <typename C>
static size_t paa_block_bytes(long long n, long long nnz) {
    const size_t b = 16 * (size_t)n;                           // b1 and cp
    const size_t r = (4 * (size_t)(n + 1) + 15) & ~(size_t)15;  // rowptr
    return b + r + sizeof(C) * (size_t)nnz;
}

template <typename C>
__global__ void __launch_bounds__(kPaaBlockThreads, 1) k_paa_sr_block(PaaArgs a) {
    extern __shared__ __align__(16) unsigned char dyn[];
    const int n = a.n;
    unsigned long long* b1 = reinterpret_cast<unsigned long long*>(dyn);
    unsigned long long* cp = b1 + n;
    int* rp = reinterpret_cast<int*>(cp + n);
    C* cl = reinterpret_cast<C*>(dyn + 16 * (size_t)n + ((4 * (size_t)(n + 1) + 15) & ~(size_t)15));
    const int t = threadIdx.x, T = blockDim.x;
    const int nnz = a.rowptr[n];
    for (int v = t; v <= n; v += T) rp[v] = a.rowptr[v];
    for (int k = t; k < nnz; k += T) cl[k] = (C)a.col[k];
    for (int v = t; v < n; v += T) {
        cp[v] = a.prio[v];
        a.root_of[v] = -1;
        a.pass_of[v] = -1;
    }
    __syncthreads();
    int pass = 0;
    while (true) {
        // sweep 1: b1[v] = max cp over N[v]; count the candidates
        int cnt = 0;
        for (int v = t; v < n; v += T) {
            unsigned long long best = 0;
            for (int k = rp[v]; k < rp[v + 1]; k++) {
                const unsigned long long pu = cp[cl[k]];
                best = pu > best ? pu : best;
            }
            b1[v] = best;
            cnt += cp[v] != 0ull;
        }
        if (__syncthreads_count(cnt) == 0) break;
        // sweep 2: a candidate whose priority tops max b1 over N[v] is a root and takes its
        // unprocessed neighbours in ascending order, at most t-1
        for (int v = t; v < n; v += T) {
            const unsigned long long pv = cp[v];
            if (pv == 0ull) continue;
            unsigned long long m = 0;
            const int k0 = rp[v], k1 = rp[v + 1];
            for (int k = k0; k < k1; k++) {
                const unsigned long long bu = b1[cl[k]];
                m = bu > m ? bu : m;
            }
            if (m != pv) continue;
            int taken = 1;
            for (int k = k0; k < k1; k++) {
                const int u = (int)cl[k];
                if (u == v) continue;
                if (a.t > 0 && taken >= a.t) break;
                if (cp[u] != 0ull) {
                    a.root_of[u] = v;
                    a.pass_of[u] = pass;
                    cp[u] = 0ull;
                    taken++;
                }
            }
            a.root_of[v] = v;
            a.pass_of[v] = pass;
            a.agg_size[v] = taken;
            cp[v] = 0ull;
        }
        __syncthreads();
        if (++pass >= a.nslots) {
            if (t == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
    }
    if (t == 0) a.ctrl->npasses = pass;
}

// The same single-round passes on one thread-block cluster (levels of at most kPaaClMaxN
// vertices whose data fit): block c owns the vertices [c chunk, (c + 1) chunk).  Every block
// keeps full copies of cp and b1 and its own rows of the CSR (16-bit columns) in its shared
// memory, so both sweeps read shared memory only; a block writes an entry into every block's
// copy (distributed shared memory) only where it changes (b1 of its own vertices, cp of the
// vertices its roots aggregate), a few entries per pass on these levels.  Cluster barriers
// (release / acquire) separate the sweeps; each block's candidate count goes to every block
// before the first, so every thread reads the total locally.  The sweeps read the same
// snapshots as the grid version, so the passes, roots and aggregates are identical.
constexpr int kPaaClThreads = 1024;
constexpr int kPaaClMaxN = 12800;
constexpr int kPaaClSmem = 220 * 1024;  // dynamic shared memory of a block, at most

__device__ __forceinline__ uint32_t paa_map(const void* p, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void paa_bcast(unsigned long long* p, unsigned long long v, int C) {
    for (int r = 0; r < C; r++)
        asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(paa_map(p, r)), "l"(v) : "memory");
}
__device__ __forceinline__ void paa_bcast(int* p, int v, int C) {
    for (int r = 0; r < C; r++)
        asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(paa_map(p, r)), "r"(v) : "memory");
}
__device__ __forceinline__ void paa_st(int* p, int rank, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(paa_map(p, rank)), "r"(v) : "memory");
}
constexpr int kPaaClBatch = 8;  // entries whose loads a lane issues together

// max over the lane's entries k0 + sub, k0 + sub + G, ... < k1 of x[col[k]], the column
// loads of kPaaClBatch entries issued together, then their gathers
template <int G, typename CI>
__device__ __forceinline__ unsigned long long paa_row_max(const CI* col, int k0, int k1, int sub,
                                                          const unsigned long long* x) {
    unsigned long long best = 0;
    for (int k = k0 + sub; k < k1; k += G * kPaaClBatch) {
        int u[kPaaClBatch];
#pragma unroll
        for (int b = 0; b < kPaaClBatch; b++) u[b] = k + b * G < k1 ? (int)col[k + b * G] : -1;
#pragma unroll
        for (int b = 0; b < kPaaClBatch; b++) {
            const unsigned long long v = u[b] >= 0 ? x[u[b]] : 0ull;
            best = v > best ? v : best;
        }
    }
    return best;
}

// Updates a block queues per sweep before all its threads write them into every block
// (a single thread writing one entry into 16 blocks serialises 16 remote stores).
__host__ __device__ inline int paa_cl_evcap(int chunk) { return 2 * chunk + 64; }

// Bytes of dynamic shared memory for a level (cp and b1; the two update queues; root, pass
// and aggregate size of the block's vertices; its row offsets; up to `ecap` entries of its
// rows).
__host__ __device__ inline size_t paa_cl_bytes(int n, int chunk, int ecap) {
    return 16 * (size_t)n + 20 * (size_t)paa_cl_evcap(chunk) + 12 * (size_t)chunk +
           4 * (size_t)(chunk + 1) + ((2 * (size_t)ecap + 15) & ~(size_t)15);
}

template <int G>
__global__ void __launch_bounds__(kPaaClThreads, 1) k_paa_cl(PaaArgs a, int chunk, int ecap) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int s_cnt[kPaaClThreads / 32];
    __shared__ int s_part[16];  // the blocks' candidates of the pass, written by each block
    __shared__ int s_nq1, s_nq2;  // queued updates of sweep 1 and sweep 2
    const int n = a.n;
    unsigned long long* cp = reinterpret_cast<unsigned long long*>(dyn);
    unsigned long long* b1 = cp + n;
    const int qcap = paa_cl_evcap(chunk);
    unsigned long long* q1b = b1 + n;  // sweep 1: new b1 value of vertex q1w
    int* q1w = reinterpret_cast<int*>(q1b + qcap);
    int* q2u = q1w + qcap;  // sweep 2: vertex q2u joins the aggregate of root q2v
    int* q2v = q2u + qcap;
    // the block's vertices' root, pass and aggregate size, written to global memory at the
    // end: global stores before a release barrier would make it wait for their completion
    int* ro = q2v + qcap;
    int* po = ro + chunk;
    int* as = po + chunk;
    int* rp = as + chunk;  // this block's row offsets
    uint16_t* cl = reinterpret_cast<uint16_t*>(rp + chunk + 1);
    const int C = (int)gridDim.x, rank = (int)blockIdx.x;  // the grid is one cluster
    const int t = threadIdx.x;
    const int r0 = min(rank * chunk, n), r1 = min(r0 + chunk, n), rows = r1 - r0;
    const int e0 = a.rowptr[r0], E = a.rowptr[r1] - e0;
    // a block whose rows exceed the capacity the host sized reads them from global memory
    const bool staged = E <= ecap;
    const int* gcl = a.col + e0;
    for (int v = t; v < n; v += kPaaClThreads) {
        cp[v] = a.prio[v];
        b1[v] = 0ull;
    }
    for (int i = t; i <= rows; i += kPaaClThreads) rp[i] = a.rowptr[r0 + i] - e0;
    if (staged)
        for (int k = t; k < E; k += kPaaClThreads) cl[k] = (uint16_t)a.col[e0 + k];
    for (int i = t; i < rows; i += kPaaClThreads) {
        ro[i] = -1;
        po[i] = -1;
    }
    if (t == 0) s_nq1 = s_nq2 = 0;
    paa_cluster_barrier();  // every block's copies exist before any block writes into them
    const int lane = t & 31, sub = lane & (G - 1);
    const int g0 = t / G, gs = kPaaClThreads / G;  // this thread's group, groups per block
    const int wg = g0 % (32 / G);                   // group within the warp
    int pass = 0;
    while (true) {
        // sweep 1: b1[w] = max cp over N[w] for this block's w; count its candidates
        int cnt = 0;
        for (int q0 = g0 - wg; q0 < rows; q0 += gs) {  // uniform over the warp
            const int q = q0 + wg;
            const bool valid = q < rows;
            const int k0 = valid ? rp[q] : 0, k1 = valid ? rp[q + 1] : 0;
            unsigned long long best = staged ? paa_row_max<G>(cl, k0, k1, sub, cp)
                                             : paa_row_max<G>(gcl, k0, k1, sub, cp);
            best = group_max<G>(best);
            if (valid && sub == 0) {
                const int w = r0 + q;
                if (best != b1[w]) {
                    const int e = atomicAdd(&s_nq1, 1);
                    if (e < qcap) {
                        q1w[e] = w;
                        q1b[e] = best;
                    } else {
                        paa_bcast(b1 + w, best, C);
                    }
                }
                cnt += cp[w] != 0ull;
            }
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) s_cnt[t >> 5] = cnt;
        __syncthreads();
        if (t < 32) {
            int c = s_cnt[t];
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (t == 0) paa_bcast(&s_part[rank], c, C);
        }
        {  // the queued b1 updates, one (entry, block) pair per thread
            const int nq = min(s_nq1, qcap);
            for (int j = t; j < nq * C; j += kPaaClThreads) {
                const int e = j / C, r = j - e * C;
                asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(paa_map(b1 + q1w[e], r)),
                             "l"(q1b[e])
                             : "memory");
            }
        }
        paa_cluster_barrier();
        if (t == 0) s_nq1 = 0;  // (sweep 1 of the next pass follows the next barrier)
        int tot = 0;
        for (int r = 0; r < C; r++) tot += s_part[r];
        if (t == 0 && rank == 0) a.slots[pass] = tot;
        if (tot == 0) break;
        // sweep 2: a candidate whose priority tops max b1 over N[v] is a root and takes its
        // unprocessed neighbours in ascending order, at most t-1
        for (int q0 = g0 - wg; q0 < rows; q0 += gs) {
            const int q = q0 + wg;
            const int v = r0 + q;
            const unsigned long long pv = q < rows ? cp[v] : 0ull;
            const int k0 = pv ? rp[q] : 0, k1 = pv ? rp[q + 1] : 0;
            unsigned long long m = staged ? paa_row_max<G>(cl, k0, k1, sub, b1)
                                          : paa_row_max<G>(gcl, k0, k1, sub, b1);
            m = group_max<G>(m);
            if (!(pv != 0ull && m == pv && sub == 0)) continue;
            int taken = 1;
            for (int k = k0; k < k1; k++) {
                const int u = staged ? (int)cl[k] : __ldg(gcl + k);
                if (u == v) continue;
                if (a.t > 0 && taken >= a.t) break;
                if (cp[u] != 0ull) {
                    const int e = atomicAdd(&s_nq2, 1);
                    if (e < qcap) {
                        q2u[e] = u;
                        q2v[e] = v;
                    } else {
                        const int o = u / chunk, iu = u - o * chunk;  // u's block and row there
                        paa_st(ro + iu, o, v);
                        paa_st(po + iu, o, pass);
                        paa_bcast(cp + u, 0ull, C);
                    }
                    taken++;
                }
            }
            ro[q] = v;
            po[q] = pass;
            as[q] = taken;
            const int e = atomicAdd(&s_nq2, 1);
            if (e < qcap) {
                q2u[e] = v;
                q2v[e] = -1;  // the root itself: cp only
            } else {
                paa_bcast(cp + v, 0ull, C);
            }
        }
        __syncthreads();
        {  // the queued updates: cp = 0 in every block, root and pass in the owner's block
            const int nq = min(s_nq2, qcap);
            for (int j = t; j < nq * C; j += kPaaClThreads) {
                const int e = j / C, r = j - e * C;
                const int u = q2u[e];
                asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(paa_map(cp + u, r)), "l"(0ull)
                             : "memory");
                const int o = u / chunk;
                if (r == o && q2v[e] >= 0) {
                    paa_st(ro + (u - o * chunk), o, q2v[e]);
                    paa_st(po + (u - o * chunk), o, pass);
                }
            }
        }
        paa_cluster_barrier();
        if (t == 0) s_nq2 = 0;  // (sweep 2 of the next pass follows the next barrier)
        if (++pass >= a.nslots) {
            if (t == 0 && rank == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
    }
    // every write into this block's ro / po preceded the last barrier
    for (int i = t; i < rows; i += kPaaClThreads) {
        a.root_of[r0 + i] = ro[i];
        a.pass_of[r0 + i] = po[i];
        if (ro[i] == r0 + i) a.agg_size[r0 + i] = as[i];
    }
    if (t == 0 && rank == 0) a.ctrl->npasses = pass;
}

// Maximal mode: every vertex per sweep, rounds of coarse-vertex selection then aggregation.
__global__ void __launch_bounds__(kThreads) k_paa(PaaArgs a) {
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int gs = gridDim.x * blockDim.x;
    for (int v = g0; v < a.n; v += gs) {
        a.state[v] = ST_CAND;
        a.root_of[v] = -1;
        a.pass_of[v] = -1;
    }
    if (!grid_barrier(a.ctrl)) return;
    int slot = 0, pass = 0;
    while (true) {
        // (A) coarse vertices of this pass
        while (true) {
            for (int v = g0; v < a.n; v += gs) {
                const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
                uint64_t best = 0;
                int blk = 0;
                for (int k = k0; k < k1; k++) {
                    const int u = a.col[k];
                    const uint8_t s = ld_state(a.state + u);
                    blk |= (s == ST_ROOT);
                    if (s == ST_CAND) {
                        const uint64_t pu = a.prio[u];
                        best = pu > best ? pu : best;
                    }
                }
                a.b1[v] = best;
                a.blocked[v] = (uint8_t)blk;
            }
            if (!grid_barrier(a.ctrl)) return;
            int cnt = 0;
            for (int v = g0; v < a.n; v += gs) {
                if (ld_state(a.state + v) != ST_CAND) continue;
                const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
                uint64_t m = 0;
                int blk = 0;
                for (int k = k0; k < k1; k++) {
                    const int u = a.col[k];
                    blk |= ld_state(a.blocked + u);
                    const uint64_t bu = __ldcg(reinterpret_cast<const unsigned long long*>(a.b1 + u));
                    m = bu > m ? bu : m;
                }
                if (blk) a.state[v] = ST_EXCL;
                else if (m == a.prio[v]) a.state[v] = ST_ROOT;
                else cnt++;
            }
            cnt = block_sum_int(cnt);
            if (threadIdx.x == 0 && cnt) atomicAdd(&a.slots[slot], cnt);
            if (!grid_barrier(a.ctrl)) return;
            const int remaining = *(volatile int*)&a.slots[slot];
            slot++;
            if (slot >= a.nslots) {
                if (g0 == 0) atomicOr(&a.ctrl->err, kErrSlots);
                return;
            }
            if (remaining == 0 || a.mode == UAAMG_PASS_SINGLE_ROUND) break;
        }
        // (B) star aggregates around the roots of this pass
        for (int v = g0; v < a.n; v += gs) {
            if (ld_state(a.state + v) != ST_ROOT) continue;
            const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
            int taken = 1;
            for (int k = k0; k < k1; k++) {
                const int u = a.col[k];
                if (u == v) continue;
                if (a.t > 0 && taken >= a.t) break;
                const uint8_t s = ld_state(a.state + u);
                if (s == ST_CAND || s == ST_EXCL) {
                    a.root_of[u] = v;
                    a.pass_of[u] = pass;
                    a.state[u] = ST_DONE;
                    taken++;
                }
            }
            a.root_of[v] = v;
            a.pass_of[v] = pass;
            a.agg_size[v] = taken;
            a.state[v] = ST_DONE;
        }
        if (!grid_barrier(a.ctrl)) return;
        // end of pass: unprocessed vertices become candidates of the next pass
        int cnt = 0;
        for (int v = g0; v < a.n; v += gs) {
            const uint8_t s = ld_state(a.state + v);
            if (s == ST_EXCL) a.state[v] = ST_CAND;
            cnt += (s == ST_EXCL || s == ST_CAND);
        }
        cnt = block_sum_int(cnt);
        if (threadIdx.x == 0 && cnt) atomicAdd(&a.slots[slot], cnt);
        if (!grid_barrier(a.ctrl)) return;
        const int remaining = *(volatile int*)&a.slots[slot];
        slot++;
        pass++;
        if (remaining == 0) break;
        if (slot >= a.nslots) {
            if (g0 == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
    }
    if (g0 == 0) a.ctrl->npasses = pass;
}

// The same passes for a small level in one thread block: the vertex states and b1 live in
// shared memory ("staged in shared memory"), and __syncthreads replaces the grid barriers,
// which on levels of a few thousand vertices cost more than the sweeps themselves.
constexpr int kPaaSmallN = 8192;
constexpr int kPaaSmallThreads = 1024;

__device__ __forceinline__ int block_sum_big(int v, int* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kPaaSmallThreads, 1) k_paa_small(PaaArgs a) {
    extern __shared__ __align__(16) unsigned char dyn[];
    uint64_t* b1 = reinterpret_cast<uint64_t*>(dyn);
    uint8_t* state = dyn + sizeof(uint64_t) * kPaaSmallN;
    uint8_t* blocked = state + kPaaSmallN;
    __shared__ int red[kPaaSmallThreads / 32];
    const int t = threadIdx.x, T = blockDim.x;
    for (int v = t; v < a.n; v += T) {
        state[v] = ST_CAND;
        a.root_of[v] = -1;
        a.pass_of[v] = -1;
    }
    __syncthreads();
    int pass = 0, rounds = 0;
    while (true) {
        // maximal set per pass: rounds until no candidate remains, then aggregation
        while (true) {
            for (int v = t; v < a.n; v += T) {
                uint64_t best = 0;
                int blk = 0;
                for (int k = a.rowptr[v]; k < a.rowptr[v + 1]; k++) {
                    const int u = a.col[k];
                    const uint8_t s = state[u];
                    blk |= (s == ST_ROOT);
                    if (s == ST_CAND) {
                        const uint64_t pu = a.prio[u];
                        best = pu > best ? pu : best;
                    }
                }
                b1[v] = best;
                blocked[v] = (uint8_t)blk;
            }
            __syncthreads();
            int cnt = 0;
            for (int v = t; v < a.n; v += T) {
                if (state[v] != ST_CAND) continue;
                uint64_t m = 0;
                int blk = 0;
                for (int k = a.rowptr[v]; k < a.rowptr[v + 1]; k++) {
                    const int u = a.col[k];
                    blk |= blocked[u];
                    m = b1[u] > m ? b1[u] : m;
                }
                if (blk) state[v] = ST_EXCL;
                else if (m == a.prio[v]) state[v] = ST_ROOT;
                else cnt++;
            }
            const int remaining = block_sum_big(cnt, red);
            if (++rounds >= a.nslots) {
                if (t == 0) atomicOr(&a.ctrl->err, kErrSlots);
                return;
            }
            if (remaining == 0) break;
        }
        for (int v = t; v < a.n; v += T) {
            if (state[v] != ST_ROOT) continue;
            int taken = 1;
            for (int k = a.rowptr[v]; k < a.rowptr[v + 1]; k++) {
                const int u = a.col[k];
                if (u == v) continue;
                if (a.t > 0 && taken >= a.t) break;
                const uint8_t s = state[u];
                if (s == ST_CAND || s == ST_EXCL) {
                    a.root_of[u] = v;
                    a.pass_of[u] = pass;
                    state[u] = ST_DONE;
                    taken++;
                }
            }
            a.root_of[v] = v;
            a.pass_of[v] = pass;
            a.agg_size[v] = taken;
            state[v] = ST_DONE;
        }
        __syncthreads();
        int cnt = 0;
        for (int v = t; v < a.n; v += T) {
            const uint8_t s = state[v];
            if (s == ST_EXCL) state[v] = ST_CAND;
            cnt += (s == ST_EXCL || s == ST_CAND);
        }
        if (block_sum_big(cnt, red) == 0) {
            pass++;
            break;
        }
        pass++;
        if (++rounds >= a.nslots) {
            if (t == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
    }
    if (t == 0) a.ctrl->npasses = pass;
}

constexpr int kPaaLanesMaxN = 32768;  // largest level that shares lanes over a row

constexpr int kPaaHandoff = 2048;  // candidates of a pass at which the cluster kernel takes over

// Blocks of the cluster that continues the passes (16 where the device runs such a
// cluster of k_paa_sr<G, true>, else 8, else 0: no hand-off).
template <int G>
static int paa_cluster_blocks(int device) {
    static DevCache cache;  // blocks + 1
    int v = cache.get(device);
    if (!v) {
        int c = 0;
        for (int want : {16, 8}) {
            if (want > 8 && cudaFuncSetAttribute(k_paa_sr<G, true>,
                                                 cudaFuncAttributeNonPortableClusterSizeAllowed,
                                                 1) != cudaSuccess)
                continue;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(want);
            cfg.blockDim = dim3(kPaaThreads);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = want;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_paa_sr<G, true>, &cfg) == cudaSuccess && nc >= 1) {
                c = want;
                break;
            }
        }
        cudaGetLastError();
        v = c + 1;
        cache.set(device, v);
    }
    return v - 1;
}

// The cooperative grid kernel, then (where the device runs the cluster) the cluster kernel
// that takes over once a pass has at most kPaaHandoff candidates; the cluster kernel returns
// at once when the grid kernel finished.  Counts its launches.
template <int G>
static int launch_paa_sr(Handle* h, const PaaArgs& a0, int* grid) {
    static DevCache occ;
    int blocks_per_sm = occ.get(h->device);
    if (!blocks_per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_paa_sr<G, false>,
                                                          kPaaThreads, 0) != cudaSuccess ||
            blocks_per_sm < 1)
            blocks_per_sm = 1;
        occ.set(h->device, blocks_per_sm);
    }
    *grid = blocks_per_sm * h->num_sms;
    const int need = grid_for((long long)a0.n * G, kPaaThreads);
    if (*grid > need) *grid = need;
    const int C = paa_cluster_blocks<G>(h->device);
    PaaArgs a = a0;
    a.handoff = C ? kPaaHandoff : 0;
    int st = check_cuda(cudaMemsetAsync(&h->ctrl->npasses, 0, sizeof(int), h->work));
    if (st) return st;
    void* args[] = {&a};
    st = check_cuda(cudaLaunchCooperativeKernel((const void*)k_paa_sr<G, false>, dim3(*grid),
                                                dim3(kPaaThreads), args, 0, h->work));
    count_launch(h);
    if (st || !C) return st;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kPaaThreads);
    cfg.stream = h->work;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    a.handoff = 0;
    st = check_cuda(cudaLaunchKernelEx(&cfg, k_paa_sr<G, true>, a));
    count_launch(h);
    return st;
}

// Blocks of the cluster for k_paa_cl (16 where the device runs such a cluster with the
// largest shared memory, else 8, else 0) and the attributes, once per device.
static int paa_cl_blocks(int device) {
    static DevCache cache;  // blocks + 1
    int v = cache.get(device);
    if (!v) {
        const int smem = kPaaClSmem;
        int c = 0;
        bool ok = true;
        auto attrs = [&](auto k) {
            ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                           cudaSuccess;
            cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        };
        attrs(k_paa_cl<1>);
        attrs(k_paa_cl<2>);
        attrs(k_paa_cl<4>);
        attrs(k_paa_cl<8>);
        attrs(k_paa_cl<16>);
        attrs(k_paa_cl<32>);
        for (int want : {16, 8}) {
            if (!ok) break;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(want);
            cfg.blockDim = dim3(kPaaClThreads);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = want;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_paa_cl<1>, &cfg) == cudaSuccess && nc >= 1) {
                c = want;
                break;
            }
        }
        cudaGetLastError();
        v = c + 1;
        cache.set(device, v);
    }
    return v - 1;
}

// Entry capacity of a block's rows for k_paa_cl: twice the mean share (rows of these levels
// are within a small factor of the mean length), limited by the shared memory; 0 when the
// level does not fit.
static int paa_cl_ecap(int n, long long nnz, int C) {
    const int chunk = (n + C - 1) / C;
    long long ecap = 2 * ((nnz + C - 1) / C) + 256;
    if (ecap > nnz) ecap = nnz;
    const size_t fixed = paa_cl_bytes(n, chunk, 0);
    if (fixed >= (size_t)kPaaClSmem) return 0;
    const long long room = ((long long)kPaaClSmem - (long long)fixed) / 2;
    if (ecap > room) return 0;  // would not fit with the bound: the grid kernel runs instead
    return (int)ecap;
}

// k_paa_cl on a cluster of C blocks, G lanes per vertex: as many lanes as leave every block's
// vertices one group each, up to the mean row length.
static int launch_paa_cl(Handle* h, const PaaArgs& a, long long nnz, int C, int ecap) {
    const int chunk = (a.n + C - 1) / C;
    const long long avg = a.n > 0 ? (nnz + a.n - 1) / a.n : 1;
    int G = 1;
    while (G < 32 && (long long)chunk * G * 2 <= kPaaClThreads && G * 2 <= avg) G *= 2;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kPaaClThreads);
    cfg.dynamicSmemBytes = paa_cl_bytes(a.n, chunk, ecap);
    cfg.stream = h->work;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    switch (G) {
        case 1: e = cudaLaunchKernelEx(&cfg, k_paa_cl<1>, a, chunk, ecap); break;
        case 2: e = cudaLaunchKernelEx(&cfg, k_paa_cl<2>, a, chunk, ecap); break;
        case 4: e = cudaLaunchKernelEx(&cfg, k_paa_cl<4>, a, chunk, ecap); break;
        case 8: e = cudaLaunchKernelEx(&cfg, k_paa_cl<8>, a, chunk, ecap); break;
        case 16: e = cudaLaunchKernelEx(&cfg, k_paa_cl<16>, a, chunk, ecap); break;
        default: e = cudaLaunchKernelEx(&cfg, k_paa_cl<32>, a, chunk, ecap); break;
    }
    return check_cuda(e);
}

int launch_paa(Handle* h, int level, int n, long long nnz, const int* rowptr, const int* col,
               const uint64_t* prio, int t, int mode, const PaaBuffers& b, int* pass_of) {
    PaaArgs a{n, rowptr, col, prio, b.state, b.b1, b.blocked, b.list, b.cprio, b.root_of,
              pass_of, b.agg_size, t, mode, b.slots, kMaxRoundSlots, h->ctrl};
    cudaMemsetAsync(b.slots, 0, sizeof(int) * kMaxRoundSlots, h->work);
    if (mode == UAAMG_PASS_MAXIMAL && n <= kPaaSmallN) {  // one block, state in shared memory
        static DevCache attr;
        const size_t smem = (sizeof(uint64_t) + 2) * (size_t)kPaaSmallN;
        if (!attr.get(h->device)) {
            cudaFuncSetAttribute(k_paa_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr.set(h->device, 1);
        }
        k_paa_small<<<1, kPaaSmallThreads, smem, h->work>>>(a);
        count_launch(h);
        return check_cuda(cudaGetLastError());
    }
    cudaMemsetAsync(&h->ctrl->bar_count, 0, sizeof(unsigned int), h->work);
    ProfSlot ps{};
    const bool prof = (h->prof_class == UAAMG_KCLASS_PAA && level == 0);
    if (prof) {
        cudaEventCreate(&ps.a);
        cudaEventCreate(&ps.b);
        cudaEventRecord(ps.a, h->work);
    }
    int st = UAAMG_OK;
    bool counted = false;
    const bool u16 = n <= 65536;
    const size_t blk_bytes = u16 ? paa_block_bytes<uint16_t>(n, nnz) : paa_block_bytes<int>(n, nnz);
    const int ccl = mode == UAAMG_PASS_SINGLE_ROUND && n <= kPaaClMaxN ? paa_cl_blocks(h->device) : 0;
    const int ecap = ccl ? paa_cl_ecap(n, nnz, ccl) : 0;
    if (ecap > 0) {  // the level in the shared memory of one cluster
        st = launch_paa_cl(h, a, nnz, ccl, ecap);
    } else if (mode == UAAMG_PASS_SINGLE_ROUND && n <= kPaaBlockMaxN && blk_bytes <= kPaaBlockSmem) {
        // the whole level in one block's shared memory
        static DevCache attr;
        if (!attr.get(h->device)) {
            cudaFuncSetAttribute(k_paa_sr_block<uint16_t>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPaaBlockSmem);
            cudaFuncSetAttribute(k_paa_sr_block<int>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPaaBlockSmem);
            attr.set(h->device, 1);
        }
        if (u16)
            k_paa_sr_block<uint16_t><<<1, kPaaBlockThreads, blk_bytes, h->work>>>(a);
        else
            k_paa_sr_block<int><<<1, kPaaBlockThreads, blk_bytes, h->work>>>(a);
        st = check_cuda(cudaGetLastError());
    } else if (mode == UAAMG_PASS_SINGLE_ROUND) {
        // Large levels are throughput-bound: one lane per vertex.  Small ones are bound by
        // the latency of each sweep's load chain: lanes per vertex from the row length.
        const long long avg = n > 0 ? (nnz + n - 1) / n : 1;
        int grid = 0;
        if (n > kPaaLanesMaxN) st = launch_paa_sr<1>(h, a, &grid);
        else if (avg <= 8) st = launch_paa_sr<8>(h, a, &grid);
        else if (avg <= 16) st = launch_paa_sr<16>(h, a, &grid);
        else st = launch_paa_sr<32>(h, a, &grid);
        counted = true;  // the launcher counts its launches
    } else {
        static DevCache occ;
        int blocks_per_sm = occ.get(h->device);
        if (!blocks_per_sm) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_paa, kThreads, 0) !=
                    cudaSuccess ||
                blocks_per_sm < 1)
                blocks_per_sm = 1;
            occ.set(h->device, blocks_per_sm);
        }
        int grid = blocks_per_sm * h->num_sms;
        const int need = grid_for(n, kThreads);
        if (grid > need) grid = need;
        void* args[] = {&a};
        st = check_cuda(cudaLaunchCooperativeKernel((const void*)k_paa, dim3(grid),
                                                    dim3(kThreads), args, 0, h->work));
    }
    if (prof) {
        cudaEventRecord(ps.b, h->work);
        h->prof_slots.push_back(ps);
    }
    if (!counted) count_launch(h);
    return st;
}

// ---------------------------------------------------------------------------------------
// Coarse numbering (Section 5.1): the k-th root in ascending vertex index is coarse vertex
// k.  cid = exclusive scan of the root flags, start = exclusive scan of the aggregate
// sizes over the roots; each root lists its members (itself and the neighbours it took)
// in ascending order, read off its sorted CSR row.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_root_flags(int n, const int* __restrict__ root_of, const int* __restrict__ agg_size,
             int* __restrict__ f, int* __restrict__ g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool r = (root_of[i] == i);
    f[i] = r ? 1 : 0;
    g[i] = r ? agg_size[i] : 0;
}

int launch_root_flags(Handle* h, int n, const int* root_of, const int* agg_size, int* f,
                      int* g) {
    k_root_flags<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, root_of, agg_size, f, g);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

__global__ void __launch_bounds__(kThreads)
k_renumber(int n, const int* __restrict__ root_of, const int* __restrict__ cid,
           const int* __restrict__ start, const int* __restrict__ rowptr,
           const int* __restrict__ col, const int* __restrict__ d_nc, int* __restrict__ agg,
           int* __restrict__ aggptr, int* __restrict__ members) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) aggptr[*d_nc] = n;
    if (i >= n) return;
    const int r = root_of[i];
    agg[i] = cid[r];
    if (r != i) return;
    int pos = start[i];
    aggptr[cid[i]] = pos;
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
        int u = col[k];
        if (root_of[u] == i) members[pos++] = u;
    }
}

int launch_renumber(Handle* h, int n, const int* root_of, const int* cid, const int* start,
                    const int* rowptr, const int* col, const int* d_nc, int* agg, int* aggptr,
                    int* members) {
    k_renumber<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, root_of, cid, start, rowptr,
                                                                col, d_nc, agg, aggptr, members);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Coarse operator, Eq. (2.4): (A_c)_IJ = sum_{s in G_I} sum_{t in G_J} a_st.
// One warp per coarse row I: (1) gather the entries (J = agg[t], a_st) of the member rows
// in fine CSR order (members ascending, then stored order), (2) stable rank sort by J,
// (3) one sum per distinct J, added from +0.0 in that order -- the same order as the plain
// statement, so the sums are bit-identical to it.  The pattern is structural (no entry is
// dropped) and the columns come out sorted.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_coarse_m(int nc, const int* __restrict__ aggptr, const int* __restrict__ members,
           const int* __restrict__ rowptr, int* __restrict__ m) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int s = 0;
    for (int q = aggptr[I]; q < aggptr[I + 1]; q++) {
        int v = members[q];
        s += rowptr[v + 1] - rowptr[v];
    }
    m[I] = s;
}

int launch_coarse_m(Handle* h, int nc, const int* aggptr, const int* members,
                    const int* rowptr, int* m) {
    k_coarse_m<<<grid_for(nc, kThreads), kThreads, 0, h->work>>>(nc, aggptr, members, rowptr, m);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// Per coarse row, in one warp.  Rows whose members hold at most kCbMax entries run from
// shared memory: the members' row bounds are read once, every entry's (agg[col], val) is
// gathered with its loads in flight together, the stable rank sort reads the warp's keys
// as shared-memory broadcasts, and each column's run is summed there.  Longer rows use the
// same three steps through the global scratch buffers.  Both add every column's entries
// from +0.0 in gather order (members ascending, then stored order) with rounded adds.
constexpr int kCbMax = 128;
constexpr int kCbWarps = kThreads / 32;

__device__ void coarse_row_global(int I, int lane, const int* __restrict__ aggptr,
                                  const int* __restrict__ members, const int* __restrict__ rowptr,
                                  const int* __restrict__ col, const double* __restrict__ val,
                                  const int* __restrict__ agg, long long base, int* tJ,
                                  double* tV, int* sJ, double* sV, int* __restrict__ cnt) {
    // (1) gather
    int m = 0;
    for (int q = aggptr[I]; q < aggptr[I + 1]; q++) {
        const int s = members[q];
        const int k0 = rowptr[s], k1 = rowptr[s + 1];
        for (int k = k0 + lane; k < k1; k += 32) {
            tJ[base + m + (k - k0)] = agg[col[k]];
            tV[base + m + (k - k0)] = val[k];
        }
        m += k1 - k0;
    }
    __syncwarp();
    // (2) stable rank sort by coarse column
    for (int e = lane; e < m; e += 32) {
        const int J = __ldcg(tJ + base + e);
        int rank = 0;
        for (int f = 0; f < m; f++) {
            const int Jf = __ldcg(tJ + base + f);
            rank += (Jf < J) || (Jf == J && f < e);
        }
        sJ[base + rank] = J;
        sV[base + rank] = __ldcg(tV + base + e);
    }
    __syncwarp();
    // (3) one ordered sum per distinct column, written compacted over the gather buffers
    int seg = 0;
    for (int p0 = 0; p0 < m; p0 += 32) {
        const int p = p0 + lane;
        bool start = false;
        int J = 0;
        if (p < m) {
            J = __ldcg(sJ + base + p);
            start = (p == 0) || (__ldcg(sJ + base + p - 1) != J);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, start);
        if (start) {
            const int idx = seg + __popc(bal & ((1u << lane) - 1u));
            double sum = 0.0;
            for (int q = p; q < m && __ldcg(sJ + base + q) == J; q++)
                sum = __dadd_rn(sum, __ldcg(sV + base + q));
            tJ[base + idx] = J;
            tV[base + idx] = sum;
        }
        seg += __popc(bal);
    }
    if (lane == 0) cnt[I] = seg;
}

__global__ void __launch_bounds__(kThreads)
k_coarse_build(int nc, const int* __restrict__ aggptr, const int* __restrict__ members,
               const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, const int* __restrict__ agg,
               const int* __restrict__ off, int* tJ, double* tV, int* sJ, double* sV,
               int* __restrict__ cnt) {
    __shared__ int gj[kCbWarps][kCbMax], rj[kCbWarps][kCbMax];
    __shared__ double gv[kCbWarps][kCbMax], rv[kCbWarps][kCbMax];
    __shared__ int mk0[kCbWarps][32], moff[kCbWarps][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int I = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (I >= nc) return;  // whole warps leave together
    const long long base = off[I];
    const int q0 = aggptr[I], nm = aggptr[I + 1] - q0;
    // row bounds of up to 32 members at once, and the entry offsets of their rows
    int len = 0, k0 = 0;
    if (nm <= 32 && lane < nm) {
        const int s = members[q0 + lane];
        k0 = rowptr[s];
        len = rowptr[s + 1] - k0;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int m = __shfl_sync(0xffffffffu, incl, 31);
    if (nm > 32 || m > kCbMax) {
        coarse_row_global(I, lane, aggptr, members, rowptr, col, val, agg, base, tJ, tV, sJ, sV,
                          cnt);
        return;
    }
    mk0[w][lane] = k0;
    moff[w][lane + 1] = incl;
    if (lane == 0) moff[w][0] = 0;
    __syncwarp();
    // (1) gather, all of a lane's entries in flight together
    int ee[kCbMax / 32], cc[kCbMax / 32];
    double vv[kCbMax / 32];
#pragma unroll
    for (int u = 0; u < kCbMax / 32; u++) {
        const int e = lane + 32 * u;
        ee[u] = -1;
        if (e < m) {
            int q = 0;
            while (moff[w][q + 1] <= e) q++;  // the member holding entry e
            const int k = mk0[w][q] + (e - moff[w][q]);
            ee[u] = e;
            cc[u] = col[k];
            vv[u] = val[k];
        }
    }
#pragma unroll
    for (int u = 0; u < kCbMax / 32; u++) {
        if (ee[u] < 0) continue;
        gj[w][ee[u]] = agg[cc[u]];
        gv[w][ee[u]] = vv[u];
    }
    __syncwarp();
    // (2) stable rank sort by coarse column
#pragma unroll
    for (int u = 0; u < kCbMax / 32; u++) {
        const int e = lane + 32 * u;
        if (e >= m) continue;
        const int J = gj[w][e];
        int rank = 0;
        for (int f = 0; f < m; f++) {
            const int Jf = gj[w][f];
            rank += (Jf < J) || (Jf == J && f < e);
        }
        rj[w][rank] = J;
        rv[w][rank] = gv[w][e];
    }
    __syncwarp();
    // (3) one ordered sum per distinct column, written compacted
    int seg = 0;
    for (int p0 = 0; p0 < m; p0 += 32) {
        const int p = p0 + lane;
        bool start = false;
        int J = 0;
        if (p < m) {
            J = rj[w][p];
            start = (p == 0) || (rj[w][p - 1] != J);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, start);
        if (start) {
            const int idx = seg + __popc(bal & ((1u << lane) - 1u));
            double sum = 0.0;
            for (int q = p; q < m && rj[w][q] == J; q++) sum = __dadd_rn(sum, rv[w][q]);
            tJ[base + idx] = J;
            tV[base + idx] = sum;
        }
        seg += __popc(bal);
    }
    if (lane == 0) cnt[I] = seg;
}

int launch_coarse_build(Handle* h, int level, int nc, const int* aggptr, const int* members,
                        const int* rowptr, const int* col, const double* val, const int* agg,
                        const int* off, int* tJ, double* tV, int* sJ, double* sV, int* cnt) {
    ProfSlot ps{};
    bool prof = (h->prof_class == UAAMG_KCLASS_COARSE && level == 0);
    if (prof) {
        cudaEventCreate(&ps.a);
        cudaEventCreate(&ps.b);
        cudaEventRecord(ps.a, h->work);
    }
    int grid = grid_for((long long)nc * 32, kThreads);
    k_coarse_build<<<grid, kThreads, 0, h->work>>>(nc, aggptr, members, rowptr, col, val, agg,
                                                   off, tJ, tV, sJ, sV, cnt);
    if (prof) {
        cudaEventRecord(ps.b, h->work);
        h->prof_slots.push_back(ps);
    }
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

__global__ void __launch_bounds__(kThreads)
k_coarse_compact(int nc, const int* __restrict__ off, const int* __restrict__ rowptr_c,
                 const int* __restrict__ cnt, const int* __restrict__ tJ,
                 const double* __restrict__ tV, int* __restrict__ col_c,
                 double* __restrict__ val_c) {
    const int lane = threadIdx.x & 31;
    const int I = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (I >= nc) return;
    const long long src = off[I];
    const int dst = rowptr_c[I], c = cnt[I];
    for (int k = lane; k < c; k += 32) {
        col_c[dst + k] = tJ[src + k];
        val_c[dst + k] = tV[src + k];
    }
}

int launch_coarse_compact(Handle* h, int nc, const int* off, const int* rowptr_c,
                          const int* cnt, const int* tJ, const double* tV, int* col_c,
                          double* val_c) {
    int grid = grid_for((long long)nc * 32, kThreads);
    k_coarse_compact<<<grid, kThreads, 0, h->work>>>(nc, off, rowptr_c, cnt, tJ, tV, col_c, val_c);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Aggregating twice (Section 3.3): the level's aggregates are unions of first-stage
// aggregates, agg = agg2[agg1]; the member list of each union is kept in ascending fine
// index, as for a single stage.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_compose_sizes(int nc, const int* __restrict__ aggptr2, const int* __restrict__ members2,
                const int* __restrict__ aggptr1, int* __restrict__ sizes) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int s = 0;
    for (int q = aggptr2[I]; q < aggptr2[I + 1]; q++) {
        int J = members2[q];
        s += aggptr1[J + 1] - aggptr1[J];
    }
    sizes[I] = s;
}

__global__ void __launch_bounds__(kThreads)
k_compose_members(int nc, const int* __restrict__ aggptr2, const int* __restrict__ members2,
                  const int* __restrict__ aggptr1, const int* __restrict__ members1,
                  const int* __restrict__ aggptr, int* tmp, int* __restrict__ members) {
    const int lane = threadIdx.x & 31;
    const int I = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (I >= nc) return;
    const int base = aggptr[I];
    int m = 0;
    for (int q = aggptr2[I]; q < aggptr2[I + 1]; q++) {
        const int J = members2[q];
        const int k0 = aggptr1[J], k1 = aggptr1[J + 1];
        for (int k = k0 + lane; k < k1; k += 32) tmp[base + m + (k - k0)] = members1[k];
        m += k1 - k0;
    }
    __syncwarp();
    for (int e = lane; e < m; e += 32) {  // distinct values: rank = number of smaller ones
        const int v = __ldcg(tmp + base + e);
        int rank = 0;
        for (int f = 0; f < m; f++) rank += (__ldcg(tmp + base + f) < v);
        members[base + rank] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
k_compose_agg(int n, const int* __restrict__ agg1, const int* __restrict__ agg2,
              int* __restrict__ agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = agg2[agg1[i]];
}

int launch_compose(Handle* h, int n, int nc, const int* agg1, const int* aggptr1,
                   const int* members1, const int* agg2, const int* aggptr2,
                   const int* members2, int* agg, int* aggptr, int* members, int* tmp,
                   int* scan_tmp) {
    k_compose_sizes<<<grid_for(nc, kThreads), kThreads, 0, h->work>>>(nc, aggptr2, members2, aggptr1, aggptr);
    count_launch(h);
    int st = scan_exclusive(h, aggptr, aggptr, nc, aggptr + nc, scan_tmp);
    if (st) return st;
    k_compose_members<<<grid_for((long long)nc * 32, kThreads), kThreads, 0, h->work>>>(
        nc, aggptr2, members2, aggptr1, members1, aggptr, tmp, members);
    k_compose_agg<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, agg1, agg2, agg);
    count_launch(h, 2);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Smoother data, Section 4.1: l1-Jacobi Minv_i = 1 / (a_ii + sum_{j!=i} |a_ij|) (row sum in
// stored order), or damped Jacobi Minv_i = omega / a_ii; FP32 copies for the mixed cycle.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_minv(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
       const double* __restrict__ val, double omega, double* __restrict__ minv64,
       float* __restrict__ minv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double diag = 0.0, off = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
        if (col[k] == i) diag = val[k];
        else off = __dadd_rn(off, fabs(val[k]));
    }
    // l1-Jacobi, or damped Jacobi omega / a_ii when omega > 0
    double m = omega > 0.0 ? __ddiv_rn(omega, diag) : __ddiv_rn(1.0, __dadd_rn(diag, off));
    minv64[i] = m;
    if (minv32) minv32[i] = __double2float_rn(m);
}

__global__ void __launch_bounds__(kThreads)
k_cast32(long long nnz, const double* __restrict__ v64, float* __restrict__ v32) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) v32[k] = __double2float_rn(v64[k]);
}

int launch_level_finish(Handle* h, int n, long long nnz, const int* rowptr, const int* col,
                        const double* val64, double* minv64, float* minv32, float* val32) {
    k_minv<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, rowptr, col, val64,
                                                             h->p.jacobi_omega, minv64, minv32);
    count_launch(h);
    if (val32) {
        k_cast32<<<grid_for(nnz, kThreads), kThreads, 0, h->work>>>(nnz, val64, val32);
        count_launch(h);
    }
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Coarsest level, Algorithm 1 "solve exactly": the explicit FP64 inverse of the coarsest
// matrix (k_gj_inverse below), so that each coarsest solve of the cycle is a dense
// matrix-vector product.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_dense_gather(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, double* __restrict__ D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) D[(size_t)i * n + col[k]] = val[k];
}

// Inverse of the SPD coarsest matrix by Gauss-Jordan elimination without pivoting: the
// pivots are the leading diagonal entries of successive Schur complements, positive for an
// SPD matrix, and a pivot <= 0 reports kErrNotSpd.  Step j maps the current iterate (one
// buffer) to the next (the other) entry by entry,
//   new_jj = 1/p,  new_jk = a_jk/p,  new_ij = -a_ij/p,  new_ik = a_ik - a_ij (a_jk/p),
// with p = a_jj, so the whole grid works on one step and one grid barrier separates steps.
// Buffers written by other blocks are read through L2 only (__ldcg).
__global__ void __launch_bounds__(kThreads)
k_gj_inverse(int n, double* __restrict__ A, double* __restrict__ B, Ctrl* ctrl) {
    const int nn = n * n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    double* src = A;
    double* dst = B;
    for (int j = 0; j < n; j++) {
        const double p = __ldcg(&src[(size_t)j * n + j]);
        if (!(p > 0.0)) {  // every thread sees the same pivot, so all leave together
            if (tid == 0) atomicOr(&ctrl->err, kErrNotSpd);
            return;
        }
        const double q = 1.0 / p;
        for (int e = tid; e < nn; e += stride) {
            const int i = e / n, k = e - i * n;
            double v;
            if (i == j) {
                v = (k == j) ? q : __ldcg(&src[(size_t)j * n + k]) * q;
            } else if (k == j) {
                v = -__ldcg(&src[(size_t)i * n + j]) * q;
            } else {
                const double ajk = __ldcg(&src[(size_t)j * n + k]) * q;
                v = fma(-__ldcg(&src[(size_t)i * n + j]), ajk, __ldcg(&src[e]));
            }
            dst[e] = v;
        }
        if (!grid_barrier(ctrl)) return;
        double* t = src;
        src = dst;
        dst = t;
    }
    if (src != B)  // n even: the inverse ended in A
        for (int e = tid; e < nn; e += stride) B[e] = __ldcg(&src[e]);
}

int launch_dense_coarsest(Handle* h, int n, const int* rowptr, const int* col,
                          const double* val, double* work, double* inv) {
    static DevCache occ;
    int blocks_per_sm = occ.get(h->device);
    if (!blocks_per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_gj_inverse, kThreads,
                                                          0) != cudaSuccess ||
            blocks_per_sm < 1)
            blocks_per_sm = 1;
        occ.set(h->device, blocks_per_sm);
    }
    cudaMemsetAsync(work, 0, sizeof(double) * (size_t)n * n, h->work);
    k_dense_gather<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, rowptr, col, val, work);
    int grid = blocks_per_sm * h->num_sms;
    const int need = grid_for((long long)n * n, kThreads);
    if (grid > need) grid = need;
    cudaMemsetAsync(&h->ctrl->bar_count, 0, sizeof(unsigned int), h->work);
    Ctrl* ctrl = h->ctrl;
    void* args[] = {&n, &work, &inv, &ctrl};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_gj_inverse, dim3(grid),
                                                dim3(kThreads), args, 0, h->work);
    count_launch(h, 2);
    if (e != cudaSuccess) return check_cuda(e);
    return check_cuda(cudaGetLastError());
}

}  // namespace uaamg
