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
// Parallel aggregation, Algorithm 2: one persistent cooperative kernel runs every pass of
// a level.  A pass is (A) rounds of coarse-vertex selection and (B) star aggregation.
//
// Round (two sweeps, separated by grid barriers; the state array is a snapshot per sweep,
// so the result does not depend on thread order):
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
    int* root_of;
    int* pass_of;
    int* agg_size;
    int t;
    int mode;
    int* slots;
    int nslots;
    Ctrl* ctrl;
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
    if (a.mode == UAAMG_PASS_SINGLE_ROUND) {
        // One round per pass (Algorithm 2 as printed), two sweeps and two grid barriers per
        // pass: (1) b1 and the count of unprocessed vertices; (2) every local maximum becomes
        // a root and takes its neighbours at once.  Fusing selection and aggregation is safe:
        // a neighbour w of a root v is never a root itself (P_v > P_w within distance 2) and
        // no other root reaches it (roots are >= 3 apart), so w has a single writer, and w's
        // own thread selects nothing whether it reads w's old or new state.
        while (true) {
            int cnt = 0;
            for (int v = g0; v < a.n; v += gs) {
                const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
                uint64_t best = 0;
                for (int k = k0; k < k1; k++) {
                    const int u = a.col[k];
                    if (ld_state(a.state + u) == ST_CAND) {
                        const uint64_t pu = a.prio[u];
                        best = pu > best ? pu : best;
                    }
                }
                a.b1[v] = best;
                cnt += (ld_state(a.state + v) == ST_CAND);
            }
            cnt = block_sum_int(cnt);
            if (threadIdx.x == 0 && cnt) atomicAdd(&a.slots[slot], cnt);
            if (!grid_barrier(a.ctrl)) return;
            const int remaining = *(volatile int*)&a.slots[slot];
            slot++;
            if (remaining == 0) break;
            if (slot >= a.nslots) {
                if (g0 == 0) atomicOr(&a.ctrl->err, kErrSlots);
                return;
            }
            for (int v = g0; v < a.n; v += gs) {
                if (ld_state(a.state + v) != ST_CAND) continue;
                const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
                uint64_t m = 0;
                for (int k = k0; k < k1; k++) {
                    const uint64_t bu = __ldcg(reinterpret_cast<const unsigned long long*>(a.b1 + a.col[k]));
                    m = bu > m ? bu : m;
                }
                if (m != a.prio[v]) continue;
                int taken = 1;  // v is a root: its star aggregate
                for (int k = k0; k < k1; k++) {
                    const int u = a.col[k];
                    if (u == v) continue;
                    if (a.t > 0 && taken >= a.t) break;
                    if (ld_state(a.state + u) == ST_CAND) {
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
            pass++;
        }
        if (g0 == 0) a.ctrl->npasses = pass;
        return;
    }
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
        if (a.mode == UAAMG_PASS_SINGLE_ROUND) {
            // sweep 1: b1 and the count of unprocessed vertices
            int cnt = 0;
            for (int v = t; v < a.n; v += T) {
                uint64_t best = 0;
                for (int k = a.rowptr[v]; k < a.rowptr[v + 1]; k++) {
                    const int u = a.col[k];
                    if (state[u] == ST_CAND) {
                        const uint64_t pu = a.prio[u];
                        best = pu > best ? pu : best;
                    }
                }
                b1[v] = best;
                cnt += (state[v] == ST_CAND);
            }
            if (block_sum_big(cnt, red) == 0) break;
            // sweep 2: local maxima become roots and take their neighbours (see k_paa)
            for (int v = t; v < a.n; v += T) {
                if (state[v] != ST_CAND) continue;
                const int k0 = a.rowptr[v], k1 = a.rowptr[v + 1];
                uint64_t m = 0;
                for (int k = k0; k < k1; k++) {
                    const uint64_t bu = b1[a.col[k]];
                    m = bu > m ? bu : m;
                }
                if (m != a.prio[v]) continue;
                int taken = 1;
                for (int k = k0; k < k1; k++) {
                    const int u = a.col[k];
                    if (u == v) continue;
                    if (a.t > 0 && taken >= a.t) break;
                    if (state[u] == ST_CAND) {
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
        } else {
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
        }
        pass++;
        if (++rounds >= a.nslots) {
            if (t == 0) atomicOr(&a.ctrl->err, kErrSlots);
            return;
        }
    }
    if (t == 0) a.ctrl->npasses = pass;
}

int launch_paa(Handle* h, int level, int n, const int* rowptr, const int* col,
               const uint64_t* prio, int t, int mode, const PaaBuffers& b, int* pass_of) {
    static int blocks_per_sm = 0;
    if (!blocks_per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_paa, kThreads, 0) !=
                cudaSuccess ||
            blocks_per_sm < 1)
            blocks_per_sm = 1;
    }
    if (n <= kPaaSmallN) {  // one block, state in shared memory
        static bool attr_set = false;
        const size_t smem = (sizeof(uint64_t) + 2) * (size_t)kPaaSmallN;
        if (!attr_set) {
            cudaFuncSetAttribute(k_paa_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr_set = true;
        }
        PaaArgs a{n, rowptr, col, prio, b.state, b.b1, b.blocked, b.root_of, pass_of, b.agg_size,
                  t, mode, b.slots, kMaxRoundSlots, h->ctrl};
        k_paa_small<<<1, kPaaSmallThreads, smem, h->work>>>(a);
        count_launch(h);
        return check_cuda(cudaGetLastError());
    }
    int grid = blocks_per_sm * h->num_sms;
    int need = grid_for(n, kThreads);
    if (grid > need) grid = need;
    cudaMemsetAsync(b.slots, 0, sizeof(int) * kMaxRoundSlots, h->work);
    cudaMemsetAsync(&h->ctrl->bar_count, 0, 2 * sizeof(unsigned int), h->work);
    PaaArgs a{n, rowptr, col, prio, b.state, b.b1, b.blocked, b.root_of, pass_of, b.agg_size,
              t, mode, b.slots, kMaxRoundSlots, h->ctrl};
    void* args[] = {&a};
    ProfSlot ps{};
    bool prof = (h->prof_class == UAAMG_KCLASS_PAA && level == 0);
    if (prof) {
        cudaEventCreate(&ps.a);
        cudaEventCreate(&ps.b);
        cudaEventRecord(ps.a, h->work);
    }
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_paa, dim3(grid), dim3(kThreads),
                                                args, 0, h->work);
    if (prof) {
        cudaEventRecord(ps.b, h->work);
        h->prof_slots.push_back(ps);
    }
    count_launch(h);
    return check_cuda(e);
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

__global__ void __launch_bounds__(kThreads)
k_coarse_build(int nc, const int* __restrict__ aggptr, const int* __restrict__ members,
               const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, const int* __restrict__ agg,
               const int* __restrict__ off, int* tJ, double* tV, int* sJ, double* sV,
               int* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int I = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (I >= nc) return;
    const long long base = off[I];
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
// Coarsest level, Algorithm 1 "solve exactly": dense Cholesky factor L L^T of the coarsest
// matrix (one block), then its inverse by one forward and one backward substitution per
// column, so that each coarsest solve of the cycle is a dense matrix-vector product.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_dense_gather(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, double* __restrict__ D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) D[(size_t)i * n + col[k]] = val[k];
}

// Left-looking Cholesky in one block: for column j, warp w computes the dot products of
// rows i = j + w, j + w + 32, ... with row j over k < j (lanes over k), first the diagonal.
__global__ void __launch_bounds__(1024)
k_chol_factor(int n, double* __restrict__ D, Ctrl* ctrl) {
    __shared__ int bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (warp == 0) {
            double s = 0.0;
            for (int k = lane; k < j; k += 32) s += D[(size_t)j * n + k] * D[(size_t)j * n + k];
            s = warp_sum(s);
            if (lane == 0) {
                const double d = D[(size_t)j * n + j] - s;
                if (!(d > 0.0)) bad = 1;
                else D[(size_t)j * n + j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) {
            if (threadIdx.x == 0) atomicOr(&ctrl->err, kErrNotSpd);
            return;
        }
        const double ljj = D[(size_t)j * n + j];
        for (int i = j + 1 + warp; i < n; i += nw) {
            double s = 0.0;
            for (int k = lane; k < j; k += 32) s += D[(size_t)i * n + k] * D[(size_t)j * n + k];
            s = warp_sum(s);
            if (lane == 0) D[(size_t)i * n + j] = (D[(size_t)i * n + j] - s) / ljj;
        }
        __syncthreads();
    }
}

// Column c of the inverse, one warp per column: L y = e_c forward, then L^T x = y backward,
// each step a warp-parallel dot product; y lives in shared memory.
__global__ void __launch_bounds__(32)
k_chol_inverse_cols(int n, const double* __restrict__ L, double* __restrict__ X) {
    __shared__ double y[kMaxCoarsest];
    const int c = blockIdx.x, lane = threadIdx.x;
    for (int i = lane; i < n; i += 32) y[i] = 0.0;
    __syncwarp();
    for (int i = c; i < n; i++) {
        double s = 0.0;
        for (int k = c + lane; k < i; k += 32) s += L[(size_t)i * n + k] * y[k];
        s = warp_sum(s);
        if (lane == 0) y[i] = ((i == c ? 1.0 : 0.0) - s) / L[(size_t)i * n + i];
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s += L[(size_t)k * n + i] * y[k];
        s = warp_sum(s);
        if (lane == 0) y[i] = (y[i] - s) / L[(size_t)i * n + i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) X[(size_t)i * n + c] = y[i];
}

int launch_dense_coarsest(Handle* h, int n, const int* rowptr, const int* col,
                          const double* val, double* work, double* inv) {
    cudaMemsetAsync(work, 0, sizeof(double) * (size_t)n * n, h->work);
    k_dense_gather<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, rowptr, col, val, work);
    k_chol_factor<<<1, 1024, 0, h->work>>>(n, work, h->ctrl);
    k_chol_inverse_cols<<<n, 32, 0, h->work>>>(n, work, inv);
    count_launch(h, 3);
    return check_cuda(cudaGetLastError());
}

}  // namespace uaamg
