// kern_sra.cu -- subgraph reshaping of an aggregation (Section 3.2, Algorithm 3, Eq. 3.8).
//
// A round reshapes the pairs of a matching of neighbouring aggregates, all at once:
//   k_sra_init     per aggregate: size, no partner, no proposal
//   k_sra_propose  per fine row: propose to the eligible neighbouring aggregate of largest
//                  pair weight (64-bit atomicMax on (weight, ~J))
//   k_sra_match    mutual proposals = the round's pairs, appended to a list
//   k_sra_pairs    persistent half-warps, one pair at a time each: the union's local graph
//                  Laplacian (a small CSR in shared memory), every balanced split with both
//                  halves connected (Algorithm 3 step 2), the split of largest energy
//                  (step 3), the new aggregate numbers
//   scan           new sizes -> new aggregate offsets
//   k_sra_members  per aggregate: its member list, ascending (unchanged ones are copied)
//
// Energy of a split (S, S^c) of the union: |T(span psi)|_A^2 with psi = 1_S/|S| -
// 1_{S^c}/|S^c|, T = Q (I - R A), Q the A-orthogonal projection onto span psi and R the
// l1-Jacobi smoother of A.  It is the trace of the rank-one W of Eq. 3.8.  Because A 1 = 0,
// psi = (1/|S| + 1/|S^c|) 1_S modulo the constants, and the trace reduces to
//     J(S) = (c - 2 g^T R g + h^T A h) / c,   g = A 1_S,  h = R g,  c = 1_S^T A 1_S,
// which needs no pseudo-inverse.  A is a graph Laplacian, so g lives on the cut edges and
// h^T A h is the sum over the edges of w_kl (h_k - h_l)^2.  FP64 throughout.  Each lane of
// a pair's group enumerates a contiguous range of candidate masks in ascending order (colex
// ranks), and the group keeps the largest J.  Energies within a relative kSraTie count as
// equal, and the smallest mask among them wins (symmetric splits have equal energies up to
// rounding).
#include "common.cuh"
#include "kern_sra.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kSraWarps = 4;  // warps per block of k_sra_pairs
constexpr double kSraTie = 1e-9;

__device__ __forceinline__ uint32_t sra_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static uint32_t host_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t sra_round_salt(uint64_t seed, int level, int round) {
    const uint32_t s = (uint32_t)(seed ^ (seed >> 32));
    return host_fmix32(s + 0x9E3779B9u * (uint32_t)(64 * level + round + 1));
}

__global__ void __launch_bounds__(kThreads)
k_sra_init(int nc, const int* __restrict__ aggptr, int* __restrict__ newsize,
           int* __restrict__ pair_of, unsigned long long* __restrict__ prop,
           int* __restrict__ count) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I == 0) *count = 0;
    if (I >= nc) return;
    newsize[I] = aggptr[I + 1] - aggptr[I];
    pair_of[I] = -1;
    prop[I] = 0ull;
}

// Each aggregate proposes to its eligible neighbour J of largest weight
// fmix32(fmix32(min ^ salt) + max), equal weights to the smaller J: key (w << 32) | ~J.
__global__ void __launch_bounds__(kThreads)
k_sra_propose(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
              const double* __restrict__ val, const int* __restrict__ agg,
              const int* __restrict__ aggptr, uint32_t salt,
              unsigned long long* __restrict__ prop) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int I = agg[s];
    const int sI = aggptr[I + 1] - aggptr[I];
    unsigned long long best = 0ull;
    for (int q = rowptr[s]; q < rowptr[s + 1]; q++) {
        const int t = col[q];
        if (t == s || val[q] == 0.0) continue;
        const int J = agg[t];
        if (J == I) continue;
        if (sI + (aggptr[J + 1] - aggptr[J]) > kSraUnionMax) continue;
        const uint32_t lo = (uint32_t)min(I, J), hi = (uint32_t)max(I, J);
        const uint32_t w = sra_fmix32(sra_fmix32(lo ^ salt) + hi);
        const unsigned long long key =
            ((unsigned long long)w << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)J);
        if (key > best) best = key;
    }
    if (best) atomicMax(&prop[I], best);
}

__device__ __forceinline__ int sra_partner(unsigned long long p) {
    return p ? (int)(0xFFFFFFFFu - (uint32_t)(p & 0xFFFFFFFFull)) : -1;
}

// The round's pairs: aggregate I < J with mutual proposals, appended to a list (its order
// does not matter: pairs are disjoint and each writes only its own vertices).
__global__ void __launch_bounds__(kThreads)
k_sra_match(int nc, const unsigned long long* __restrict__ prop, int* __restrict__ list,
            int* __restrict__ count) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (I < nc) {
        const int J = sra_partner(prop[I]);
        take = J > I && J < nc && sra_partner(prop[J]) == I;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, take);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);  // every lane of the warp is here
    if (take) list[base + __popc(m & ((1u << lane) - 1u))] = I;
}

// Binomial coefficients C(n, k), n, k <= 16, for the colex ranks of the candidate masks.
struct SraBinom {
    uint32_t v[kSraUnionMax + 1][kSraUnionMax + 1];
};
constexpr SraBinom sra_make_binom() {
    SraBinom t{};
    for (int n = 0; n <= kSraUnionMax; n++)
        for (int k = 0; k <= kSraUnionMax; k++)
            t.v[n][k] = (k == 0) ? 1u : (n == 0 ? 0u : t.v[n - 1][k - 1] + t.v[n - 1][k]);
    return t;
}
__constant__ SraBinom kSraBinom = sra_make_binom();

// Bit-parallel search: true iff the local vertices of X induce a connected subgraph.
__device__ __forceinline__ bool sra_connected(uint32_t X, const uint32_t (&adj)[kSraUnionMax],
                                              int nu) {
    uint32_t reach = X & (0u - X);
    for (int it = 0; it < nu; it++) {
        uint32_t nb = reach;
#pragma unroll
        for (int k = 0; k < kSraUnionMax; k++) nb |= ((reach >> k) & 1u) ? adj[k] : 0u;
        nb &= X;
        if (nb == reach) break;
        reach = nb;
    }
    return reach == X;
}

constexpr int kSraMaxNb = kSraUnionMax * (kSraUnionMax - 1);  // directed local edges

constexpr int kSraGroup = 16;  // lanes per pair: each warp reshapes two pairs at a time

struct SraGroupSmem {
    union {
        double A[kSraUnionMax * kSraUnionMax];  // the local matrix, while it is built
        double h[kSraUnionMax * kSraGroup];     // then h = R A 1_S, one column per lane
    };
    double w[kSraMaxNb];  // local graph as CSR: w = -a_kl of each neighbour
    double r[kSraUnionMax];
    int u[kSraUnionMax];
    uint32_t adj[kSraUnionMax];
    uint8_t nb[kSraMaxNb];
    uint8_t ptr[kSraUnionMax + 1];
};

__global__ void __launch_bounds__(kSraWarps * 32)
k_sra_pairs(const int* __restrict__ list, const int* __restrict__ count,
            const int* __restrict__ rowptr, const int* __restrict__ col,
            const double* __restrict__ val, const int* __restrict__ aggptr,
            const int* __restrict__ members, const unsigned long long* __restrict__ prop,
            int* __restrict__ agg, int* __restrict__ newsize, int* __restrict__ pair_of,
            unsigned long long* __restrict__ flops) {
    __shared__ SraGroupSmem sm_all[kSraWarps * 2];
    const int lane = threadIdx.x & 31;
    const int grp = threadIdx.x / kSraGroup;     // group within the block
    const int gl = lane & (kSraGroup - 1);       // lane within the group
    const uint32_t gmask = 0xFFFFu << (lane & kSraGroup);
    SraGroupSmem& sm = sm_all[grp];
    const int npairs = *count;
    const int ngroups = gridDim.x * kSraWarps * 2;
    unsigned long long ops = 0ull;
    for (int pw = blockIdx.x * kSraWarps * 2 + grp; pw < npairs; pw += ngroups) {
        const int I = list[pw];
        const int J = sra_partner(prop[I]);
        const int oI = aggptr[I], a = aggptr[I + 1] - oI;
        const int oJ = aggptr[J], b = aggptr[J + 1] - oJ;
        const int nu = a + b;
        if (nu < 2 || nu > kSraUnionMax) continue;  // eligible pairs never are
        __syncwarp(gmask);  // the previous pair's shared data is no longer read

        // (1) the union, sorted ascending (the two member lists are disjoint)
        int v = 0x7FFFFFFF;
        if (gl < a) v = members[oI + gl];
        else if (gl < nu) v = members[oJ + gl - a];
        int rank = 0;
        for (int e = 0; e < nu; e++)
            rank += (__shfl_sync(gmask, v, e, kSraGroup) < v) ? 1 : 0;
        if (gl < nu) sm.u[rank] = v;
        for (int e = gl; e < kSraUnionMax * kSraUnionMax; e += kSraGroup) sm.A[e] = 0.0;
        __syncwarp(gmask);

        // (2) the union's local graph Laplacian: off-diagonal entries of the induced
        // subgraph (neighbours: the non-zero ones), diagonal = minus their row sum
        // (ascending l); l1-Jacobi weight 1 / (a_kk + sum |a_kl|)
        uint32_t nbm = 0u;
        if (gl < nu) {
            const int s = sm.u[gl];
            for (int q = rowptr[s]; q < rowptr[s + 1]; q++) {
                const int t = col[q];
                if (t == s) continue;
                int lo = 0, hi = nu - 1;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    const int x = sm.u[mid];
                    if (x == t) {
                        const double vq = val[q];
                        sm.A[gl * kSraUnionMax + mid] = vq;
                        if (vq != 0.0) nbm |= 1u << mid;
                        break;
                    }
                    if (x < t) lo = mid + 1;
                    else hi = mid - 1;
                }
            }
            double d = 0.0, absum = 0.0;
            for (uint32_t bits = nbm; bits; bits &= bits - 1u) {
                const double x = sm.A[gl * kSraUnionMax + (__ffs(bits) - 1)];
                d = __dadd_rn(d, x);
                absum = __dadd_rn(absum, fabs(x));
            }
            const double m = __dadd_rn(-d, absum);
            sm.r[gl] = (m != 0.0) ? 1.0 / m : 0.0;
            sm.adj[gl] = nbm;
        }
        // neighbour lists (local CSR), offsets by a group prefix sum of the degrees
        const int deg = __popc(nbm);
        int off = deg;
        for (int o = 1; o < kSraGroup; o <<= 1) {
            const int y = __shfl_up_sync(gmask, off, o, kSraGroup);
            if (gl >= o) off += y;
        }
        off -= deg;
        if (gl < nu) {
            int e = off;
            for (uint32_t bits = nbm; bits; bits &= bits - 1u) {
                const int l = __ffs(bits) - 1;
                sm.nb[e] = (uint8_t)l;
                sm.w[e] = -sm.A[gl * kSraUnionMax + l];
                e++;
            }
            sm.ptr[gl] = (uint8_t)off;
            if (gl == nu - 1) sm.ptr[nu] = (uint8_t)(off + deg);
        }
        __syncwarp(gmask);  // sm.A is dead from here on: its space holds h
        uint32_t adj[kSraUnionMax];
        int edges2 = 0;  // directed local edges = twice the undirected ones
#pragma unroll
        for (int k = 0; k < kSraUnionMax; k++) {
            adj[k] = (k < nu) ? sm.adj[k] : 0u;
            edges2 += __popc(adj[k]);
        }

        // (3) candidates: |S| = floor(nu/2); for even nu, S holds local vertex 0 and the
        // rest of S is a (m-1)-subset of {1..nu-1}.  Colex ranks = ascending masks.
        const int m = nu >> 1;
        const bool even = (nu & 1) == 0;
        const int N = even ? nu - 1 : nu;
        const int K = even ? m - 1 : m;
        const uint32_t total = kSraBinom.v[N][K];
        const uint32_t per = (total + kSraGroup - 1u) / kSraGroup;
        const uint32_t r0 = (uint32_t)gl * per;
        const uint32_t r1 = min(total, r0 + per);
        const uint32_t full = (1u << nu) - 1u;
        double bn = -1.0, bc = 1.0;  // best energy as the fraction bn / bc
        uint32_t bmask = 0xFFFFFFFFu;
        unsigned long long evals = 0ull;
        uint32_t x = 0u;
        if (r0 < r1 && K > 0) {  // unrank r0: the K-subset of {0..N-1} of that colex rank
            uint32_t rem = r0;
            for (int i = K; i >= 1; i--) {
                int c = i - 1;
                while (c + 1 < N && kSraBinom.v[c + 1][i] <= rem) c++;
                x |= 1u << c;
                rem -= kSraBinom.v[c][i];
            }
        }
        double* hcol = sm.h + gl;  // h_k of this lane's candidate at hcol[kSraGroup k]
        for (uint32_t rk = r0; rk < r1; rk++) {
            const uint32_t S = even ? ((x << 1) | 1u) : x;
            if (K > 0 && rk + 1 < r1) {  // next K-subset in colex order (Gosper's rule)
                const uint32_t c = x & (0u - x);
                const uint32_t y = x + c;
                x = (((y ^ x) >> 2) >> (__ffs(c) - 1)) | y;
            }
            if (!sra_connected(S, adj, nu) || !sra_connected(full ^ S, adj, nu)) continue;
            // g = A 1_S is carried by the cut edges: g_k = +w_kl (k in S) or -w_kl (k not in
            // S) for each neighbour l on the other side.  h = R g, cut = 1_S^T g,
            // q1 = g^T R g, q2 = h^T A h = sum over edges of w_kl (h_k - h_l)^2
            double cut = 0.0, q1 = 0.0;
            for (int k = 0; k < nu; k++) {
                const bool sk = ((S >> k) & 1u) != 0u;
                double g = 0.0;
                for (int e = sm.ptr[k]; e < sm.ptr[k + 1]; e++) {
                    const bool sl = ((S >> sm.nb[e]) & 1u) != 0u;
                    const double we = sm.w[e];
                    g += (sk == sl) ? 0.0 : (sk ? we : -we);
                }
                const double hk = g * sm.r[k];
                hcol[kSraGroup * k] = hk;
                q1 = fma(g, hk, q1);
                cut += sk ? g : 0.0;
            }
            double q2 = 0.0;
            for (int k = 0; k < nu; k++) {
                const double hk = hcol[kSraGroup * k];
                for (int e = sm.ptr[k]; e < sm.ptr[k + 1]; e++) {
                    const int l = sm.nb[e];
                    if (l > k) {
                        const double dh = hk - hcol[kSraGroup * l];
                        q2 = fma(sm.w[e], dh * dh, q2);
                    }
                }
            }
            if (!(cut > 0.0)) continue;
            evals++;
            const double num = cut - 2.0 * q1 + q2;
            // num / cut > (1 + tie) bn / bc (positive denominators); the ranks ascend, so
            // an equal value never replaces the earlier (smaller) mask
            const double rhs = bn * cut;
            if (bmask == 0xFFFFFFFFu || num * bc > rhs + kSraTie * fabs(rhs)) {
                bn = num;
                bc = cut;
                bmask = S;
            }
        }
        // group maximum, a fixed tree towards lane 0 over the lanes that had candidates:
        // larger energy, then smaller mask
        const uint32_t used = min(total, (uint32_t)kSraGroup);
        for (int o = kSraGroup / 2; o > 0; o >>= 1) {
            if ((uint32_t)o >= used) continue;  // same for the whole group
            const double on = __shfl_down_sync(gmask, bn, o, kSraGroup);
            const double oc = __shfl_down_sync(gmask, bc, o, kSraGroup);
            const uint32_t om = __shfl_down_sync(gmask, bmask, o, kSraGroup);
            if (gl + o < kSraGroup && om != 0xFFFFFFFFu) {
                bool take;
                if (bmask == 0xFFFFFFFFu) take = true;
                else {
                    const double lhs = on * bc, rhs = bn * oc, tol = kSraTie * fabs(rhs);
                    take = (lhs > rhs + tol) || (lhs >= rhs - tol && om < bmask);
                }
                if (take) {
                    bn = on;
                    bc = oc;
                    bmask = om;
                }
            }
        }
        bmask = __shfl_sync(gmask, bmask, 0, kSraGroup);
        // per evaluated split: g (2E adds), h (nu), q1 (nu FMAs), cut (nu), q2 (E times a
        // subtraction, a product and an FMA), the fraction and the comparison (5)
        ops += evals * (unsigned long long)(4 * nu + 3 * edges2 + 5);
        if (bmask == 0xFFFFFFFFu) continue;  // no admissible split: the pair stays as it is
        // the half holding local vertex 0 (the smallest vertex) keeps the smaller number I
        const bool zero_in_S = (bmask & 1u) != 0u;
        if (gl < nu) {
            const bool inS = ((bmask >> gl) & 1u) != 0u;
            agg[sm.u[gl]] = (inS == zero_in_S) ? I : J;
        }
        if (gl == 0) {
            const int cS = __popc(bmask);
            const int sizeI = zero_in_S ? cS : nu - cS;
            newsize[I] = sizeI;
            newsize[J] = nu - sizeI;
            pair_of[I] = J;
            pair_of[J] = I;
        }
    }
    if (flops) {
        for (int o = 16; o > 0; o >>= 1) ops += __shfl_xor_sync(0xffffffffu, ops, o);
        if (lane == 0 && ops) atomicAdd(flops, ops);
    }
}

// Member lists of the new aggregation, ascending within each aggregate: one thread per
// aggregate copies its list, or merges the two old lists of its pair keeping its own vertices.
__global__ void __launch_bounds__(kThreads)
k_sra_members(int nc, const int* __restrict__ aggptr_old, const int* __restrict__ members_old,
              const int* __restrict__ pair_of, const int* __restrict__ agg,
              const int* __restrict__ aggptr_new, int* __restrict__ members_new) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    const int o = aggptr_old[I], a = aggptr_old[I + 1] - o;
    int w = aggptr_new[I];
    const int J = pair_of[I];
    if (J < 0) {
        for (int e = 0; e < a; e++) members_new[w + e] = members_old[o + e];
        return;
    }
    const int oJ = aggptr_old[J], b = aggptr_old[J + 1] - oJ;
    int i = 0, j = 0;
    while (i < a || j < b) {
        int v;
        if (j >= b || (i < a && members_old[o + i] < members_old[oJ + j])) v = members_old[o + i++];
        else v = members_old[oJ + j++];
        if (agg[v] == I) members_new[w++] = v;
    }
}

// Rounds of subgraph reshaping on one level's aggregation.  agg is updated in place;
// *aggptr and *members are replaced by handle temporaries holding the new member lists.
int reshape_aggregation(Handle* h, int level, int n, const int* rowptr, const int* col,
                        const double* val, int nc, int* agg, int** aggptr, int** members,
                        int* scan_tmp) {
    int st = UAAMG_OK;
    unsigned long long* prop = dalloc<unsigned long long>(h, nc, &st, true);
    int* newsize = dalloc<int>(h, nc, &st, true);
    int* pair_of = dalloc<int>(h, nc, &st, true);
    int* list = dalloc<int>(h, (size_t)nc / 2 + 1, &st, true);
    int* count = dalloc<int>(h, 1, &st, true);
    int* ptr2 = dalloc<int>(h, (size_t)nc + 1, &st, true);
    int* mem2 = dalloc<int>(h, n, &st, true);
    if (st) return st;
    const bool prof = (h->prof_class == UAAMG_KCLASS_SRA && level == 0);
    unsigned long long* flops = prof ? dalloc<unsigned long long>(h, 1, &st, true) : nullptr;
    if (st) return st;
    if (prof) cudaMemsetAsync(flops, 0, sizeof(unsigned long long), h->work);
    // persistent grid of half-warp groups over the pair list (at most nc / 2 pairs)
    static DevCache occ;
    int bps = occ.get(h->device);
    if (!bps) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_sra_pairs, kSraWarps * 32, 0) !=
                cudaSuccess ||
            bps < 1)
            bps = 1;
        occ.set(h->device, bps);
    }
    const long long need = ((long long)nc / 2 + 2 * kSraWarps - 1) / (2 * kSraWarps);
    const int pair_blocks = (int)std::max(1LL, std::min((long long)bps * h->num_sms, need));
    for (int r = 0; r < h->p.sra_rounds; r++) {
        const uint32_t salt = sra_round_salt(h->p.seed, level, r);
        k_sra_init<<<grid_for(nc, kThreads), kThreads, 0, h->work>>>(nc, *aggptr, newsize,
                                                                   pair_of, prop, count);
        k_sra_propose<<<grid_for(n, kThreads), kThreads, 0, h->work>>>(n, rowptr, col, val, agg,
                                                                     *aggptr, salt, prop);
        k_sra_match<<<grid_for(nc, kThreads), kThreads, 0, h->work>>>(nc, prop, list, count);
        ProfSlot ps{};
        if (prof) {
            cudaEventCreate(&ps.a);
            cudaEventCreate(&ps.b);
            cudaEventRecord(ps.a, h->work);
        }
        k_sra_pairs<<<pair_blocks, kSraWarps * 32, 0, h->work>>>(
            list, count, rowptr, col, val, *aggptr, *members, prop, agg, newsize, pair_of, flops);
        if (prof) {
            cudaEventRecord(ps.b, h->work);
            h->prof_slots.push_back(ps);
        }
        count_launch(h, 4);
        if ((st = check_cuda(cudaGetLastError()))) return st;
        if ((st = scan_exclusive(h, newsize, ptr2, nc, ptr2 + nc, scan_tmp))) return st;
        k_sra_members<<<grid_for(nc, kThreads), kThreads, 0, h->work>>>(nc, *aggptr, *members,
                                                                       pair_of, agg, ptr2, mem2);
        count_launch(h);
        if ((st = check_cuda(cudaGetLastError()))) return st;
        std::swap(*aggptr, ptr2);
        std::swap(*members, mem2);
    }
    if (prof) {
        unsigned long long f = 0ull;
        st = check_cuda(cudaMemcpyAsync(&f, flops, sizeof(f), cudaMemcpyDeviceToHost, h->work));
        if (st == UAAMG_OK) st = check_cuda(cudaStreamSynchronize(h->work));
        h->prof_bytes = (double)f;
    }
    return st;
}

}  // namespace uaamg
