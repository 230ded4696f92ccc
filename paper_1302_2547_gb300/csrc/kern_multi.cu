// kern_multi.cu -- the solve-phase kernels for R right-hand sides at once (uaamg_solve_many).
//
// Vectors are interleaved, element (i, r) at i*R + r, so the R values of one row are
// contiguous.  A block of 256 threads owns 256/Rp rows (Rp = R rounded up to a power of
// two); thread (row, r) walks its row once, and the R threads of a row read the same matrix
// entry (one transaction) and gather x[j*R + r] from one contiguous run: every matrix
// entry is read once for all R columns.  Each column keeps its own K-cycle and outer scalars
// (per-column arrays), so column r follows exactly the single-vector algorithm.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kMColMax = 32;  // most right-hand sides one multi-vector call carries

struct MGeom {
    int R, Rp, lgRp, rows_per_block;
};

__host__ __device__ inline MGeom mgeom(int R) {
    int lg = 0;
    while ((1 << lg) < R) lg++;
    MGeom g;
    g.R = R;
    g.Rp = 1 << lg;
    g.lgRp = lg;
    g.rows_per_block = kThreads >> lg;
    return g;
}

// Deterministic per-column reduction of ND values over the whole grid: rows of a block are
// reduced by a fixed tree in shared memory, blocks by the last block in a fixed order
// (block slices per (value, column) pair, then the slices in order).
template <int ND>
__device__ void grid_reduce_cols(const double (&v)[ND], const MGeom& g, double* partials,
                                 unsigned int* counter, double* result /* [ND][R] */) {
    __shared__ double sh[ND][kThreads];
    __shared__ double sl[kThreads];
    __shared__ bool is_last;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < ND; k++) sh[k][t] = v[k];
    __syncthreads();
    for (int s = g.rows_per_block >> 1; s > 0; s >>= 1) {
        if ((t >> g.lgRp) < s) {
#pragma unroll
            for (int k = 0; k < ND; k++) sh[k][t] += sh[k][t + (s << g.lgRp)];
        }
        __syncthreads();
    }
    if (t < g.R) {
#pragma unroll
        for (int k = 0; k < ND; k++) partials[((size_t)blockIdx.x * ND + k) * g.R + t] = sh[k][t];
    }
    __threadfence();
    __syncthreads();
    if (t == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int np = ND * g.R;
    const int slices = kThreads / np;
    double acc = 0.0;
    if (t < slices * np) {
        const int pair = t % np, slice = t / np;
        for (unsigned int b = slice; b < gridDim.x; b += slices)
            acc += __ldcg(&partials[(size_t)b * np + pair]);
    }
    sl[t] = acc;
    __syncthreads();
    if (t < np) {
        double s = 0.0;
        for (int q = 0; q < slices; q++) s += sl[q * np + t];
        result[t] = s;
        if (t == 0) *counter = 0u;
    }
}

// Blocks of the row-parallel kernels: enough to fill the GPU; rows are grid-strided.
inline int mgrid(const Handle* h, int n, const MGeom& g) {
    int need = grid_for(n, g.rows_per_block);
    int cap = 16 * h->num_sms;
    return need < cap ? need : cap;
}

template <typename T, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) k_mrow(MArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    const MGeom g = mgeom(a.R);
    const int lr = threadIdx.x & (g.Rp - 1);
    const int R = a.R;
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    for (int i = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp); i < a.n;
         i += gridDim.x * g.rows_per_block) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        T acc = T(0);
        for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; k++) {
            const int j = a.col[k];
            const size_t oj = (size_t)j * R + lr;
            T xj;
            if constexpr (MODE == RB_PRE1) xj = mul_rn(a.minv[j], a.r[oj]);
            else if constexpr (MODE == RB_PROSMOOTH) xj = add_rn(a.x[oj], a.e[(size_t)a.agg[j] * R + lr]);
            else xj = a.x[oj];
            acc = fma_rn(a.val[k], xj, acc);
        }
        if constexpr (MODE == RB_PRE1) {
            a.y[o] = mul_rn(a.minv[i], a.r[o]);
            a.y2[o] = sub_rn(a.r[o], acc);
        } else if constexpr (MODE == RB_SMOOTH) {
            a.y[o] = add_rn(a.x[o], mul_rn(a.minv[i], sub_rn(a.r[o], acc)));
        } else if constexpr (MODE == RB_RESID) {
            const T yi = sub_rn(a.r[o], acc);
            a.y[o] = yi;
            if constexpr (ND >= 1) dv[0] = fma((double)yi, (double)yi, dv[0]);
        } else if constexpr (MODE == RB_PROSMOOTH) {
            const T xi = add_rn(a.x[o], a.e[(size_t)a.agg[i] * R + lr]);
            a.y[o] = add_rn(xi, mul_rn(a.minv[i], sub_rn(a.r[o], acc)));
        } else {
            a.y[o] = acc;
            const double xi = (double)a.x[o];
            if constexpr (ND >= 1) dv[0] = fma(xi, (double)acc, dv[0]);
            if constexpr (ND >= 2) dv[1] = fma(xi, (double)a.d1[o], dv[1]);
            if constexpr (ND >= 3) dv[2] = fma(xi, (double)a.d2[o], dv[2]);
        }
    }
    if constexpr (ND > 0) grid_reduce_cols<ND>(dv, g, a.partials, a.counter, a.result);
}

template <typename T>
int launch_mrow(Handle* h, int mode, int ndots, const MArgs<T>& a) {
    const MGeom g = mgeom(a.R);
    const int grid = mgrid(h, a.n, g);
    cudaStream_t st = h->work;
#define MR_CASE(M, D)                                       \
    if (mode == M && ndots == D) {                          \
        cudaError_t e = launch_k(a.n <= kPdlMaxRows, k_mrow<T, M, D>, dim3(grid), \
                                 dim3(kThreads), 0, st, a);                      \
        count_launch(h);                                    \
        return check_cuda(e);                               \
    }
    MR_CASE(RB_PRE1, 0)
    MR_CASE(RB_SMOOTH, 0)
    MR_CASE(RB_RESID, 1)
    MR_CASE(RB_PROSMOOTH, 0)
    MR_CASE(RB_SPMV, 2)
    MR_CASE(RB_SPMV, 3)
#undef MR_CASE
    return UAAMG_ERR_INVALID_ARG;
}
template int launch_mrow<float>(Handle*, int, int, const MArgs<float>&);
template int launch_mrow<double>(Handle*, int, int, const MArgs<double>&);

// (P^T s)[I][r] and the exact coarsest solve, one thread per (row, column).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mrestrict(int nc, int R, const int* __restrict__ aggptr, const int* __restrict__ members,
            const T* __restrict__ s, T* __restrict__ rc) {
    pdl_wait();
    pdl_trigger();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nc * R) return;
    const int I = (int)(t / R), r = (int)(t % R);
    const int q1 = aggptr[I + 1];
    T sum = T(0);
    for (int q = aggptr[I]; q < q1; q += 8) {  // members' loads issued together
        int m[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) m[u] = q + u < q1 ? members[q + u] : 0;
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = q + u < q1 ? s[(size_t)m[u] * R + r] : T(0);
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (q + u < q1) sum = add_rn(sum, v[u]);
    }
    rc[t] = sum;
}

// Coarsest solve for R columns: out[i][r] = sum_j inv[i][j] in[j][r] in FP64.  One block
// per row i; its threads split j into 256/Rp chunks for each column, and the chunks' sums
// are added in chunk order in shared memory (a fixed order, so the result is deterministic).
// Spreading the rows over blocks keeps the FP64 work on many SMs.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mdense(int n, int R, const double* __restrict__ inv, const T* __restrict__ in,
         T* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    __shared__ double part[kThreads];
    const MGeom g = mgeom(R);
    const int i = blockIdx.x;
    const int r = threadIdx.x & (g.Rp - 1);
    const int jc = threadIdx.x >> g.lgRp;
    const int nchunks = kThreads >> g.lgRp;
    double s = 0.0;
    if (r < R)
        for (int j = jc; j < n; j += nchunks)
            s = fma(inv[(size_t)i * n + j], (double)in[(size_t)j * R + r], s);
    part[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < R) {
        double t = 0.0;
        for (int c = 0; c < nchunks; c++) t += part[(c << g.lgRp) + threadIdx.x];
        out[(size_t)i * R + threadIdx.x] = (T)t;
    }
}

template <typename T>
int launch_mrestrict(Handle* h, int nc, int R, const int* aggptr, const int* members,
                     const T* s, T* rc) {
    cudaError_t e = launch_k(nc <= kPdlMaxRows, k_mrestrict<T>,
                             dim3(grid_for((long long)nc * R, kThreads)), dim3(kThreads), 0,
                             h->work, nc, R, aggptr, members, s, rc);
    if (e != cudaSuccess) return check_cuda(e);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template <typename T>
int launch_mdense(Handle* h, int n, int R, const double* inv, const T* in, T* out) {
    cudaError_t e = launch_k(true, k_mdense<T>, dim3(n), dim3(kThreads), 0, h->work, n, R, inv,
                             in, out);
    if (e != cudaSuccess) return check_cuda(e);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template int launch_mrestrict<float>(Handle*, int, int, const int*, const int*, const float*, float*);
template int launch_mrestrict<double>(Handle*, int, int, const int*, const int*, const double*, double*);
template int launch_mdense<float>(Handle*, int, int, const double*, const float*, float*);
template int launch_mdense<double>(Handle*, int, int, const double*, const double*, double*);

// K-cycle scalar steps per column (Section 4.3).  sc points at this level's per-column
// scalars: rows [0..R) rho1, [R..2R) alpha1, [2R..3R) beta, [3R..4R) gamma, [4R..5R) alpha2,
// [5R..6R) |rho~|^2, [6R..7R) |rho|^2.  With several columns no kernel is skipped: the
// second step is computed for every column and ignored by the combine where the
// single-vector algorithm would skip it.
template <typename T, bool TAU>
__global__ void __launch_bounds__(kThreads)
k_mkc_rt(int n, int R, const T* __restrict__ rho, const T* __restrict__ v1, T* __restrict__ rt,
         double* sc, double* partials, unsigned int* counter) {
    pdl_wait();
    pdl_trigger();
    const MGeom g = mgeom(R);
    const int lr = threadIdx.x & (g.Rp - 1);
    double dv[2] = {0.0, 0.0};
    __shared__ double sa1[kMColMax];  // alpha1 / rho1 per column, once per block
    if ((int)threadIdx.x < R) {
        const double rho1 = sc[threadIdx.x], alpha1 = sc[R + threadIdx.x];
        sa1[threadIdx.x] = rho1 > 0.0 ? alpha1 / rho1 : 0.0;
    }
    __syncthreads();
    const T a1 = (T)(lr < R ? sa1[lr] : 0.0);
    for (int i = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp); i < n;
         i += gridDim.x * g.rows_per_block) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        const T v = sub_rn(rho[o], mul_rn(a1, v1[o]));
        rt[o] = v;
        if constexpr (TAU) {
            dv[0] = fma((double)v, (double)v, dv[0]);
            dv[1] = fma((double)rho[o], (double)rho[o], dv[1]);
        }
    }
    if constexpr (TAU) grid_reduce_cols<2>(dv, g, partials, counter, sc + 5 * R);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mkc_combine(int n, int R, const T* __restrict__ c1, const T* __restrict__ c2,
              T* __restrict__ e, const double* sc, int second, double tau) {
    pdl_wait();
    pdl_trigger();
    const MGeom g = mgeom(R);
    const int lr = threadIdx.x & (g.Rp - 1);
    const int i = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp);
    __shared__ double sw[2][kMColMax];  // the column's weights, once per block
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        const double rho1 = sc[c], alpha1 = sc[R + c];
        double w1 = 0.0, w2 = 0.0;
        if (rho1 > 0.0) {
            w1 = alpha1 / rho1;
            bool two = second != 0;
            if (two && tau > 0.0 && sqrt(sc[5 * R + c]) <= tau * sqrt(sc[6 * R + c])) two = false;
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
    if (i >= n || lr >= R) return;
    const double w1 = sw[0][lr], w2 = sw[1][lr];
    const size_t o = (size_t)i * R + lr;
    T v = mul_rn((T)w1, c1[o]);
    if (w2 != 0.0) v = add_rn(v, mul_rn((T)w2, c2[o]));
    e[o] = v;
}

template <typename T>
int launch_mkc_rt(Handle* h, int n, int R, const T* rho, const T* v1, T* rt, double* sc,
                  bool tau) {
    const MGeom g = mgeom(R);
    const int grid = mgrid(h, n, g);
    if (tau)
        k_mkc_rt<T, true><<<grid, kThreads, 0, h->work>>>(n, R, rho, v1, rt, sc, h->partials, &h->ctrl->red_count);
    else
        {
            cudaError_t e = launch_k(n <= kPdlMaxRows, k_mkc_rt<T, false>, dim3(grid),
                                     dim3(kThreads), 0, h->work, n, R, rho, v1, rt, sc,
                                     h->partials, &h->ctrl->red_count);
            if (e != cudaSuccess) return check_cuda(e);
        }
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template <typename T>
int launch_mkc_combine(Handle* h, int n, int R, const T* c1, const T* c2, T* e,
                       const double* sc, int second, double tau) {
    const MGeom g = mgeom(R);
    cudaError_t err = launch_k(n <= kPdlMaxRows, k_mkc_combine<T>,
                               dim3(grid_for(n, g.rows_per_block)), dim3(kThreads), 0, h->work,
                               n, R, c1, c2, e, sc, second, tau);
    if (err != cudaSuccess) return check_cuda(err);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template int launch_mkc_rt<float>(Handle*, int, int, const float*, const float*, float*, double*, bool);
template int launch_mkc_rt<double>(Handle*, int, int, const double*, const double*, double*, double*, bool);
template int launch_mkc_combine<float>(Handle*, int, int, const float*, const float*, float*, const double*, int, double);
template int launch_mkc_combine<double>(Handle*, int, int, const double*, const double*, double*, const double*, int, double);

// ---- outer flexible CG per column (FP64) ----------------------------------------------
// os: per-column outer scalars, rows [0..R) pq, [R..2R) pr, [2R..3R) zq, [3R..4R) rr,
// [4R..5R) bb, [5R..6R) pq_prev, [6R..7R) active flag (1.0 / 0.0), [7R..8R) first flag.
__global__ void __launch_bounds__(kThreads)
k_mcast(long long m, const double* __restrict__ in, float* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) out[t] = __double2float_rn(in[t]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mzq(int n, int R, const T* __restrict__ z, const double* __restrict__ q, double* os,
      double* partials, unsigned int* counter) {
    const MGeom g = mgeom(R);
    const int lr = threadIdx.x & (g.Rp - 1);
    const int i0 = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp);
    double dv[1] = {0.0};
    for (int i = i0; i < n; i += gridDim.x * g.rows_per_block) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        dv[0] = fma((double)z[o], q[o], dv[0]);
    }
    grid_reduce_cols<1>(dv, g, partials, counter, os + 2 * R);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mp(long long m, int R, const T* __restrict__ z, double* __restrict__ p, const double* os) {
    __shared__ double sb[kMColMax];  // beta per column, once per block
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        sb[c] = (os[7 * R + c] != 0.0) ? 0.0 : os[2 * R + c] / os[5 * R + c];
    }
    __syncthreads();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const double beta = sb[(int)(t % R)];
    p[t] = fma(-beta, p[t], (double)z[t]);
}

__global__ void __launch_bounds__(kThreads)
k_mxr(int n, int R, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
      const double* __restrict__ q, double* os, double* partials, unsigned int* counter) {
    const MGeom g = mgeom(R);
    const int lr = threadIdx.x & (g.Rp - 1);
    const int i0 = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp);
    double dv[1] = {0.0};
    __shared__ double sal[kMColMax];  // alpha per column, once per block
    if ((int)threadIdx.x < R) {
        const int c = threadIdx.x;
        const double pq = os[c], active = os[6 * R + c];
        sal[c] = (active != 0.0 && pq > 0.0) ? os[R + c] / pq : 0.0;
    }
    __syncthreads();
    const double alpha = lr < R ? sal[lr] : 0.0;
    for (int i = i0; i < n; i += gridDim.x * g.rows_per_block) {
        if (lr >= R) continue;
        const size_t o = (size_t)i * R + lr;
        x[o] = fma(alpha, p[o], x[o]);
        const double ri = fma(-alpha, q[o], r[o]);
        r[o] = ri;
        dv[0] = fma(ri, ri, dv[0]);
    }
    grid_reduce_cols<1>(dv, g, partials, counter, os + 3 * R);
}

__global__ void k_mfinish(int R, double* os) {
    const int r = threadIdx.x;
    if (r < R && os[6 * R + r] != 0.0) {  // active columns advance their recurrence
        os[5 * R + r] = os[r];
        os[7 * R + r] = 0.0;
    }
}

int launch_mcast(Handle* h, long long m, const double* in, float* out) {
    k_mcast<<<grid_for(m, kThreads), kThreads, 0, h->work>>>(m, in, out);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}
template <typename T>
int launch_mouter(Handle* h, int n, int R, const T* z, double* p, const double* q, double* os) {
    const MGeom g = mgeom(R);
    const int grid = mgrid(h, n, g);
    k_mzq<T><<<grid, kThreads, 0, h->work>>>(n, R, z, q, os, h->partials, &h->ctrl->red_count);
    k_mp<T><<<grid_for((long long)n * R, kThreads), kThreads, 0, h->work>>>((long long)n * R, R, z, p, os);
    count_launch(h, 2);
    return check_cuda(cudaGetLastError());
}
template int launch_mouter<float>(Handle*, int, int, const float*, double*, const double*, double*);
template int launch_mouter<double>(Handle*, int, int, const double*, double*, const double*, double*);

int launch_mxr(Handle* h, int n, int R, double* x, double* r, const double* p, const double* q,
               double* os) {
    const MGeom g = mgeom(R);
    k_mxr<<<mgrid(h, n, g), kThreads, 0, h->work>>>(n, R, x, r, p, q, os, h->partials, &h->ctrl->red_count);
    k_mfinish<<<1, 32, 0, h->work>>>(R, os);
    count_launch(h, 2);
    return check_cuda(cudaGetLastError());
}

// (b, b) per column
__global__ void __launch_bounds__(kThreads)
k_mnorm(int n, int R, const double* __restrict__ b, double* out, double* partials,
        unsigned int* counter) {
    const MGeom g = mgeom(R);
    const int lr = threadIdx.x & (g.Rp - 1);
    const int i0 = blockIdx.x * g.rows_per_block + (threadIdx.x >> g.lgRp);
    double dv[1] = {0.0};
    for (int i = i0; i < n; i += gridDim.x * g.rows_per_block) {
        if (lr >= R) continue;
        const double v = b[(size_t)i * R + lr];
        dv[0] = fma(v, v, dv[0]);
    }
    grid_reduce_cols<1>(dv, g, partials, counter, out);
}

int launch_mnorm(Handle* h, int n, int R, const double* b, double* out) {
    const MGeom g = mgeom(R);
    k_mnorm<<<mgrid(h, n, g), kThreads, 0, h->work>>>(n, R, b, out, h->partials, &h->ctrl->red_count);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

}  // namespace uaamg
