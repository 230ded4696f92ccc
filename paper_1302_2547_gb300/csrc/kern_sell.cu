// kern_sell.cu -- sliced ELLPACK (SELL-32) copies of the large levels and the row kernels that
// read them (the ELL-style storage of Section 4.4, for levels of nearly uniform row length).
//
// Slice s holds rows [32 s, 32 s + 32).  Its width w_s is the longest of those rows; its
// entries are stored column-major, entry k of row 32 s + lane at sptr[s] + 32 k + lane, so
// the 32 lanes of a warp read each of the slice's columns with one coalesced 128-byte
// (FP32) or 256-byte (FP64) access, with no row pointers and no shared-memory staging.
// Padding entries (k >= the row's length) are zero and never used.  Each lane adds its row
// in stored order with fused multiply-adds and applies the same epilogue as the other
// row kernels, so every vector entry is bit-identical to theirs with one thread per row.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kSellBatch = 8;  // columns whose loads and gathers a lane has in flight

// One warp per slice: row lengths (16-bit) and 32 * the slice width; tot[1] = longest row.
__global__ void __launch_bounds__(kThreads)
k_sell_width(int n, const int* __restrict__ rowptr, uint16_t* __restrict__ len,
             int* __restrict__ w32, int* tot) {
    const int s = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ns = (n + 31) >> 5;
    if (s >= ns) return;  // whole warps leave together
    const int row = (s << 5) + lane;
    const int l = row < n ? rowptr[row + 1] - rowptr[row] : 0;
    if (row < n) len[row] = (uint16_t)(l < 65535 ? l : 65535);
    int w = l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (lane == 0) {
        w32[s] = 32 * w;
        atomicMax(tot + 1, w);
    }
}

// One thread per row: its entries into the slice layout.
__global__ void __launch_bounds__(kThreads)
k_sell_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
            const double* __restrict__ val64, const float* __restrict__ val32,
            const int* __restrict__ sptr, int* __restrict__ scol, double* __restrict__ sval64,
            float* __restrict__ sval32) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int k0 = rowptr[row], l = rowptr[row + 1] - k0;
    const int base = sptr[row >> 5] + (row & 31);
    for (int k = 0; k < l; k++) {
        const int d = base + 32 * k;
        scol[d] = col[k0 + k];
        sval64[d] = val64[k0 + k];
        if (sval32) sval32[d] = val32[k0 + k];
    }
}

int build_sell(Handle* h, Level& L, bool mixed) {
    int st = UAAMG_OK;
    const int ns = (L.n + 31) / 32;
    int* w32 = dalloc<int>(h, ns, &st, true);
    int* tot = dalloc<int>(h, 4, &st, true);
    int* scan_tmp = dalloc<int>(h, scan_scratch_ints(ns), &st, true);
    int* sptr = dalloc<int>(h, (size_t)ns + 1, &st);
    uint16_t* len = dalloc<uint16_t>(h, L.n, &st);
    if (st) return st;
    cudaMemsetAsync(tot, 0, 4 * sizeof(int), h->work);
    k_sell_width<<<grid_for(ns, kThreads / 32), kThreads, 0, h->work>>>(L.n, L.rowptr, len, w32, tot);
    count_launch(h);
    if ((st = check_cuda(cudaGetLastError()))) return st;
    int host[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(host, tot, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->work);
    if ((st = check_cuda(cudaStreamSynchronize(h->work)))) return st;
    // rows of at most 65535 entries, and slice offsets that fit 32-bit indices
    if (host[1] > 65535 || 32LL * ns * host[1] > 0x7fffffffLL) return UAAMG_OK;
    if ((st = scan_exclusive(h, w32, sptr, ns, tot, scan_tmp))) return st;
    cudaMemcpyAsync(sptr + ns, tot, sizeof(int), cudaMemcpyDeviceToDevice, h->work);
    cudaMemcpyAsync(host, tot, sizeof(int), cudaMemcpyDeviceToHost, h->work);
    if ((st = check_cuda(cudaStreamSynchronize(h->work)))) return st;
    const long long padded = host[0];
    if (padded > L.nnz + L.nnz / 4) return UAAMG_OK;  // only where padding stays below 25%
    int* scol = dalloc<int>(h, (size_t)padded, &st);
    double* sval64 = dalloc<double>(h, (size_t)padded, &st);
    float* sval32 = mixed ? dalloc<float>(h, (size_t)padded, &st) : nullptr;
    if (st) return st;
    cudaMemsetAsync(scol, 0, sizeof(int) * padded, h->work);
    cudaMemsetAsync(sval64, 0, sizeof(double) * padded, h->work);
    if (sval32) cudaMemsetAsync(sval32, 0, sizeof(float) * padded, h->work);
    k_sell_fill<<<grid_for(L.n, kThreads), kThreads, 0, h->work>>>(
        L.n, L.rowptr, L.col, L.val64, L.val32, sptr, scol, sval64, sval32);
    count_launch(h);
    if ((st = check_cuda(cudaGetLastError()))) return st;
    L.sl_ptr = sptr;
    L.sl_len = len;
    L.sl_col = scol;
    L.sl_val64 = sval64;
    L.sl_val32 = sval32;
    L.sl_ns = ns;
    L.sl_padded = padded;
    return UAAMG_OK;
}

// Releases the level's sliced ELLPACK copy (stream-ordered).
void drop_sell(Handle* h, Level& L) {
    if (!L.sl_ptr) return;
    dfree_one(h, L.sl_ptr, sizeof(int) * ((size_t)L.sl_ns + 1));
    dfree_one(h, L.sl_len, sizeof(uint16_t) * (size_t)L.n);
    dfree_one(h, L.sl_col, sizeof(int) * (size_t)L.sl_padded);
    dfree_one(h, L.sl_val64, sizeof(double) * (size_t)L.sl_padded);
    if (L.sl_val32) dfree_one(h, L.sl_val32, sizeof(float) * (size_t)L.sl_padded);
    L.sl_ptr = nullptr;
    L.sl_len = nullptr;
    L.sl_col = nullptr;
    L.sl_val64 = nullptr;
    L.sl_val32 = nullptr;
    L.sl_ns = 0;
    L.sl_padded = 0;
}

template <typename T, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) k_sell(RBArgs<T> a) {
    if (!rb_enter<T, MODE>(a)) return;
    const KScal<T> ks = kscal<T, MODE>(a);
    const int lane = threadIdx.x & 31;
    const int W = gridDim.x * (kThreads / 32);
    double dv[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); k++) dv[k] = 0.0;
    for (int s = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); s < a.nslices; s += W) {
        const int row = (s << 5) + lane;
        const bool valid = row < a.n;
        const int p0 = a.sptr[s];
        const int width = (a.sptr[s + 1] - p0) >> 5;
        const int len = valid ? (int)a.slen[row] : 0;
        RowOps<T> o{};
        if (valid) o = rb_row_ops<T, MODE, ND>(a, ks, row);
        const int* cp = a.scol + p0 + lane;
        const T* vp = a.sval + p0 + lane;
        T acc = T(0);
        for (int k0 = 0; k0 < width; k0 += kSellBatch) {
            int c[kSellBatch];
            T v[kSellBatch], x[kSellBatch];
#pragma unroll
            for (int u = 0; u < kSellBatch; u++) {
                const bool in = k0 + u < width;
                c[u] = in ? __ldcs(cp + 32 * (k0 + u)) : 0;
                v[u] = in ? __ldcs(vp + 32 * (k0 + u)) : T(0);
            }
#pragma unroll
            for (int u = 0; u < kSellBatch; u++)
                x[u] = (k0 + u < len) ? rb_gather<T, MODE>(a, ks, c[u]) : T(0);
#pragma unroll
            for (int u = 0; u < kSellBatch; u++)
                if (k0 + u < len) acc = fma_rn(v[u], x[u], acc);
        }
        if (valid) rb_row_out<T, MODE, ND>(a, ks, row, acc, o, dv);
    }
    if constexpr (ND > 0) {
        if (grid_reduce<ND>(dv, a.partials, a.counter, a.result)) rb_last_block(a);
    }
}

// A persistent grid (resident blocks x SMs) walks the slices: few blocks arrive at the
// final reduction, and each warp keeps several slices' loads coming.
template <typename T, int MODE, int ND>
static int launch_sell_one(Handle* h, const RBArgs<T>& a) {
    static DevCache occ;
    int per_sm = occ.get(h->device);
    if (!per_sm) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sell<T, MODE, ND>, kThreads, 0);
        per_sm = b > 0 ? b : 1;
        occ.set(h->device, per_sm);
    }
    int grid = grid_for(a.nslices, kThreads / 32);
    if (grid > per_sm * h->num_sms) grid = per_sm * h->num_sms;
    k_sell<T, MODE, ND><<<grid, kThreads, 0, h->work>>>(a);
    count_launch(h);
    return check_cuda(cudaGetLastError());
}

template <typename T>
int launch_sell(Handle* h, int mode, int ndots, const RBArgs<T>& a) {
#define SELL_CASE(M, D) \
    if (mode == M && ndots == D) return launch_sell_one<T, M, D>(h, a);
    SELL_CASE(RB_PRE1, 0)
    SELL_CASE(RB_PRE1_RT, 0)
    SELL_CASE(RB_PROSMOOTH_E, 0)
    SELL_CASE(RB_SMOOTH, 0)
    SELL_CASE(RB_RESID, 0)
    SELL_CASE(RB_RESID, 1)
    SELL_CASE(RB_PROSMOOTH, 0)
    SELL_CASE(RB_SPMV, 0)
    SELL_CASE(RB_SPMV, 2)
    SELL_CASE(RB_SPMV, 3)
#undef SELL_CASE
    return UAAMG_ERR_INVALID_ARG;
}
template int launch_sell<float>(Handle*, int, int, const RBArgs<float>&);
template int launch_sell<double>(Handle*, int, int, const RBArgs<double>&);

}  // namespace uaamg
