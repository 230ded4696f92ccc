// kern_scan.cu -- exclusive prefix sum of int32 arrays (Blelloch-style, three launches:
// tile sums, scan of the tile sums in one block, scan of each tile with its offset; one
// launch for arrays of at most 16384 ints).  Used for the ascending coarse numbering of
// Section 5.1 and for CSR row pointers.
#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;
constexpr int kScanTopThreads = 1024;

template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
    __shared__ int ws[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < NT / 32) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) ws[lane] = w;
    }
    __syncthreads();
    int pre = wid > 0 ? ws[wid - 1] : 0;
    *total = ws[NT / 32 - 1];
    __syncthreads();
    return pre + x - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_tile_sums(const int* __restrict__ in, int n,
                                                             int* __restrict__ bsum) {
    const long long base = (long long)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = threadIdx.x; k < kScanTile; k += kThreads) {
        long long i = base + k;
        if (i < n) s += in[i];
    }
    int tot;
    block_exclusive_scan<kThreads>(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanTopThreads) k_scan_top(int* __restrict__ bsum, int nb,
                                                             int* __restrict__ total) {
    const int seg = (nb + kScanTopThreads - 1) / kScanTopThreads;
    const int lo = min(nb, (int)threadIdx.x * seg), hi = min(nb, lo + seg);
    int s = 0;
    for (int i = lo; i < hi; i++) s += bsum[i];
    int tot;
    int pre = block_exclusive_scan<kScanTopThreads>(s, &tot);
    for (int i = lo; i < hi; i++) {
        int v = bsum[i];
        bsum[i] = pre;
        pre += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int* __restrict__ in, int n,
                                                         const int* __restrict__ boff,
                                                         int* __restrict__ out) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + k;
        v[k] = (i < n) ? in[i] : 0;
        s += v[k];
    }
    int tot;
    int pre = block_exclusive_scan<kThreads>(s, &tot) + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
}

// Arrays of at most kScanSmallN ints in one launch: each of 1024 threads scans a contiguous
// run of kScanSmallItems, and one block scan adds the runs' offsets.
constexpr int kScanSmallItems = 16;
constexpr int kScanSmallN = kScanTopThreads * kScanSmallItems;

__global__ void __launch_bounds__(kScanTopThreads) k_scan_small(const int* __restrict__ in, int n,
                                                               int* __restrict__ out,
                                                               int* __restrict__ total) {
    const int lo = min(n, (int)threadIdx.x * kScanSmallItems);
    const int hi = min(n, lo + kScanSmallItems);
    int v[kScanSmallItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanSmallItems; k++) {
        v[k] = (lo + k < hi) ? in[lo + k] : 0;
        s += v[k];
    }
    int tot;
    int pre = block_exclusive_scan<kScanTopThreads>(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanSmallItems; k++) {
        if (lo + k < hi) out[lo + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

size_t scan_scratch_ints(long long n) { return (size_t)grid_for(n, kScanTile) + 1; }

// out[i] = sum_{k<i} in[i]; *d_total = sum of all (device int, may be null).  `scratch`
// holds scan_scratch_ints(n) ints.  in and out may alias.
int scan_exclusive(Handle* h, const int* in, int* out, int n, int* d_total, int* scratch) {
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(int), h->work);
        return check_cuda(cudaGetLastError());
    }
    if (n <= kScanSmallN) {
        k_scan_small<<<1, kScanTopThreads, 0, h->work>>>(in, n, out, d_total);
        count_launch(h);
        return check_cuda(cudaGetLastError());
    }
    int nb = grid_for(n, kScanTile);
    k_scan_tile_sums<<<nb, kThreads, 0, h->work>>>(in, n, scratch);
    k_scan_top<<<1, kScanTopThreads, 0, h->work>>>(scratch, nb, d_total);
    k_scan_tiles<<<nb, kThreads, 0, h->work>>>(in, n, scratch, out);
    count_launch(h, 3);
    return check_cuda(cudaGetLastError());
}

}  // namespace uaamg
