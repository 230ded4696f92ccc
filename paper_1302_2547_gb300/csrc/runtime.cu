// runtime.cu -- device-memory pool, page-locked host blocks, budget accounting, launch
// counters, status strings.
//
// All device memory of a handle comes from a per-device CUDA memory pool owned by the
// library (stream-ordered allocation on the handle's stream, release threshold = never),
// so repeated setups reuse pool memory instead of calling the driver allocator.  A
// library-wide byte budget lets a serving layer admit work by device memory.
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "pinned.cuh"

namespace uaamg {

static std::atomic<long long> g_launches{0};
static std::atomic<unsigned long long> g_bytes{0};
static std::atomic<unsigned long long> g_budget{0};
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_ok[64];

int check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return UAAMG_OK;
    if (e == cudaErrorMemoryAllocation) return UAAMG_ERR_OOM;
    return UAAMG_ERR_CUDA;
}

static cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) return nullptr;
        uint64_t never = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &never);
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}

// ---- page-locked host blocks (pinned.cuh) --------------------------------------------------
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free[48];           // free blocks by size class 2^c
static std::unordered_map<void*, int> g_pin_class;  // every block handed out, by class

void* pinned_get(size_t bytes) {
    int c = 8;  // 256 bytes at least
    while (c < 47 && ((size_t)1 << c) < bytes) c++;
    if (((size_t)1 << c) < bytes) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free[c].empty()) {
            void* p = g_pin_free[c].back();
            g_pin_free[c].pop_back();
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, (size_t)1 << c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_class[p] = c;
    return p;
}

void pinned_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_pin_class.find(p);
    if (it != g_pin_class.end()) g_pin_free[it->second].push_back(p);
}

void* dalloc_bytes(Handle* h, size_t bytes, int* status, bool temp) {
    if (*status != UAAMG_OK) return nullptr;
    // at least 32 bytes of tail padding: bulk copies round their ranges up to 16-byte
    // boundaries, which can reach 3 FP64 elements (24 bytes) past the end
    bytes = (bytes + 32 + 255) & ~(size_t)255;
    unsigned long long budget = g_budget.load();
    unsigned long long now = g_bytes.fetch_add(bytes) + bytes;
    if (budget && now > budget) {
        g_bytes.fetch_sub(bytes);
        *status = UAAMG_ERR_BUDGET;
        return nullptr;
    }
    cudaMemPool_t pool = pool_for(h->device);
    void* ptr = nullptr;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&ptr, bytes, pool, h->work)
                         : cudaErrorInitializationError;
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_bytes.fetch_sub(bytes);
        *status = check_cuda(e);
        return nullptr;
    }
    if (temp) {
        h->temps.push_back({ptr, bytes});
    } else {
        h->allocs.push_back(ptr);
        h->bytes += bytes;
    }
    return ptr;
}

void dfree_one(Handle* h, void* ptr, size_t bytes) {
    if (!ptr) return;
    bytes = (bytes + 32 + 255) & ~(size_t)255;  // as dalloc_bytes rounded it
    for (size_t k = 0; k < h->allocs.size(); k++) {
        if (h->allocs[k] != ptr) continue;
        h->allocs[k] = h->allocs.back();
        h->allocs.pop_back();
        cudaFreeAsync(ptr, h->work);
        g_bytes.fetch_sub(bytes);
        h->bytes -= bytes;
        return;
    }
}

void dfree_temps(Handle* h) {
    for (auto& t : h->temps) {
        cudaFreeAsync(t.first, h->work);
        g_bytes.fetch_sub(t.second);
    }
    h->temps.clear();
}

void dfree_all(Handle* h) {
    dfree_temps(h);
    for (void* p : h->allocs) cudaFreeAsync(p, h->work);
    h->allocs.clear();
    g_bytes.fetch_sub(h->bytes);
    h->bytes = 0;
}

void count_launch(Handle* h, long long k) {
    if (h->capturing) {  // kernels recorded into a graph count once per replay
        h->graph_nodes += k;
        return;
    }
    h->launches += k;
    g_launches.fetch_add(k);
}

int grid_for(long long items, int per_block) {
    long long g = (items + per_block - 1) / per_block;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace uaamg

extern "C" {

int64_t uaamg_total_launches(void) { return uaamg::g_launches.load(); }

int uaamg_set_memory_budget(uint64_t bytes) {
    uaamg::g_budget.store(bytes);
    return UAAMG_OK;
}

uint64_t uaamg_memory_in_use(void) { return uaamg::g_bytes.load(); }

const char* uaamg_status_string(int s) {
    switch (s) {
        case UAAMG_OK: return "ok";
        case UAAMG_ERR_INVALID_ARG: return "invalid argument";
        case UAAMG_ERR_BAD_CSR: return "malformed CSR matrix";
        case UAAMG_ERR_NOT_SPD: return "coarsest matrix is not positive definite";
        case UAAMG_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
        case UAAMG_ERR_OOM: return "device allocation failed";
        case UAAMG_ERR_BUDGET: return "device-memory budget exceeded";
        case UAAMG_ERR_CUDA: return "CUDA runtime error";
        case UAAMG_ERR_TIMEOUT: return "bounded device wait timed out";
        case UAAMG_ERR_UNSUPPORTED: return "size beyond this build's limits";
        case UAAMG_ERR_CANCELLED: return "request cancelled";
        default: return "unknown status";
    }
}

}  // extern "C"
