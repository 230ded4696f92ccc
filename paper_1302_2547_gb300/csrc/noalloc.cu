// noalloc.cu -- uaamg_aggregate_static: the aggregation of one graph level (priorities,
// aggregation passes, ascending coarse numbering) without any device allocation.
//
// Some callers cannot allocate device memory: code that runs under an external memory
// manager that owns all of the device's memory, or a host thread that must not call
// cudaMalloc / cudaFree because those calls synchronise the device or are forbidden while
// other work is in flight.  This entry point takes only the caller's input and output
// buffers.  Its scratch lives in the file-scope device array below, which every GPU that
// loads the library holds until the process exits (kStaticBytes, about 19 MB), so the
// graph may have at most kStaticMaxN vertices.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace uaamg {

constexpr int kStaticMaxN = 1 << 18;  // largest graph this entry point accepts (vertices)

constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kScanInts = (size_t)kStaticMaxN / 2048 + 2;
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffTot = a256(kOffCtrl + sizeof(Ctrl));
constexpr size_t kOffSlots = a256(kOffTot + 4 * sizeof(int));
constexpr size_t kOffPrio = a256(kOffSlots + sizeof(int) * (size_t)kMaxRoundSlots);
constexpr size_t kOffB1 = a256(kOffPrio + sizeof(uint64_t) * kStaticMaxN);
constexpr size_t kOffState = a256(kOffB1 + 2 * sizeof(uint64_t) * kStaticMaxN);
constexpr size_t kOffBlocked = a256(kOffState + kStaticMaxN);
constexpr size_t kOffList = a256(kOffBlocked + kStaticMaxN);
constexpr size_t kOffCprio = a256(kOffList + 2 * sizeof(int) * kStaticMaxN);
constexpr size_t kOffRootOf = a256(kOffCprio + sizeof(uint64_t) * kStaticMaxN);
constexpr size_t kOffAggSize = a256(kOffRootOf + sizeof(int) * kStaticMaxN);
constexpr size_t kOffPassOf = a256(kOffAggSize + sizeof(int) * kStaticMaxN);
constexpr size_t kOffF = a256(kOffPassOf + sizeof(int) * kStaticMaxN);
constexpr size_t kOffG = a256(kOffF + sizeof(int) * kStaticMaxN);
constexpr size_t kOffAggptr = a256(kOffG + sizeof(int) * kStaticMaxN);
constexpr size_t kOffMembers = a256(kOffAggptr + sizeof(int) * (kStaticMaxN + 1));
constexpr size_t kOffScan = a256(kOffMembers + sizeof(int) * kStaticMaxN);
constexpr size_t kStaticBytes = a256(kOffScan + sizeof(int) * kScanInts);

// The scratch of uaamg_aggregate_static.  In host code this name is only a host-side
// stand-in; the kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

static std::mutex g_static_mu;
static unsigned char* g_static_addr[64];  // device address of the array, per device

// Once per device, with that device current: look up the array's device address.
static int static_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return UAAMG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return check_cuda(e);
        }
        g_static_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_addr[dev];
    return UAAMG_OK;
}

static uint32_t static_level_salt(uint64_t seed) { return (uint32_t)(seed ^ (seed >> 32)); }

}  // namespace uaamg

using namespace uaamg;

extern "C" int uaamg_aggregate_static(const uaamg_csr* A, int32_t max_agg_size,
                                      int32_t pass_mode, uint64_t seed, int32_t* agg,
                                      int32_t* nc, void* stream) {
    if (!A || !agg || !nc || !A->rowptr || !A->col || !A->val || !A->on_device || A->n < 1 ||
        A->nnz < A->n || max_agg_size < 0 || max_agg_size == 1 ||
        (pass_mode != UAAMG_PASS_SINGLE_ROUND && pass_mode != UAAMG_PASS_MAXIMAL))
        return UAAMG_ERR_INVALID_ARG;
    if (A->n > kStaticMaxN) return UAAMG_ERR_UNSUPPORTED;
    Handle h;  // no allocation: every buffer below points into the static array
    int st = check_cuda(cudaGetDevice(&h.device));
    if (st == UAAMG_OK)
        st = check_cuda(cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device));
    unsigned char* s = nullptr;
    if (st == UAAMG_OK) st = static_scratch(h.device, &s);
    if (st != UAAMG_OK) return st;
    h.work = (cudaStream_t)stream;
    h.user = h.work;
    h.ctrl = reinterpret_cast<Ctrl*>(s + kOffCtrl);
    int* d_tot = reinterpret_cast<int*>(s + kOffTot);
    PaaBuffers pb;
    pb.state = s + kOffState;
    pb.b1 = reinterpret_cast<uint64_t*>(s + kOffB1);
    pb.blocked = s + kOffBlocked;
    pb.list = reinterpret_cast<int*>(s + kOffList);
    pb.cprio = reinterpret_cast<uint64_t*>(s + kOffCprio);
    pb.root_of = reinterpret_cast<int*>(s + kOffRootOf);
    pb.agg_size = reinterpret_cast<int*>(s + kOffAggSize);
    pb.slots = reinterpret_cast<int*>(s + kOffSlots);
    uint64_t* prio = reinterpret_cast<uint64_t*>(s + kOffPrio);
    int* pass_of = reinterpret_cast<int*>(s + kOffPassOf);
    int* f = reinterpret_cast<int*>(s + kOffF);
    int* g = reinterpret_cast<int*>(s + kOffG);
    int* aggptr = reinterpret_cast<int*>(s + kOffAggptr);
    int* members = reinterpret_cast<int*>(s + kOffMembers);
    int* scan_tmp = reinterpret_cast<int*>(s + kOffScan);
    const int n = A->n;

    // the array keeps the previous call's contents: clear the words that must start at zero
    if ((st = check_cuda(cudaMemsetAsync(h.ctrl, 0, sizeof(Ctrl), h.work)))) return st;
    if ((st = check_cuda(cudaMemsetAsync(d_tot, 0, 4 * sizeof(int), h.work)))) return st;
    Ctrl hc{};
    int tot[4] = {0, 0, 0, 0};
    if ((st = launch_validate(&h, n, A->nnz, A->rowptr, A->col, A->val))) return st;
    cudaMemcpyAsync(&hc, h.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h.work);
    if ((st = check_cuda(cudaStreamSynchronize(h.work)))) return st;
    if (hc.err) return UAAMG_ERR_BAD_CSR;
    if ((st = launch_priority(&h, n, A->rowptr, A->col, static_level_salt(seed), prio))) return st;
    if ((st = launch_paa(&h, 0, n, A->nnz, A->rowptr, A->col, prio, max_agg_size, pass_mode, pb,
                          pass_of)))
        return st;
    if ((st = launch_root_flags(&h, n, pb.root_of, pb.agg_size, f, g))) return st;
    if ((st = scan_exclusive(&h, f, f, n, d_tot, scan_tmp))) return st;
    if ((st = scan_exclusive(&h, g, g, n, nullptr, scan_tmp))) return st;
    // the numbering indexes by the roots the passes wrote: only after they all finished
    cudaMemcpyAsync(&hc, h.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h.work);
    if ((st = check_cuda(cudaStreamSynchronize(h.work)))) return st;
    if (hc.err & kErrTimeout) return UAAMG_ERR_TIMEOUT;
    if (hc.err & kErrSlots) return UAAMG_ERR_UNSUPPORTED;
    if (hc.err) return UAAMG_ERR_CUDA;
    if ((st = launch_renumber(&h, n, pb.root_of, f, g, A->rowptr, A->col, d_tot, agg, aggptr,
                              members)))
        return st;
    cudaMemcpyAsync(&hc, h.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h.work);
    cudaMemcpyAsync(tot, d_tot, sizeof(tot), cudaMemcpyDeviceToHost, h.work);
    if ((st = check_cuda(cudaStreamSynchronize(h.work)))) return st;
    if (hc.err & kErrTimeout) return UAAMG_ERR_TIMEOUT;
    if (hc.err & kErrSlots) return UAAMG_ERR_UNSUPPORTED;
    if (hc.err) return UAAMG_ERR_CUDA;
    *nc = tot[0];
    return UAAMG_OK;
}
