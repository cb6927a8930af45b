// Changed-set extraction that allocates nothing (gs_extract_delta_noalloc).
//
// Some callers cannot allocate device memory when they need a delta: a
// streaming sender on a real-time thread (an engine render-thread callback
// that ships tensor deltas every frame) must not call cudaMalloc, which can
// block on the device for an unbounded time, and a host whose device memory
// belongs to another allocator (an engine's fixed budget, a caching
// allocator) may have no way to hand this library a workspace or a context.
// This entry point needs neither: its scratch (one flag byte per Gaussian and
// one count per 256 Gaussians) lives in a file-scope device array of fixed
// size, which every GPU that loads the library holds until the process exits.
//
// Limits and sharing:
//  - n must not exceed GS_NOALLOC_MAX_GAUSSIANS (larger n is rejected with
//    GS_ERR_CAPACITY before anything is enqueued);
//  - all calls on one device share the array; its previous contents never
//    matter, because each call writes every flag and every count it reads
//    before reading it, so nothing is cleared;
//  - calls whose work overlaps on the GPU (different streams without an
//    ordering between them) race on the shared array and must not be issued;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current) and keeps it for the
//    life of the process; make that first call outside any stream capture;
//  - the kept address belongs to the device's primary context: after a
//    reset of that context (cudaDeviceReset) it is stale, and the call must
//    not be used again in that process.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int64_t kMaxN = GS_NOALLOC_MAX_GAUSSIANS;
// flags (kMaxN bytes) and block counts, laid out as gs::launch_delta carves
// them (256-byte aligned pieces)
constexpr size_t kScratchBytes = ((kMaxN + 255) / 256) * 256 + ((kMaxN + 255) / 256 + 1) * 4 + 256;

static __device__ __align__(256) unsigned char g_delta_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
gs_status_t scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_delta_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GS_OK;
}

}  // namespace

extern "C" gs_status_t gs_extract_delta_noalloc(const float* theta, float* baseline, int64_t n, float thr,
                                                uint32_t* d_idx, uint8_t* d_records, uint32_t* d_count,
                                                void* stream) {
    if (n < 0 || !d_count || (n > 0 && (!theta || !baseline || !d_idx || !d_records)) || !(thr >= 0.f))
        return GS_ERR_ARG;
    if (n > kMaxN || gs::delta_scratch_bytes(n) > kScratchBytes) return GS_ERR_CAPACITY;
    void* scratch = nullptr;
    const gs_status_t s = scratch_address(&scratch);
    if (s != GS_OK) return s;
    gs::launch_delta(theta, baseline, n, thr, d_idx, d_records, d_count, static_cast<char*>(scratch),
                     static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
