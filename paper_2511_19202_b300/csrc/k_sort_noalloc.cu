// nvgs_sort_pairs_noalloc: the S5 radix sort for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits or too costly -- a plugin inside a
// host application that owns every device allocation, a real-time render loop with a fixed
// memory budget where cudaMalloc's implicit device synchronisation would stall the frame, or a
// caller that must not touch the CUDA allocator while its stream is being recorded.  The regular
// entry point (nvgs_sort_pairs) grows context-owned scratch buffers on demand; this one only
// uses a fixed array that lives in the library's device image.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes bytes.  Every GPU that loads
// the library holds it until the process exits.  Host code cannot pass the symbol itself to a
// kernel (in host code it names a host-side stand-in), so the first call on each device looks up
// its device address with cudaGetSymbolAddress while that device is current, and later calls on
// that device reuse it.  Make the first call on a device before any stream capture.  The cached
// address assumes that each device keeps its primary CUDA context for the life of the process:
// after cudaDeviceReset, or from a thread whose current context is another driver-API context
// of the same device, the cached address no longer names the array, so do not call this entry
// point there.  The stream must belong to the current device (checked: a stream of another
// device returns NVGS_ERR_INVALID_ARG).
//
// Every call shares the one array, and the array keeps whatever the last call left in it.
// Nothing in it has to start at zero: each radix pass writes every histogram entry, scan entry
// and alternate key/value slot before reading it.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array; serialise them.
#include <mutex>

#include "nvgs_internal.cuh"

namespace {

constexpr uint64_t kNoAllocMaxPairs = NVGS_SORT_NOALLOC_MAX_PAIRS;
constexpr uint64_t kNoAllocKeys = kNoAllocMaxPairs * 8;   // alternate keys
constexpr uint64_t kNoAllocVals = kNoAllocMaxPairs * 4;   // alternate values
constexpr uint64_t kNoAllocRadix = 1u << 20;              // histograms + scan levels (<= 1 MiB)
constexpr uint64_t kNoAllocBytes = kNoAllocKeys + kNoAllocVals + kNoAllocRadix;

static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" nvgs_status nvgs_sort_pairs_noalloc(uint64_t* keys, uint32_t* values, int64_t n,
                                               int key_bits, void* cuda_stream) {
    if (n < 0 || key_bits < 0 || key_bits > 64) return NVGS_ERR_INVALID_ARG;
    if ((uint64_t)n > kNoAllocMaxPairs) return NVGS_ERR_CAPACITY;
    if (n > 0 && (!keys || !values)) return NVGS_ERR_INVALID_ARG;
    if (n <= 1 || key_bits == 0) return NVGS_OK;
    if (nvgs::radix_scratch_bytes((uint64_t)n) > kNoAllocRadix) return NVGS_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NVGS_ERR_CUDA;
    if (cuda_stream) {   // the scratch address is the current device's: the stream must match
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev) != cudaSuccess) return NVGS_ERR_INVALID_ARG;
        if (sdev != dev) return NVGS_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return NVGS_ERR_CUDA;
    unsigned char* b = static_cast<unsigned char*>(base);
    auto* keys_alt = reinterpret_cast<unsigned long long*>(b);
    auto* vals_alt = reinterpret_cast<uint32_t*>(b + kNoAllocKeys);
    void* radix = b + kNoAllocKeys + kNoAllocVals;
    nvgs::LaunchLog log;  // counting only: records no events
    int passes = 0, in_alt = 0;
    cudaError_t e = nvgs::radix_sort_pairs(reinterpret_cast<unsigned long long*>(keys), values,
                                           keys_alt, vals_alt, (uint64_t)n, key_bits, radix,
                                           (cudaStream_t)cuda_stream, &log, &passes, 1, &in_alt);
    return e == cudaSuccess ? NVGS_OK : NVGS_ERR_CUDA;
}
