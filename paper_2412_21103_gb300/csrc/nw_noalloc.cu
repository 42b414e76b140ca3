// Allocation-free score-only alignment of one pair.
//
// Some callers cannot allocate device memory when they align: a serving
// process that reserved all device memory up front for its own pool, a
// plug-in hosted by a runtime that owns the allocator, or code on a
// latency-critical path where cudaMalloc/cudaFree would synchronize the
// device and stall every other stream.  For them, nw_align_score_noalloc
// keeps the fill kernel's scratch (the stripe boundary rows, the per-stripe
// progress counters and the device error word) in one file-scope device
// array, reserved when the library is loaded and held by every GPU that
// loads it until the process exits.  The call allocates nothing: no
// context, no cudaMalloc/cudaFree, no allocating library routine.
#include <mutex>

#include "nw_internal.cuh"

namespace {

// 12 MiB of scratch per device: 64 words for the error word, 4096 progress
// counters, the rest for boundary rows.
constexpr size_t kStaticWords = 3u << 20;
constexpr uint32_t kErrWords = 64;
constexpr uint32_t kMaxStripes = 4096;
constexpr size_t kRowWords = kStaticWords - kErrWords - kMaxStripes;
constexpr uint32_t kStripeRows = 32u * 16u;  // rows per stripe of the fill used here

__device__ __align__(256) uint32_t g_noalloc_scratch[kStaticWords];

struct DeviceSlot {
    bool ready = false;
    uint32_t *base = nullptr;  // device address of g_noalloc_scratch on that device
    int sm_count = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

}  // namespace

using namespace nw;

extern "C" int nw_align_score_noalloc(const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n,
                                      nw_scoring sc, int32_t *score, void *stream) {
    if (check_scoring(nullptr, sc) != NW_OK) return NW_ERR_ARG;
    if (!score || (m && !a2b) || (n && !b2b)) return NW_ERR_ARG;
    if (m >= (1ull << 30) || n >= (1ull << 30)) return NW_ERR_ARG;
    const uint64_t mn = m < n ? m : n;
    const uint64_t sp = sc.match > 2 * sc.gap ? (uint64_t)(sc.match - 2 * sc.gap) : 0;  // W <= sp * min(i, j)
    if (sp * mn >= (1ull << 29)) return NW_ERR_ARG;
    const uint64_t S = (m + kStripeRows - 1) / kStripeRows;
    const uint64_t bstride = ((n + 1 + 31) / 32) * 32;
    if (S > kMaxStripes || (S > 0 ? (S - 1) * bstride : 0) > kRowWords) return NW_ERR_ARG;  // beyond the maximum

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NW_ERR_CUDA;
    DeviceSlot slot;
    {
        // One-time set-up per device, with that device current: find where
        // the static array lives on it.  Host code cannot use the array's
        // name as a device address.
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceSlot &ds = g_slots[dev];
        if (!ds.ready) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) {
                cudaGetLastError();
                return NW_ERR_CUDA;
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NW_ERR_CUDA;
            ds.base = (uint32_t *)ptr;
            ds.sm_count = sms;
            ds.ready = true;
        }
        slot = ds;
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *err = slot.base;
    uint32_t *progress = slot.base + kErrWords;
    uint32_t *rows = slot.base + kErrWords + kMaxStripes;
    if (m == 0 || n == 0) {
        const int32_t v = sc.gap * (int32_t)(m + n);
        if (cudaMemcpyAsync(score, &v, sizeof v, cudaMemcpyHostToDevice, st) != cudaSuccess) return NW_ERR_CUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? NW_OK : NW_ERR_CUDA;
    }
    // The array keeps the previous call's contents: clear the error word and
    // the progress counters this call waits on.
    if (cudaMemsetAsync(slot.base, 0, (size_t)(kErrWords + S) * sizeof(uint32_t), st) != cudaSuccess)
        return NW_ERR_CUDA;
    if (fill_score_with_scratch(a2b, (uint32_t)m, b2b, (uint32_t)n, sc, score, rows, progress, err, st,
                                slot.sm_count) != cudaSuccess)
        return NW_ERR_CUDA;
    // Read the error word on the caller's stream, then wait for that stream
    // only (a plain cudaMemcpy would also wait for every blocking stream).
    uint32_t h[2] = {0, 0};
    if (cudaMemcpyAsync(h, err, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return NW_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return NW_ERR_CUDA;
    return h[0] ? (int)h[0] : NW_OK;
}
