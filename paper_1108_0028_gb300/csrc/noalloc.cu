// Neighbour-list offsets for callers that cannot allocate device memory.
//
// rcb_neighbours keeps its per-particle counts and the scan's partial sums in scratch arrays
// that rcb_build allocates with the tree.  Some callers cannot allocate at all when they need the
// offsets: an application whose own memory manager owns the whole device and does not let
// libraries allocate after start-up, for example.  rcb_neighbour_offsets_noalloc gives them the
// same offsets without any allocation: the count pass writes straight into the caller's offsets
// array, and the only other scratch, the exclusive scan's per-tile sums plus the status words,
// lives in the fixed-size array below, compiled into the library and reused by every call.  The
// call reads the total back to the host and synchronises its stream before it returns.
#include <cuda_runtime.h>

#include <mutex>

#include "rcb_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxN = (int64_t)1 << 25;  // 33,554,432 particles
// the scan over N + 1 counts needs scan_tmp_words(N + 1) words; the array holds that for the
// largest N it accepts
constexpr int64_t kScanWords = rcb::scan_tmp_words(kNoAllocMaxN + 1);
constexpr int64_t kStatusWords = 8;  // 16 int32 status words
constexpr int64_t kScratchWords = kScanWords + kStatusWords;

// The static scratch (about 33 KB).  In host code this name is only a stand-in for the symbol;
// the device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) int64_t g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int64_t *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device, looked up once per device and kept
// for the life of the process.  This assumes the device's primary context stays alive: after a
// cudaDeviceReset the cached address is stale and must not be used (the library does not reset
// devices itself).
int scratch_for_current_device(int64_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RCB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RCB_ERR_CUDA;
        g_scratch_ptr[dev] = reinterpret_cast<int64_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return RCB_OK;
}

}  // namespace

extern "C" int rcb_neighbour_offsets_noalloc(rcb_tree *tree, int64_t *offsets, int64_t *needed, void *stream) {
    if (!tree || !offsets || !needed) return RCB_ERR_ARG;
    if (tree->N > kNoAllocMaxN) return RCB_ERR_CAPACITY;
    int64_t *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    tree->stream = st;
    int *status = reinterpret_cast<int *>(scratch + kScanWords);
    // the FP64-decision counter accumulates with atomics: it must start at zero on every call
    RCB_CUDA_TRY(cudaMemsetAsync(status, 0, kStatusWords * sizeof(int64_t), st));
    rc = rcb::neighbour_counts(tree, offsets, status);
    if (rc) return rc;
    rc = rcb::scan_i64(offsets, offsets, tree->N, offsets + tree->N, scratch, st);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemcpyAsync(needed, offsets + tree->N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    return RCB_OK;
}
