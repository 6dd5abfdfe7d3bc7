// Neighbor search for callers that cannot allocate device memory.
//
// tnet_neighbors needs a context, and a context needs a caller-allocated
// workspace.  Some callers cannot allocate at all: code running inside
// another framework's memory pool or a strict real-time loop (no cudaMalloc
// allowed after start-up), or plain C callers that have no allocator of
// their own.  tnet_neighbors_noalloc runs the same cell-list search with its
// scratch (system bounds, cell grid, cell histogram, sorted atoms, row
// counts) in one file-scope __device__ array of fixed size.  The caller
// still owns and passes the inputs and outputs.
//
// The array exists once per GPU that loads this library, for the life of
// the process.  All calls share it, so calls whose GPU work overlaps (on
// different streams, or from different threads) race on it; calls ordered
// on one stream are safe.  Each call zeroes what must start at zero.
#include <mutex>
#include <string.h>

#include "internal.cuh"

namespace tnet {
namespace {

constexpr int kNoAllocMaxAtoms = 16384;
constexpr int kNoAllocMaxSystems = 1024;
constexpr size_t kNoAllocScratchBytes = 2u << 20;  // 2 MiB per GPU

static __device__ __align__(256) char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol itself as a device address).
int scratch_address(void **out) {
    int dev = 0;
    TNET_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TNET_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        TNET_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TNET_OK;
}

}  // namespace
}  // namespace tnet

using namespace tnet;

extern "C" int tnet_neighbors_noalloc(int n_atoms, int n_systems, const float *pos, const int32_t *batch,
                                      const float *box, float cutoff, int32_t *row_ptr, int32_t *col,
                                      int64_t cap, int64_t *n_pairs_dev, int32_t *status_dev,
                                      tnet_stream_t stream) {
    if (!pos || !status_dev || !row_ptr || !n_pairs_dev || (cap > 0 && !col)) return TNET_ERR_ARG;
    if (n_atoms < 1 || n_systems < 1 || cap < 0 || cap > 0x7fffffffLL) return TNET_ERR_ARG;
    if (!(cutoff > 0.f) || !isfinite(cutoff) || (n_systems > 1 && !batch)) return TNET_ERR_ARG;
    if (n_atoms > kNoAllocMaxAtoms || n_systems > kNoAllocMaxSystems) {
        fprintf(stderr, "libtnet: tnet_neighbors_noalloc handles at most %d atoms and %d systems "
                        "(got %d, %d)\n", kNoAllocMaxAtoms, kNoAllocMaxSystems, n_atoms, n_systems);
        return TNET_ERR_WORKSPACE;
    }
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // a host-side context whose workspace is the static array, laid out for
    // this call's sizes (so the zeroing and scans scale with the input, not
    // with the limits); only the neighbor-search part is used
    tnet_ctx c;
    memset(&c, 0, sizeof c);
    c.d = tnet_model_desc{64, 8, 0, 1, cutoff, 0.f, 0};
    rc = build_layout(&c.d, n_atoms, n_systems, 0, &c.lay);
    if (rc) return rc;
    if (c.lay.rev > kNoAllocScratchBytes) return TNET_ERR_WORKSPACE;
    c.lay.slab_width = 0;  // two-pass search: no row slab in the static array
    c.max_atoms = n_atoms;
    c.max_systems = n_systems;
    c.max_pairs = cap;
    c.ws = (char *)scratch;
    c.ws_bytes = kNoAllocScratchBytes;
    return neighbors_impl(&c, n_atoms, n_systems, pos, batch, box, cutoff, row_ptr, col, cap, n_pairs_dev,
                          status_dev, (cudaStream_t)stream);
}
