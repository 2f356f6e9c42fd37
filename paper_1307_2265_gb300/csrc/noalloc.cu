// Allocation-free variant of the sweep entry point.
//
// Some host codes cannot allocate device memory for this library.  An example
// is a simulation that owns every device buffer through its own pool and hands
// over only its field arrays.  Another is a caller whose memory budget is fixed
// once time stepping starts.  Such callers cannot provide the workspace that
// enzo_ppm_sweep asks for.  enzo_ppm_sweep_noalloc runs the same sweep kernel,
// but keeps the kernel's scratch in a fixed array of device memory that belongs
// to this library.  The scratch holds the per-patch tile prefix and the
// dynamic tile counter.
//
// Facts a caller must know (also stated in include/enzo_ppm.h):
//  * The array holds kNoAllocScratchBytes bytes.  That limits a batch to
//    kNoAllocMaxPatches patches; larger batches get ENZO_ERR_RANGE.
//  * Every GPU that loads the library keeps the array until the process exits.
//  * The first call on each device looks up the array's device address (with
//    that device current) and caches it.  Make that first call before any
//    stream capture.  The cached address belongs to the device's primary
//    context: do not keep using the library after cudaDeviceReset.
//  * All calls share the one array, and it keeps the contents of the last
//    call.  The prefix kernel rewrites the tile table and zeroes the counter at
//    the start of every call.  Calls whose kernels overlap on the GPU (for
//    example on two streams) race on the array and must not be issued.
//  * No cudaMalloc, cudaFree or allocating library routine is called.
//  * Everything else (argument checks, tile sizes, flux registers, the gas
//    energy) is exactly what enzo_ppm_sweep does with the same arguments.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "internal.cuh"

namespace enzo {

constexpr size_t kNoAllocScratchBytes = 128 * 1024;
constexpr int kNoAllocMaxPatches = 32000;
static_assert(kWsPrefix + sizeof(int) * (kNoAllocMaxPatches + 1) <= kNoAllocScratchBytes,
              "scratch array too small for the patch limit");

// The library-owned scratch.  In host code this name is only a host-side
// stand-in: kernels must be given the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
static int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ENZO_ERR_CUDA;
    if (dev < 0 || dev >= 64) return ENZO_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return ENZO_ERR_CUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return ENZO_OK;
}

}  // namespace enzo

using namespace enzo;

extern "C" int enzo_ppm_sweep_noalloc(const enzo_patch_batch *b, int32_t dir, double dt,
                                      int32_t cover_mask, const enzo_params *p)
{
    if (!b || !p) return ENZO_ERR_ARG;
    if (b->npatch < 0) return ENZO_ERR_ARG;
    if (b->npatch > kNoAllocMaxPatches) return ENZO_ERR_RANGE;
    if (dir < 0 || dir > 2 || !(dt >= 0.0) || !(dt < INFINITY) || cover_mask < 0 || cover_mask > 7)
        return ENZO_ERR_ARG;
    MethodParams m;
    int r = resolve_params(p, m);      // the checks and defaults of enzo_ppm_sweep
    if (r) return r;
    // the learned guess keeps its network state in memory the caller allocates
    if (m.guess == ENZO_GUESS_MLP) return ENZO_ERR_UNSUPPORTED;
    if (b->npatch == 0) return ENZO_OK;
    if (!b->patches || !b->status || b->field_len <= 0) return ENZO_ERR_ARG;
    for (int f = 0; f < 5; ++f)
        if (!b->U[f]) return ENZO_ERR_ARG;
    void *scratch = nullptr;
    r = noalloc_scratch(&scratch);
    if (r) return r;
    return sweep_with_scratch(b, static_cast<char *>(scratch), dir, dt, nullptr, cover_mask, m, p->precision,
                              p->tile[dir]);
}
