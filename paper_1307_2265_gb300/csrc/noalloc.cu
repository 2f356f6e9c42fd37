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
//    stream capture.
//  * All calls share the one array, and it keeps the contents of the last
//    call.  The prefix kernel rewrites the tile table and zeroes the counter at
//    the start of every call.  Calls whose kernels overlap on the GPU (for
//    example on two streams) race on the array and must not be issued.
//  * No cudaMalloc, cudaFree or allocating library routine is called.
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
    if (!(p->gamma > 1.0) || !(p->gamma < 100.0)) return ENZO_ERR_ARG;
    if (p->precision != ENZO_FP64 && p->precision != ENZO_FP32) return ENZO_ERR_ARG;
    if (p->guess != ENZO_GUESS_PLAIN) return p->guess == ENZO_GUESS_MLP ? ENZO_ERR_UNSUPPORTED : ENZO_ERR_ARG;
    if (!(p->rho_floor > 0.0) || !(p->p_floor > 0.0)) return ENZO_ERR_ARG;
    if (p->precision == ENZO_FP32 && (p->rho_floor < 1e-37 || p->p_floor < 1e-37)) return ENZO_ERR_ARG;
    if (b->npatch == 0) return ENZO_OK;
    if (!b->patches || !b->status || b->field_len <= 0) return ENZO_ERR_ARG;
    for (int f = 0; f < 5; ++f)
        if (!b->U[f]) return ENZO_ERR_ARG;
    const bool f64 = p->precision == ENZO_FP64;
    MethodParams m;
    m.gamma = p->gamma;
    m.rho_floor = p->rho_floor;
    m.p_floor = p->p_floor;
    m.newton_tol = p->newton_tol > 0.0 ? p->newton_tol : (f64 ? 1e-14 : 1e-6);
    m.newton_max = p->newton_max > 0 ? p->newton_max : (f64 ? 20 : 12);
    if (m.newton_max > 200) return ENZO_ERR_ARG;
    if (p->fallback < 0 || p->fallback > 2) return ENZO_ERR_ARG;
    m.fallback = p->fallback;
    m.guess = p->guess;
    m.mlp = nullptr;
    m.mlp_gate = 0.0;
    if (p->solver != ENZO_SOLVER_TWOSHOCK && p->solver != ENZO_SOLVER_HLL && p->solver != ENZO_SOLVER_HLLC)
        return ENZO_ERR_ARG;
    m.solver = p->solver;
    if (p->options & ~(ENZO_OPT_STEEPEN | ENZO_OPT_FLATTEN | ENZO_OPT_DIFFUSE | ENZO_OPT_DUAL)) return ENZO_ERR_ARG;
    if ((p->options & ENZO_OPT_DUAL) && (p->solver != ENZO_SOLVER_TWOSHOCK || !b->ge)) return ENZO_ERR_ARG;
    m.options = p->options;

    void *scratch = nullptr;
    int r = noalloc_scratch(&scratch);
    if (r) return r;
    char *ws = static_cast<char *>(scratch);
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    launch_tile_prefix(b->patches, b->npatch, b->field_len, 0, dir, cover_mask,
                       reinterpret_cast<int *>(ws + kWsPrefix), reinterpret_cast<unsigned *>(ws + kWsCounter),
                       nullptr, b->status, s);
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    note_launch();

    SweepArgs a;
    a.patches = b->patches;
    a.npatch = b->npatch;
    a.dir = dir;
    a.cover_mask = cover_mask;
    a.field_len = b->field_len;
    for (int f = 0; f < 5; ++f) a.U[f] = b->U[f];
    a.dt = dt;
    a.dt_ptr = nullptr;
    a.mp = m;
    a.prefix = reinterpret_cast<const int *>(ws + kWsPrefix);
    a.tile_counter = reinterpret_cast<unsigned *>(ws + kWsCounter);
    a.status = b->status;
    a.ge = (m.options & ENZO_OPT_DUAL) ? b->ge : nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ENZO_ERR_CUDA;
    const cudaError_t e = f64 ? launch_sweep_fp64(a, sweep_grid_fp64(dev), s)
                              : launch_sweep_fp32(a, sweep_grid_fp32(dev), s);
    note_launch();
    return e == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}
