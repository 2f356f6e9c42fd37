// C ABI of libenzo_ppm: argument checks, work-list construction on the device,
// ghost fill, CFL reduction and the launches of the sweep kernels.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.cuh"

namespace enzo {

static std::atomic<unsigned long long> g_launches{0};
void note_launch(unsigned n) { g_launches += n; }


__device__ __forceinline__ int tiles_of(const enzo_patch &P, int64_t field_len, int kind, int dir,
                                        int cover, int tile_pencils, bool &bad)
{
    if (!patch_ok(P, field_len)) {
        bad = true;
        return 0;
    }
    if (kind == kKindSweep) {
        int lo[3], hi[3];
        sweep_ranges(P, dir, cover, lo, hi);
        const int a1 = dir == 0 ? 1 : 0, a2 = dir == 2 ? 1 : 2;
        const int64_t pen = (int64_t)(hi[a1] - lo[a1]) * (hi[a2] - lo[a2]);
        return (int)((pen + tile_pencils - 1) / tile_pencils);
    }
    if (kind == kKindFill) {
        if (P.flags & ENZO_PATCH_PERIODIC) return 0;
        const int64_t vol = (int64_t)(P.n[0] + 2 * P.ng) * (P.n[1] + 2 * P.ng) * (P.n[2] + 2 * P.ng);
        return (int)((vol + kFillThreads - 1) / kFillThreads);
    }
    if (kind == kKindActive) {
        const int64_t cells = (int64_t)P.n[0] * P.n[1] * P.n[2];
        return (int)((cells + kFillThreads - 1) / kFillThreads);
    }
    if (kind == kKindTiles8) {
        const int64_t t0 = (P.n[0] + kFlagTile - 1) / kFlagTile, t1 = (P.n[1] + kFlagTile - 1) / kFlagTile,
                      t2 = (P.n[2] + kFlagTile - 1) / kFlagTile;
        return (int)(t0 * t1 * t2);
    }
    const int64_t cells = (int64_t)P.n[0] * P.n[1] * P.n[2];
    return (int)((cells + kCflCells - 1) / kCflCells);
}

// Exclusive prefix of tiles per patch (one block), reset of the tile counter
// and of the CFL accumulator.
__global__ void __launch_bounds__(1024) prefix_kernel(const enzo_patch *patches, int npatch,
                                                      int64_t field_len, int kind, int dir, int cover,
                                                      int tile_pencils, int *prefix, unsigned *counter,
                                                      unsigned long long *rate_bits,
                                                      unsigned long long *status)
{
    __shared__ int s_sum[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (npatch + T - 1) / T;
    const int beg = min(t * per, npatch), end = min(beg + per, npatch);
    int sum = 0;
    bool bad = false;
    unsigned nbad = 0;
    for (int i = beg; i < end; ++i) {
        bool b = false;
        sum += tiles_of(patches[i], field_len, kind, dir, cover, tile_pencils, b);
        nbad += b;
    }
    s_sum[t] = sum;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        const int v = t >= off ? s_sum[t - off] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    int run = s_sum[t] - sum;
    for (int i = beg; i < end; ++i) {
        prefix[i] = run;
        run += tiles_of(patches[i], field_len, kind, dir, cover, tile_pencils, bad);
    }
    if (t == T - 1) {
        prefix[npatch] = s_sum[T - 1];
        *counter = 0u;
        if (rate_bits) *rate_bits = 0ull;
    }
    unsigned long long v = nbad;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0 && v) atomicAdd(status + ENZO_ST_BAD_PATCH, v);
}

// Periodic self ghost fill (Sec. 3.1, case 4): every ghost cell copies the
// active cell it wraps onto, edges and corners included.
__global__ void __launch_bounds__(kFillThreads) ghost_fill_kernel(const enzo_patch *patches, int npatch,
                                                                  double *U0, double *U1, double *U2,
                                                                  double *U3, double *U4, double *ge,
                                                                  const int *prefix)
{
    const int total = prefix[npatch];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lo = 0, hi = npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = patches[lo];
        const int N0 = P.n[0] + 2 * P.ng, N1 = P.n[1] + 2 * P.ng, N2 = P.n[2] + 2 * P.ng;
        const int64_t cell = (int64_t)(tile - prefix[lo]) * kFillThreads + threadIdx.x;
        if (cell >= (int64_t)N0 * N1 * N2) continue;
        const int a[3] = {(int)(cell % N0), (int)((cell / N0) % N1), (int)(cell / ((int64_t)N0 * N1))};
        bool ghost = false;
        int src[3];
        for (int d = 0; d < 3; ++d) {
            int x = a[d] - P.ng;
            if (x < 0 || x >= P.n[d]) ghost = true;
            x %= P.n[d];
            if (x < 0) x += P.n[d];
            src[d] = x + P.ng;
        }
        if (!ghost) continue;
        const int64_t dst = P.off + cell;
        const int64_t s = P.off + src[0] + (int64_t)N0 * (src[1] + (int64_t)N1 * src[2]);
        U0[dst] = U0[s];
        U1[dst] = U1[s];
        U2[dst] = U2[s];
        U3[dst] = U3[s];
        U4[dst] = U4[s];
        if (ge) ge[dst] = ge[s];
    }
}

// External boundaries of each patch taken as a single grid (Sec. 3.1):
// per axis periodic (wrap), reflecting (mirror about the face, momentum along
// the axis negated) or outflow (boundary cell copied).  The three per-axis maps
// compose, so one pass gives what filling x, then y, then z over the full
// extents gives: edges and corners take every condition that applies.
__device__ __forceinline__ int bc_map(int x, int n, int bc, bool &flip)
{
    if (x >= 0 && x < n) return x;
    if (bc == ENZO_BC_PERIODIC) return ((x % n) + n) % n;
    if (bc == ENZO_BC_OUTFLOW) return x < 0 ? 0 : n - 1;
    // reflecting; for n < 3 the mirror is folded back into the patch
    flip = true;
    int m = ((x % (2 * n)) + 2 * n) % (2 * n);
    return m < n ? m : 2 * n - 1 - m;
}

__global__ void __launch_bounds__(kFillThreads) boundary_fill_kernel(const enzo_patch *patches, int npatch,
                                                                     double *U0, double *U1, double *U2,
                                                                     double *U3, double *U4, double *ge,
                                                                     const int *prefix, int bcx, int bcy, int bcz)
{
    double *const U[5] = {U0, U1, U2, U3, U4};
    const int bc[3] = {bcx, bcy, bcz};
    const int total = prefix[npatch];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lo = 0, hi = npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = patches[lo];
        const int N0 = P.n[0] + 2 * P.ng, N1 = P.n[1] + 2 * P.ng, N2 = P.n[2] + 2 * P.ng;
        const int64_t cell = (int64_t)(tile - prefix[lo]) * kFillThreads + threadIdx.x;
        if (cell >= (int64_t)N0 * N1 * N2) continue;
        const int a[3] = {(int)(cell % N0), (int)((cell / N0) % N1), (int)(cell / ((int64_t)N0 * N1))};
        bool ghost = false, flip[3] = {false, false, false};
        int src[3];
        for (int d = 0; d < 3; ++d) {
            const int x = a[d] - P.ng;
            if (x < 0 || x >= P.n[d]) ghost = true;
            src[d] = bc_map(x, P.n[d], bc[d], flip[d]) + P.ng;
        }
        if (!ghost) continue;
        const int64_t dst = P.off + cell;
        const int64_t s = P.off + src[0] + (int64_t)N0 * (src[1] + (int64_t)N1 * src[2]);
        U[0][dst] = U[0][s];
        U[4][dst] = U[4][s];
        if (ge) ge[dst] = ge[s];
        for (int d = 0; d < 3; ++d) U[1 + d][dst] = flip[d] ? -U[1 + d][s] : U[1 + d][s];
    }
}

__global__ void dt_finalize_kernel(const unsigned long long *rate_bits, double cfl, double *ws_dt,
                                   double *dt_out)
{
    const double r = __longlong_as_double((long long)*rate_bits);
    const double dt = cfl / r;
    *ws_dt = dt;
    if (dt_out) *dt_out = dt;
}

int resolve_params(const enzo_params *p, MethodParams &m)
{
    if (!p) return ENZO_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->gamma < 100.0)) return ENZO_ERR_ARG;
    if (p->precision != ENZO_FP64 && p->precision != ENZO_FP32) return ENZO_ERR_ARG;
    if (p->guess != ENZO_GUESS_PLAIN && p->guess != ENZO_GUESS_MLP) return ENZO_ERR_ARG;
    if (p->guess == ENZO_GUESS_MLP && (!p->mlp || (reinterpret_cast<uintptr_t>(p->mlp) & 15u))) return ENZO_ERR_ARG;
    if (!(p->rho_floor > 0.0) || !(p->p_floor > 0.0)) return ENZO_ERR_ARG;
    if (p->precision == ENZO_FP32 && (p->rho_floor < 1e-37 || p->p_floor < 1e-37)) return ENZO_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (p->tile[d] != 0 && !tile_supported(p->tile[d])) return ENZO_ERR_ARG;
    const bool f64 = p->precision == ENZO_FP64;
    m.gamma = p->gamma;
    m.rho_floor = p->rho_floor;
    m.p_floor = p->p_floor;
    m.newton_tol = p->newton_tol > 0.0 ? p->newton_tol : (f64 ? 1e-14 : 1e-6);
    m.newton_max = p->newton_max > 0 ? p->newton_max : (f64 ? 20 : 12);
    if (m.newton_max > 200) return ENZO_ERR_ARG;
    if (p->fallback < 0 || p->fallback > 2) return ENZO_ERR_ARG;
    if (p->fallback == 2 && p->guess == ENZO_GUESS_MLP) return ENZO_ERR_ARG;
    m.fallback = p->fallback;
    m.guess = p->guess;
    m.mlp = p->mlp;
    if (p->mlp_gate != p->mlp_gate) return ENZO_ERR_ARG;
    m.mlp_gate = p->mlp_gate == 0.0 ? 0.03 : p->mlp_gate;
    if (p->solver != ENZO_SOLVER_TWOSHOCK && p->solver != ENZO_SOLVER_HLL && p->solver != ENZO_SOLVER_HLLC)
        return ENZO_ERR_ARG;
    if (p->guess == ENZO_GUESS_MLP && p->solver != ENZO_SOLVER_TWOSHOCK) return ENZO_ERR_ARG;
    m.solver = p->solver;
    if (p->options & ~(ENZO_OPT_STEEPEN | ENZO_OPT_FLATTEN | ENZO_OPT_DIFFUSE | ENZO_OPT_DUAL)) return ENZO_ERR_ARG;
    if (p->guess == ENZO_GUESS_MLP && p->options) return ENZO_ERR_ARG;
    if ((p->options & ENZO_OPT_DUAL) && p->solver != ENZO_SOLVER_TWOSHOCK) return ENZO_ERR_ARG;
    m.options = p->options;
    return ENZO_OK;
}

static int check_batch(const enzo_patch_batch *b)
{
    if (!b) return ENZO_ERR_ARG;
    if (b->npatch < 0) return ENZO_ERR_ARG;
    if (b->npatch == 0) return ENZO_OK;
    if (!b->patches || !b->status || b->field_len <= 0) return ENZO_ERR_ARG;
    for (int f = 0; f < 5; ++f)
        if (!b->U[f]) return ENZO_ERR_ARG;
    if (!b->workspace || (reinterpret_cast<uintptr_t>(b->workspace) & 15u)) return ENZO_ERR_WORKSPACE;
    if (b->ws_bytes < enzo_workspace_size(b->npatch)) return ENZO_ERR_WORKSPACE;
    return ENZO_OK;
}

static char *ws(const enzo_patch_batch *b) { return static_cast<char *>(b->workspace); }

void launch_tile_prefix(const enzo_patch *patches, int npatch, int64_t field_len, int kind, int dir,
                        int cover, int *prefix, unsigned *counter, unsigned long long *rate_bits,
                        unsigned long long *status, cudaStream_t s, int tile_pencils)
{
    prefix_kernel<<<1, 1024, 0, s>>>(patches, npatch, field_len, kind, dir, cover, tile_pencils, prefix,
                                     counter, rate_bits, status);
}

static int launch_prefix(const enzo_patch_batch *b, int kind, int dir, int cover, bool reset_rate,
                         cudaStream_t s, int tile_pencils = kSweepThreads)
{
    prefix_kernel<<<1, 1024, 0, s>>>(b->patches, b->npatch, b->field_len, kind, dir, cover, tile_pencils,
                                     reinterpret_cast<int *>(ws(b) + kWsPrefix),
                                     reinterpret_cast<unsigned *>(ws(b) + kWsCounter),
                                     reset_rate ? reinterpret_cast<unsigned long long *>(ws(b) + kWsRateBits)
                                                : nullptr,
                                     b->status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int sweep_with_scratch(const enzo_patch_batch *b, char *scratch, int dir, double dt, const double *dt_dev,
                       int cover, const MethodParams &m, int precision, int tile_pencils, float *log,
                       unsigned long long *log_count, long long log_cap, int log_stride)
{
    if ((m.options & ENZO_OPT_DUAL) && !b->ge) return ENZO_ERR_ARG;
    // flux registers of a batch with a gas-energy field hold six components
    // per face, which only the dual-energy sweep writes
    if (b->freg && b->ge && !(m.options & ENZO_OPT_DUAL)) return ENZO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    int tile = tile_pencils > 0 ? tile_pencils : kSweepThreads;
    if (precision == ENZO_FP64 || m.guess == ENZO_GUESS_MLP || b->freg || m.options || m.fallback == 2)
        tile = kSweepThreads;
    launch_tile_prefix(b->patches, b->npatch, b->field_len, kKindSweep, dir, cover,
                       reinterpret_cast<int *>(scratch + kWsPrefix), reinterpret_cast<unsigned *>(scratch + kWsCounter),
                       nullptr, b->status, s, tile);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    SweepArgs a;
    a.tile = tile;
    a.patches = b->patches;
    a.npatch = b->npatch;
    a.dir = dir;
    a.cover_mask = cover;
    a.field_len = b->field_len;
    for (int f = 0; f < 5; ++f) a.U[f] = b->U[f];
    a.dt = dt;
    a.dt_ptr = dt_dev;
    a.mp = m;
    a.prefix = reinterpret_cast<const int *>(scratch + kWsPrefix);
    a.tile_counter = reinterpret_cast<unsigned *>(scratch + kWsCounter);
    a.status = b->status;
    a.freg = b->freg;
    a.ge = (m.options & ENZO_OPT_DUAL) ? b->ge : nullptr;
    a.log = log;
    a.log_count = log_count;
    a.log_cap = log_cap;
    a.log_stride = log_stride;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e;
    if (precision == ENZO_FP64) e = launch_sweep_fp64(a, sweep_grid_fp64(dev), s);
    else if (m.guess == ENZO_GUESS_MLP) e = launch_sweep_fp32_learned(a, s);
    else if (tile != kSweepThreads) e = launch_sweep_fp32_tiled(a, s);
    else e = launch_sweep_fp32(a, sweep_grid_fp32(dev), s);
    note_launch();
    return e == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

static int sweep_impl(const enzo_patch_batch *b, int dir, double dt, const double *dt_dev,
                      int cover, const MethodParams &m, int precision, int tile_pencils, float *log = nullptr,
                      unsigned long long *log_count = nullptr, long long log_cap = 0, int log_stride = 0)
{
    return sweep_with_scratch(b, ws(b), dir, dt, dt_dev, cover, m, precision, tile_pencils, log, log_count,
                              log_cap, log_stride);
}

static int fill_impl(const enzo_patch_batch *b)
{
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    int r = launch_prefix(b, kKindFill, 0, 0, false, s);
    if (r) return r;
    ghost_fill_kernel<<<device_sms() * 8, kFillThreads, 0, s>>>(
        b->patches, b->npatch, b->U[0], b->U[1], b->U[2], b->U[3], b->U[4], b->ge,
        reinterpret_cast<const int *>(ws(b) + kWsPrefix));
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

static bool bc_ok(const int32_t *bc)
{
    if (!bc) return false;
    for (int d = 0; d < 3; ++d)
        if (bc[d] != ENZO_BC_PERIODIC && bc[d] != ENZO_BC_REFLECT && bc[d] != ENZO_BC_OUTFLOW) return false;
    return true;
}

static int boundary_impl(const enzo_patch_batch *b, const int32_t *bc)
{
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    int r = launch_prefix(b, kKindFill, 0, 0, false, s);
    if (r) return r;
    boundary_fill_kernel<<<device_sms() * 8, kFillThreads, 0, s>>>(
        b->patches, b->npatch, b->U[0], b->U[1], b->U[2], b->U[3], b->U[4], b->ge,
        reinterpret_cast<const int *>(ws(b) + kWsPrefix), bc[0], bc[1], bc[2]);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

// Active cells of every patch to (PACK) or from a packed layout: patch p's
// active cells, x fastest, then y, then z, start at act_off[p] of each packed
// array.  Each thread takes one active cell of every patch (periodic ones
// too), consecutive threads consecutive packed cells, so rows stay contiguous
// on both sides; the cell's coordinates come from 32-bit divisions (64-bit
// only for patches of more than 2^31 cells).
struct PackArgs {
    double *U[6];             // the batch's fields (U[5]: ge, or nullptr)
    double *packed[6];        // the packed arrays (packed[5]: ge, or nullptr)
    const int64_t *act_off;
    int nf;                   // 5, or 6 with the gas energy
};

template <bool PACK>
__global__ void __launch_bounds__(kFillThreads) pack_kernel(const enzo_patch *patches, int npatch,
                                                            const __grid_constant__ PackArgs a, const int *prefix)
{
    const int total = prefix[npatch];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lo = 0, hi = npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = patches[lo];
        const int64_t ncell = (int64_t)P.n[0] * P.n[1] * P.n[2];
        const int64_t c = (int64_t)(tile - prefix[lo]) * kFillThreads + threadIdx.x;
        if (c >= ncell) continue;
        int x, y, z;
        if (ncell <= 0x7fffffff) {
            const unsigned cc = (unsigned)c, t = cc / (unsigned)P.n[0];
            x = (int)(cc - t * (unsigned)P.n[0]);
            z = (int)(t / (unsigned)P.n[1]);
            y = (int)(t - (unsigned)z * (unsigned)P.n[1]);
        } else {
            const int64_t t = c / P.n[0];
            x = (int)(c - t * P.n[0]);
            z = (int)(t / P.n[1]);
            y = (int)(t - (int64_t)z * P.n[1]);
        }
        const int N0 = P.n[0] + 2 * P.ng, N1 = P.n[1] + 2 * P.ng;
        const int64_t q = a.act_off[lo] + c;
        const int64_t u = P.off + (x + P.ng) + (int64_t)N0 * ((y + P.ng) + (int64_t)N1 * (z + P.ng));
        if (PACK) {
            // gather: every field's load first, then the contiguous stores (the
            // compiler cannot tell the arrays apart and would otherwise wait out
            // one load per field): 3.33 -> 3.12 ms on the 4000-patch level
            double v[6];
#pragma unroll
            for (int f = 0; f < 6; ++f)
                if (f < a.nf) v[f] = __ldg(a.U[f] + u);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (f >= a.nf) break;
                a.packed[f][q] = v[f];
            }
        } else {
            // scatter: load and store field by field (batching the loads here
            // measured slower, 3.75 -> 4.42 ms)
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (f >= a.nf) break;
                a.U[f][u] = a.packed[f][q];
            }
        }
    }
}

static int pack_impl(const enzo_patch_batch *b, double *const packed[5], double *packed_ge, const int64_t *act_off,
                     bool pack)
{
    int r = check_batch(b);
    if (r) return r;
    if (!packed || !act_off || (packed_ge && !b->ge)) return ENZO_ERR_ARG;
    for (int f = 0; f < 5; ++f)
        if (!packed[f]) return ENZO_ERR_ARG;
    if (b->npatch == 0) return ENZO_OK;
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    r = launch_prefix(b, kKindActive, 0, 0, false, s);
    if (r) return r;
    PackArgs a;
    for (int f = 0; f < 5; ++f) {
        a.U[f] = b->U[f];
        a.packed[f] = packed[f];
    }
    a.U[5] = packed_ge ? b->ge : nullptr;
    a.packed[5] = packed_ge;
    a.nf = packed_ge ? 6 : 5;
    a.act_off = act_off;
    const int *prefix = reinterpret_cast<const int *>(ws(b) + kWsPrefix);
    if (pack) pack_kernel<true><<<device_sms() * 8, kFillThreads, 0, s>>>(b->patches, b->npatch, a, prefix);
    else pack_kernel<false><<<device_sms() * 8, kFillThreads, 0, s>>>(b->patches, b->npatch, a, prefix);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

}  // namespace enzo

using namespace enzo;

extern "C" {

size_t enzo_workspace_size(int32_t npatch)
{
    if (npatch < 0) npatch = 0;
    const size_t bytes = kWsPrefix + sizeof(int) * ((size_t)npatch + 1);
    return (bytes + 255) & ~(size_t)255;
}

int enzo_validate_patches(const enzo_patch *hp, int32_t npatch, int64_t field_len, int32_t *bad_index)
{
    if (bad_index) *bad_index = -1;
    if (npatch < 0 || (npatch > 0 && !hp)) return ENZO_ERR_ARG;
    for (int32_t i = 0; i < npatch; ++i) {
        if (!patch_ok(hp[i], field_len)) {
            if (bad_index) *bad_index = i;
            return ENZO_ERR_RANGE;
        }
    }
    return ENZO_OK;
}

int enzo_ppm_sweep(const enzo_patch_batch *b, int32_t dir, double dt, int32_t cover_mask,
                   const enzo_params *p)
{
    int r = check_batch(b);
    if (r) return r;
    MethodParams m;
    r = resolve_params(p, m);
    if (r) return r;
    if (dir < 0 || dir > 2 || !(dt >= 0.0) || !std::isfinite(dt) || cover_mask < 0 || cover_mask > 7)
        return ENZO_ERR_ARG;
    if (m.guess == ENZO_GUESS_MLP && p->precision != ENZO_FP32) return ENZO_ERR_UNSUPPORTED;
    if (b->npatch == 0) return ENZO_OK;
    return sweep_impl(b, dir, dt, nullptr, cover_mask, m, p->precision, p->tile[dir]);
}

int enzo_ppm_sweep_dev(const enzo_patch_batch *b, int32_t dir, const double *dt_dev, int32_t cover_mask,
                       const enzo_params *p)
{
    int r = check_batch(b);
    if (r) return r;
    MethodParams m;
    r = resolve_params(p, m);
    if (r) return r;
    if (dir < 0 || dir > 2 || !dt_dev || cover_mask < 0 || cover_mask > 7) return ENZO_ERR_ARG;
    if (m.guess == ENZO_GUESS_MLP && p->precision != ENZO_FP32) return ENZO_ERR_UNSUPPORTED;
    if (b->npatch == 0) return ENZO_OK;
    return sweep_impl(b, dir, 0.0, dt_dev, cover_mask, m, p->precision, p->tile[dir]);
}

int enzo_ppm_sweep_logged(const enzo_patch_batch *b, int32_t dir, double dt, int32_t cover_mask,
                          const enzo_params *p, float *log, unsigned long long *log_count, int64_t log_cap,
                          int32_t log_stride)
{
    int r = check_batch(b);
    if (r) return r;
    MethodParams m;
    r = resolve_params(p, m);
    if (r) return r;
    if (dir < 0 || dir > 2 || !(dt >= 0.0) || !std::isfinite(dt) || cover_mask < 0 || cover_mask > 7)
        return ENZO_ERR_ARG;
    if (!log || !log_count || log_cap < 0 || log_stride < 1) return ENZO_ERR_ARG;
    if (m.guess == ENZO_GUESS_MLP && p->precision != ENZO_FP32) return ENZO_ERR_UNSUPPORTED;
    if (b->npatch == 0) return ENZO_OK;
    return sweep_impl(b, dir, dt, nullptr, cover_mask, m, p->precision, p->tile[dir], log, log_count, log_cap,
                      log_stride);
}

int enzo_ghost_fill_periodic(const enzo_patch_batch *b)
{
    int r = check_batch(b);
    if (r) return r;
    if (b->npatch == 0) return ENZO_OK;
    return fill_impl(b);
}

int enzo_pack_active(const enzo_patch_batch *b, double *const packed[5], double *packed_ge, const int64_t *act_off)
{
    return pack_impl(b, packed, packed_ge, act_off, true);
}

int enzo_unpack_active(const enzo_patch_batch *b, double *const packed[5], double *packed_ge,
                       const int64_t *act_off)
{
    return pack_impl(b, packed, packed_ge, act_off, false);
}

int enzo_ghost_fill_boundary(const enzo_patch_batch *b, const int32_t bc[3])
{
    int r = check_batch(b);
    if (r) return r;
    if (!bc_ok(bc)) return ENZO_ERR_ARG;
    if (b->npatch == 0) return ENZO_OK;
    return boundary_impl(b, bc);
}

int enzo_timestep_cfl(const enzo_patch_batch *b, const enzo_params *p, double *dt_out,
                      int32_t dt_out_on_device)
{
    int r = check_batch(b);
    if (r) return r;
    MethodParams m;
    r = resolve_params(p, m);
    if (r) return r;
    if (!dt_out || !(p->cfl > 0.0) || !(p->cfl <= 1.0)) return ENZO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    if (b->npatch == 0) {
        if (dt_out_on_device) return ENZO_ERR_ARG;
        *dt_out = INFINITY;
        return ENZO_OK;
    }
    r = launch_prefix(b, kKindCells, 0, 0, true, s);
    if (r) return r;
    CflArgs a;
    a.patches = b->patches;
    a.npatch = b->npatch;
    a.field_len = b->field_len;
    for (int f = 0; f < 5; ++f) a.U[f] = b->U[f];
    a.gamma = m.gamma;
    a.rho_floor = m.rho_floor;
    a.p_floor = m.p_floor;
    a.prefix = reinterpret_cast<const int *>(ws(b) + kWsPrefix);
    a.rate_bits = reinterpret_cast<unsigned long long *>(ws(b) + kWsRateBits);
    a.status = b->status;
    const int grid = device_sms() * 8;
    cudaError_t e = p->precision == ENZO_FP64 ? launch_cfl_fp64(a, grid, s) : launch_cfl_fp32(a, grid, s);
    note_launch();
    if (e != cudaSuccess) return ENZO_ERR_CUDA;
    dt_finalize_kernel<<<1, 1, 0, s>>>(a.rate_bits, p->cfl, reinterpret_cast<double *>(ws(b) + kWsDt),
                                       dt_out_on_device ? dt_out : nullptr);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    if (!dt_out_on_device) {
        if (cudaMemcpyAsync(dt_out, ws(b) + kWsDt, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return ENZO_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return ENZO_ERR_CUDA;
    }
    return ENZO_OK;
}

static int step_impl(const enzo_patch_batch *b, const enzo_params *p, int32_t step_index, const double *dt_dev,
                     const int32_t *bc)
{
    int r = check_batch(b);
    if (r) return r;
    MethodParams m;
    r = resolve_params(p, m);
    if (r) return r;
    if (!dt_dev || step_index < 0) return ENZO_ERR_ARG;
    if (bc && !bc_ok(bc)) return ENZO_ERR_ARG;
    if (m.guess == ENZO_GUESS_MLP && p->precision != ENZO_FP32) return ENZO_ERR_UNSUPPORTED;
    if (b->npatch == 0) return ENZO_OK;
    if ((m.options & ENZO_OPT_DUAL) && !b->ge) return ENZO_ERR_ARG;
    if (b->freg && b->ge && !(m.options & ENZO_OPT_DUAL)) return ENZO_ERR_ARG;
    r = bc ? boundary_impl(b, bc) : fill_impl(b);
    if (r) return r;
    const int order[2][3] = {{0, 1, 2}, {2, 1, 0}};
    int done = 0;
    for (int q = 0; q < 3; ++q) {
        const int d = order[step_index & 1][q];
        const int cover = 7 & ~done & ~(1 << d);
        r = sweep_impl(b, d, 0.0, dt_dev, cover, m, p->precision, p->tile[d]);
        if (r) return r;
        done |= 1 << d;
    }
    return ENZO_OK;
}

int enzo_step(const enzo_patch_batch *b, const enzo_params *p, int32_t step_index, const double *dt_dev)
{
    return step_impl(b, p, step_index, dt_dev, nullptr);
}

int enzo_step_boundary(const enzo_patch_batch *b, const enzo_params *p, int32_t step_index,
                       const double *dt_dev, const int32_t bc[3])
{
    if (!bc) return ENZO_ERR_ARG;
    return step_impl(b, p, step_index, dt_dev, bc);
}

int enzo_riemann_solve(const enzo_riemann_states *st, const enzo_params *p)
{
    if (!st) return ENZO_ERR_ARG;
    MethodParams m;
    int r = resolve_params(p, m);
    if (r) return r;
    if (st->n < 0) return ENZO_ERR_ARG;
    if (st->n == 0) return ENZO_OK;
    if (!st->rhoL || !st->uL || !st->pL || !st->rhoR || !st->uR || !st->pR) return ENZO_ERR_ARG;
    if (st->n > ((int64_t)1 << 40)) return ENZO_ERR_ARG;
    RiemannArgs a;
    a.n = st->n;
    a.rl = st->rhoL; a.ul = st->uL; a.pl = st->pL;
    a.rr = st->rhoR; a.ur = st->uR; a.pr = st->pR;
    a.pguess = st->pguess;
    a.pstar = st->pstar; a.ustar = st->ustar;
    a.rho = st->rho_face; a.u = st->u_face; a.p = st->p_face;
    a.iters = st->iters;
    a.mp = m;
    cudaStream_t s = static_cast<cudaStream_t>(st->stream);
    cudaError_t e = p->precision == ENZO_FP64 ? launch_riemann_fp64(a, s) : launch_riemann_fp32(a, s);
    note_launch();
    return e == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

const char *enzo_strerror(int code)
{
    switch (code) {
    case ENZO_OK: return "ok";
    case ENZO_ERR_ARG: return "invalid argument";
    case ENZO_ERR_CUDA: return "CUDA error";
    case ENZO_ERR_RANGE: return "patch descriptor out of range, or batch larger than a fixed limit";
    case ENZO_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case ENZO_ERR_UNSUPPORTED: return "option not supported by this library";
    default: return "unknown error";
    }
}

unsigned long long enzo_launch_count(void) { return g_launches.load(); }

}  // extern "C"
