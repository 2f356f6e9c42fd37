// Internal declarations shared by the CUDA translation units of libenzo_ppm.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "enzo_ppm.h"

namespace enzo {

constexpr int kSweepThreads = 128;     // default pencils per tile (one per thread)
// Pencils per CTA tile a sweep may use (the autotuner picks among these); the
// learned guess needs 128 (one tensor-core MMA row per pencil).
__host__ __device__ constexpr bool tile_supported(int t) { return t == 64 || t == 128 || t == 256; }
constexpr int kFillThreads = 256;      // stored cells per ghost-fill tile
constexpr int kCflCells = 4096;        // active cells per CFL tile
constexpr int kMaxN = 4096;            // per-axis active size limit

// Workspace layout (bytes from the 256-aligned start).
constexpr size_t kWsCounter = 0;       // uint32 dynamic tile counter
constexpr size_t kWsRateBits = 8;      // uint64: bits of the max CFL rate (double >= 0)
constexpr size_t kWsDt = 16;           // double: last dt computed on the device
constexpr size_t kWsPrefix = 256;      // int32 prefix[npatch + 1] of tiles per patch

// Per-thread counts of frequent events (32-bit, flushed once per thread);
// rare events are added to the caller's status words when they happen.
struct Counters {
    unsigned iters = 0, restarts = 0, guesses = 0;
    unsigned gep = 0;   // dual energy: zone loads that took the gas-energy pressure
    unsigned long long *st = nullptr;
#ifdef __CUDACC__
    __device__ __forceinline__ void rare(int word) const
    {
        if (st) atomicAdd(st + word, 1ull);
    }
#endif
};

// Method parameters after defaults are applied.
struct MethodParams {
    double gamma, rho_floor, p_floor, newton_tol;
    int newton_max, fallback, guess;
    const void *mlp;
    double mlp_gate;   // < 0: learned guess at every interface
    int solver;        // ENZO_SOLVER_*: interface flux
    int options;       // ENZO_OPT_* bits of the reconstruction
};

struct SweepArgs {
    const enzo_patch *patches;
    int npatch;
    int dir;
    int cover_mask;
    int64_t field_len;
    double *U[5];
    double dt;                 // used when dt_ptr == nullptr
    const double *dt_ptr;      // device dt (enzo_step)
    MethodParams mp;
    int tile = kSweepThreads;  // pencils per CTA tile (= threads per CTA)
    const int *prefix;         // [npatch + 1]
    unsigned *tile_counter;
    unsigned long long *status;
    // interface-state log (optional): every log_stride-th interface of a
    // pencil, by a hash of (pencil, position), writes its traced left/right
    // states (rho, u, p) x 2 as float32 into log[slot][6]
    float *log = nullptr;
    unsigned long long *log_count = nullptr;
    long long log_cap = 0;
    int log_stride = 0;
    double *freg = nullptr;    // flux registers (enzo_patch.freg_all / freg_bnd)
    double *ge = nullptr;      // gas energy of the dual-energy option, else nullptr
};

// Tiles of a sweep along dir for one patch: ceil(pencils / kSweepThreads).
__host__ __device__ inline void sweep_ranges(const enzo_patch &P, int dir, int cover_mask,
                                             int lo[3], int hi[3])
{
    const bool wrap = (P.flags & ENZO_PATCH_PERIODIC) != 0;
    for (int a = 0; a < 3; ++a) {
        const bool cov = !wrap && a != dir && ((cover_mask >> a) & 1);
        lo[a] = cov ? 0 : P.ng;
        hi[a] = cov ? P.n[a] + 2 * P.ng : P.ng + P.n[a];
    }
}

__host__ __device__ inline bool patch_ok(const enzo_patch &P, int64_t field_len)
{
    if (P.ng != 3) return false;
    for (int a = 0; a < 3; ++a) {
        if (P.n[a] < 1 || P.n[a] > kMaxN) return false;
        if (!(P.dx[a] > 0.0) || !(P.dx[a] < 1e300)) return false;
    }
    const int64_t vol = (int64_t)(P.n[0] + 6) * (P.n[1] + 6) * (P.n[2] + 6);
    return P.off >= 0 && P.off + vol <= field_len;
}

// Launch helpers implemented in the precision translation units.
cudaError_t launch_sweep_fp64(const SweepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_sweep_fp32(const SweepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_sweep_fp32_learned(const SweepArgs &a, cudaStream_t s);
int sweep_grid_fp64(int device);
int sweep_grid_fp32(int device);
// FP32 plain sweep with a chosen tile size (64, 128 or 256 pencils per CTA).
cudaError_t launch_sweep_fp32_tiled(const SweepArgs &a, cudaStream_t s);

// Checks and defaults of enzo_params shared by every sweep entry point
// (ENZO_OK or an ENZO_ERR_* code).
int resolve_params(const enzo_params *p, MethodParams &m);
// One sweep of batch b whose tile table and tile counter live at `scratch`
// (the workspace layout: kWsCounter, kWsPrefix).  The batch is checked except
// for its workspace; dt_dev, when set, replaces dt.
int sweep_with_scratch(const enzo_patch_batch *b, char *scratch, int dir, double dt, const double *dt_dev,
                       int cover, const MethodParams &m, int precision, int tile_pencils, float *log = nullptr,
                       unsigned long long *log_count = nullptr, long long log_cap = 0, int log_stride = 0);

struct CflArgs {
    const enzo_patch *patches;
    int npatch;
    int64_t field_len;
    const double *U[5];
    double gamma, rho_floor, p_floor;
    const int *prefix;
    unsigned long long *rate_bits;
    unsigned long long *status;
};
cudaError_t launch_cfl_fp64(const CflArgs &a, int grid, cudaStream_t s);
cudaError_t launch_cfl_fp32(const CflArgs &a, int grid, cudaStream_t s);

struct RiemannArgs {
    int64_t n;
    const void *rl, *ul, *pl, *rr, *ur, *pr, *pguess;
    void *pstar, *ustar, *rho, *u, *p;
    int32_t *iters;
    MethodParams mp;
};
cudaError_t launch_riemann_fp64(const RiemannArgs &a, cudaStream_t s);
cudaError_t launch_riemann_fp32(const RiemannArgs &a, cudaStream_t s);

void note_launch(unsigned n = 1);

// Work-list kinds of the tile prefix: sweep pencils, ghost-fill cells (whole
// stored block, non-periodic patches), active cells (kCflCells per tile), 8^3
// blocks of active cells, active cells of every patch (kFillThreads per tile;
// packing).
enum { kKindSweep = 0, kKindFill = 1, kKindCells = 2, kKindTiles8 = 3, kKindActive = 4 };
constexpr int kFlagTile = 8;            // flag kernel: 8^3 active cells per CTA

// Launch of the per-patch tile prefix kernel (kind: kKind*) on stream s.
void launch_tile_prefix(const enzo_patch *patches, int npatch, int64_t field_len, int kind, int dir,
                        int cover, int *prefix, unsigned *counter, unsigned long long *rate_bits,
                        unsigned long long *status, cudaStream_t s, int tile_pencils = kSweepThreads);

#ifdef __CUDACC__
// float <-> double conversions on the integer pipe.  On GB300 the FP64 pipe
// retires 2 thread-operations per clock per SM (1/64 of FP32) and F2F
// conversions run on it, so FP32 work converts with bit operations.
//
// d2f_rz: double -> float rounded toward zero (error below one FP32 ulp): the
// exponent is rebiased by 1023 - 127 = 896 in place and the top 23 mantissa
// bits follow through a funnel shift; values below the FP32 normal range
// flush to signed zero, values above it (and NaN) become signed infinity.
__device__ __forceinline__ float d2f_rz(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned ah = hi & 0x7fffffffu;
    const unsigned t = __funnelshift_l(lo, ah - 0x38000000u, 3);
    const unsigned r = ah < 0x38100000u ? 0u : (ah >= 0x47f00000u ? 0x7f800000u : t);
    return __uint_as_float(r | (hi & 0x80000000u));
}

// f2d_exact: float -> double, exact for normal floats, zero and infinity
// (denormals are flushed to zero by -ftz before they get here; NaN keeps its
// top payload bits).
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned a = b & 0x7fffffffu;
    const unsigned mag = (a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u);
    const unsigned hi = (a < 0x00800000u ? 0u : mag) | (b & 0x80000000u);
    const unsigned lo = a < 0x00800000u ? 0u : b << 29;
    return __hiloint2double((int)hi, (int)lo);
}
#endif

}  // namespace enzo
