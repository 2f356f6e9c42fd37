// FP32 path: reconstruction, tracing and the Riemann solve in single precision
// (fast reciprocal and square root), conserved variables accumulated in FP64
// and E - KE recovered in FP64 in high-Mach cells.
#include "ppm_device.cuh"

namespace enzo {

cudaError_t launch_sweep_fp32(const SweepArgs &a, int grid, cudaStream_t s)
{
    return launch_sweep_dir<float>(a, grid, s);
}

int sweep_grid_fp32(int device) { return sweep_grid_for<float>(device); }

// Sweep with the learned Newton guess (tensor cores inside the sweep).  TMEM
// holds 128 columns per CTA, so at most 4 CTAs share an SM.
template <int DIR, bool REG>
static cudaError_t launch_learned_dir(const SweepArgs &a, cudaStream_t s)
{
    static int grid[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const size_t smem = learned_smem_bytes<DIR>();
    if (!grid[dev]) {
        cudaError_t e = cudaFuncSetAttribute(ppm_sweep_kernel<float, DIR, true, kSweepThreads, REG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // ENZO_LEARNED_CTAS CTAs per SM: the launch bounds cap registers for
        // that many and TMEM holds 4 x 128 columns.  (A CTA that cannot be
        // resident yet only starts later and finds fewer tiles, since tiles
        // come from a counter.)
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid[dev] = (sms > 0 ? sms : 1) * ENZO_LEARNED_CTAS;
    }
    ppm_sweep_kernel<float, DIR, true, kSweepThreads, REG><<<grid[dev], kSweepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_fp32_tiled(const SweepArgs &a, cudaStream_t s)
{
    switch (a.tile) {
    case 64: return launch_tiled<float, 64>(a, s);
    case 256: return launch_tiled<float, 256>(a, s);
    default: return launch_tiled<float, 128>(a, s);
    }
}

cudaError_t launch_sweep_fp32_learned(const SweepArgs &a, cudaStream_t s)
{
    if (a.freg) {
        switch (a.dir) {
        case 0: return launch_learned_dir<0, true>(a, s);
        case 1: return launch_learned_dir<1, true>(a, s);
        default: return launch_learned_dir<2, true>(a, s);
        }
    }
    switch (a.dir) {
    case 0: return launch_learned_dir<0, false>(a, s);
    case 1: return launch_learned_dir<1, false>(a, s);
    default: return launch_learned_dir<2, false>(a, s);
    }
}

cudaError_t launch_cfl_fp32(const CflArgs &a, int grid, cudaStream_t s)
{
    cfl_kernel<float><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_riemann_fp32(const RiemannArgs &a, cudaStream_t s)
{
    const int64_t blocks = (a.n + 255) / 256;
    riemann_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enzo
