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
