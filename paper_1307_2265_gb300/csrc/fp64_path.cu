// FP64 path: every step of the sweep, the CFL rule and the standalone Riemann
// solver in double precision.  Built with --fmad=false and IEEE division and
// square root so each operation rounds exactly once, in the written order.
#include "ppm_device.cuh"

namespace enzo {

cudaError_t launch_sweep_fp64(const SweepArgs &a, int grid, cudaStream_t s)
{
    return launch_sweep_dir<double>(a, grid, s);
}

int sweep_grid_fp64(int device) { return sweep_grid_for<double>(device); }

cudaError_t launch_cfl_fp64(const CflArgs &a, int grid, cudaStream_t s)
{
    cfl_kernel<double><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_riemann_fp64(const RiemannArgs &a, cudaStream_t s)
{
    const int64_t blocks = (a.n + 255) / 256;
    riemann_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enzo
