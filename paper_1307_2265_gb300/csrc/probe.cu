// Throughput probe of GB300's FP64 pipe, the denominator of the plain FP64
// sweep's ALU roofline.  Each thread runs kChains independent dependency chains
// of one FP64 operation for n steps, so the pipe, not latency, sets the rate:
//   ENZO_PROBE_DFMA  x = fma(x, a, b)     ENZO_PROBE_DADD  x = x + b
//   ENZO_PROBE_DMUL  x = x * a            ENZO_PROBE_DSQRT x = sqrt(x + b)
//   ENZO_PROBE_DDIV  x = a / (x + b)
// (a slightly below 1 and b small keep every chain finite and normal).  The
// chains' sum goes to sink so nothing is optimised away.  Built like the FP64
// path (--fmad=false, IEEE division and square root), so sqrt and division
// are the sequences that path executes.
#include "internal.cuh"

namespace enzo {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_fp64_kernel(int64_t n, double a, double b, double *sink)
{
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int64_t i = 0; i < n; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            if (OP == ENZO_PROBE_DFMA) x[c] = fma(x[c], a, b);
            else if (OP == ENZO_PROBE_DADD) x[c] = x[c] + b;
            else if (OP == ENZO_PROBE_DMUL) x[c] = x[c] * a;
            else if (OP == ENZO_PROBE_DSQRT) x[c] = sqrt(x[c] + b);
            else x[c] = a / (x[c] + b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.678) sink[blockIdx.x] = s;          // practically never: keeps the chains live
    if (threadIdx.x == 0 && blockIdx.x == 0) sink[gridDim.x] = s;
}

}  // namespace enzo

using namespace enzo;

extern "C" int enzo_probe_fp64(int32_t op, int64_t n, double *sink, int64_t *ops, void *stream)
{
    if (op < ENZO_PROBE_DFMA || op > ENZO_PROBE_DDIV || n < 1 || n > (int64_t)1 << 30 || !sink || !ops)
        return ENZO_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ENZO_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (sms > 0 ? sms : 1) * ENZO_PROBE_BLOCKS_PER_SM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double a = 0.9999999, b = 1e-7;
    switch (op) {
    case ENZO_PROBE_DFMA: probe_fp64_kernel<ENZO_PROBE_DFMA><<<grid, kProbeThreads, 0, s>>>(n, a, b, sink); break;
    case ENZO_PROBE_DADD: probe_fp64_kernel<ENZO_PROBE_DADD><<<grid, kProbeThreads, 0, s>>>(n, a, b, sink); break;
    case ENZO_PROBE_DMUL: probe_fp64_kernel<ENZO_PROBE_DMUL><<<grid, kProbeThreads, 0, s>>>(n, a, b, sink); break;
    case ENZO_PROBE_DSQRT: probe_fp64_kernel<ENZO_PROBE_DSQRT><<<grid, kProbeThreads, 0, s>>>(n, a, b, sink); break;
    default: probe_fp64_kernel<ENZO_PROBE_DDIV><<<grid, kProbeThreads, 0, s>>>(n, a, b, sink); break;
    }
    note_launch();
    *ops = (int64_t)grid * kProbeThreads * kProbeChains * n;
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}
