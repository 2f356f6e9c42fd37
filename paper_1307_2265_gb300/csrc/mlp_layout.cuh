// Parameter and weight-blob layout of the learned p* guess, shared by the MLP
// kernels and the sweep kernel that evaluates the guess.
#pragma once
#include <cstdint>

namespace enzo {

constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 64;
// FP32 master parameters, in this order: W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3
constexpr int kMW1 = 0;
constexpr int kMB1 = kMW1 + kMlpHidden * kMlpIn;
constexpr int kMW2 = kMB1 + kMlpHidden;
constexpr int kMB2 = kMW2 + kMlpHidden * kMlpHidden;
constexpr int kMW3 = kMB2 + kMlpHidden;
constexpr int kMB3 = kMW3 + kMlpHidden;
constexpr int kMlpParams = kMB3 + 1;   // 4673
// Device blob: BF16 tensor-core tiles (K-major, no swizzle) and FP32 vectors.
constexpr int kBlobW1 = 0;                     // 64 x 16 (inputs padded to 16)
constexpr int kBlobW2 = kBlobW1 + 64 * 16 * 2;  // 64 x 64, rows = output unit
constexpr int kBlobW2T = kBlobW2 + 64 * 64 * 2; // 64 x 64, rows = input unit
constexpr int kBlobF32 = kBlobW2T + 64 * 64 * 2; // b1[64], b2[64], w3[64], b3
constexpr int kBlobBytes = kBlobF32 + 4 * 256;

// Features of a Riemann problem (scale- and Galilean-invariant):
// (ln rho_L/rho_ref, (u_L-u_bar)/c_ref, ln p_L/p_ref, and the same for R),
// rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R), c_ref = sqrt(gamma p_ref/rho_ref).
__host__ __device__ inline void mlp_features(float rl, float ul, float pl, float rr, float ur, float pr,
                                             float gamma, float x[6])
{
    const float a = 0.5f * logf(rl / rr);
    const float b = 0.5f * logf(pl / pr);
    const float cref = sqrtf(gamma * sqrtf(pl * pr) / sqrtf(rl * rr));
    const float du = 0.5f * (ul - ur) / cref;
    x[0] = a;
    x[1] = du;
    x[2] = b;
    x[3] = -a;
    x[4] = -du;
    x[5] = -b;
}

}  // namespace enzo
