// Learned Newton starting guess for the two-shock p* (not in the paper; the
// Riemann solver of Sec. 4.1.2 still decides the answer).  MLP 6 -> 64 -> 64 -> 1 with
// SiLU, BF16 weights and activations, FP32 accumulation in tensor memory,
// predicting y = ln(p* / sqrt(p_L p_R)) from Riemann-invariant features.
//
// Kernels here (tcgen05.mma, operands staged in shared memory, accumulators in
// TMEM, completion on an mbarrier with bounded waits):
//   mlp_pack_kernel     FP32 master weights -> BF16 tensor-core tiles (blob)
//   mlp_forward_kernel  batched forward, 128 samples per MMA tile
//   mlp_train_kernel    forward + backward (weight gradients as MMAs over the
//                       batch), gradients summed into FP32 buffers
//   mlp_adam_kernel     Adam on the FP32 master weights
#include <cmath>
#include <cstdint>

#include "internal.cuh"
#include "mlp_layout.cuh"
#include "tc05.cuh"

namespace enzo {

using namespace tc;

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------
__global__ void mlp_pack_kernel(const float *__restrict__ m, unsigned char *__restrict__ blob)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // W1 as B operand of layer 1: rows n = hidden unit, k = input (6 used of 16)
    if (t < 64 * 16) {
        const int n = t / 16, k = t % 16;
        const float v = k < kMlpIn ? m[kMW1 + n * kMlpIn + k] : 0.0f;
        st_bf16(blob + kBlobW1, tile_off(n, k, 16), v);
    }
    if (t < 64 * 64) {
        const int n = t / 64, k = t % 64;
        st_bf16(blob + kBlobW2, tile_off(n, k, 64), m[kMW2 + n * 64 + k]);     // W2[out=n][in=k]
        st_bf16(blob + kBlobW2T, tile_off(n, k, 64), m[kMW2 + k * 64 + n]);    // W2^T: rows in, cols out
    }
    float *f = reinterpret_cast<float *>(blob + kBlobF32);
    if (t < 64) {
        f[t] = m[kMB1 + t];
        f[64 + t] = m[kMB2 + t];
        f[128 + t] = m[kMW3 + t];
    }
    if (t == 0) f[192] = m[kMB3];
}

// ---------------------------------------------------------------------------
// shared state of one CTA (128 threads, thread = sample row)
// ---------------------------------------------------------------------------
struct alignas(1024) FwdSmem {
    unsigned char w1[64 * 16 * 2];
    unsigned char w2[64 * 64 * 2];
    unsigned char a1[128 * 16 * 2];
    unsigned char a2[128 * 64 * 2];
    float bias[4 * 64 + 4];
    uint64_t mbar;
    uint32_t tmem;
    int error;
};

__device__ __forceinline__ void load_tile(unsigned char *dst, const unsigned char *src, int bytes)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// Layer 1 and layer 2 of one 128-row tile.  Rows write their bf16 input row into
// a1 first.  On return z2 (pre-activation of layer 2, bias included) for this
// thread's row is in z2[64].  Returns false if an mbarrier wait timed out.
__device__ __forceinline__ bool forward_tile(FwdSmem &S, uint32_t &phase, float z2out[64], uint32_t tcols1,
                                             uint32_t tcols2)
{
    const int row = threadIdx.x;
    const uint32_t lane_off = (uint32_t)((row & ~31) << 16);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after();
        mma_bf16(S.tmem + tcols1, smem_desc(smem_u32(S.a1), 128, 256), smem_desc(smem_u32(S.w1), 128, 256),
                 idesc_bf16_f32(128, 64), false);
        commit(&S.mbar);
    }
    if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) return false;
    phase ^= 1u;
    fence_after();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v[16];
        tmem_ld16(S.tmem + lane_off + tcols1 + c * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = c * 16 + i;
            st_bf16(S.a2, tile_off(row, j, 64), silu(v[i] + S.bias[j]));
        }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
            mma_bf16(S.tmem + tcols2, smem_desc(smem_u32(S.a2) + ks * 256, 128, 1024),
                     smem_desc(smem_u32(S.w2) + ks * 256, 128, 1024), idesc_bf16_f32(128, 64), ks > 0);
        commit(&S.mbar);
    }
    if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) return false;
    phase ^= 1u;
    fence_after();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v[16];
        tmem_ld16(S.tmem + lane_off + tcols2 + c * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) z2out[c * 16 + i] = v[i] + S.bias[64 + c * 16 + i];
    }
    return true;
}

__device__ __forceinline__ void write_a1_row(FwdSmem &S, const float x[kMlpIn])
{
    const int row = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 16; ++k) st_bf16(S.a1, tile_off(row, k, 16), k < kMlpIn ? x[k] : 0.0f);
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const unsigned char *__restrict__ blob,
                                                           const float *__restrict__ x, float *__restrict__ y,
                                                           int64_t n, unsigned long long *status)
{
    extern __shared__ unsigned char smem_raw[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    load_tile(S.w1, blob + kBlobW1, sizeof(S.w1));
    load_tile(S.w2, blob + kBlobW2, sizeof(S.w2));
    const float *f = reinterpret_cast<const float *>(blob + kBlobF32);
    for (int i = threadIdx.x; i < 193; i += blockDim.x) S.bias[i] = f[i];
    if (threadIdx.x == 0) {
        mbar_init(&S.mbar, 1);
        S.error = 0;
    }
    if (threadIdx.x < 32) tmem_alloc(&S.tmem, 128);
    fence_before();
    __syncthreads();
    fence_after();
    uint32_t phase = 0;
    const int64_t ntile = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r = tile * 128 + threadIdx.x;
        float xi[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) xi[k] = r < n ? x[r * kMlpIn + k] : 0.0f;
        write_a1_row(S, xi);
        float z2[64];
        if (!forward_tile(S, phase, z2, 0, 64)) {
            S.error = 1;   // every thread of the CTA sees the same result
            break;
        }
        float acc = S.bias[192];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc = fmaf(S.bias[128 + j], silu(z2[j]), acc);
        if (r < n) y[r] = acc;
        // the next tile rewrites a1/a2 and TMEM only after every row has read them
        fence_before();
        __syncthreads();
        fence_after();
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && S.error) atomicAdd(status + ENZO_ST_TIMEOUT, 1ull);
    if (threadIdx.x < 32) tmem_dealloc(S.tmem, 128);
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct alignas(1024) TrainSmem {
    FwdSmem f;
    unsigned char w2t[64 * 64 * 2];          // B of dH1 = dZ2 W2: rows in, cols out
    unsigned char ad2[128 * 64 * 2];         // A of dH1: rows sample, cols out (dZ2)
    unsigned char adw2[128 * 128 * 2];       // A of dW2: rows out (64 used), cols sample (dZ2^T)
    unsigned char bh1[64 * 128 * 2];         // B of dW2: rows in, cols sample (H1^T)
    unsigned char adw1[128 * 128 * 2];       // A of dW1: rows hidden (64 used), cols sample (dZ1^T)
    unsigned char bx[16 * 128 * 2];          // B of dW1: rows input (6 used), cols sample (X^T)
    float gsmall[4 * 64 + 4];                // (unused), db2, dw3, db3 partial sums
    float loss;
};

constexpr int kTZ1 = 0, kTZ2 = 64, kTDH1 = 128, kTDW2 = 192, kTDW1 = 256;

__global__ void __launch_bounds__(128) mlp_train_kernel(const unsigned char *__restrict__ blob,
                                                         const float *__restrict__ x,
                                                         const float *__restrict__ target, int64_t n,
                                                         float *__restrict__ grad, float *__restrict__ loss,
                                                         unsigned long long *status)
{
    extern __shared__ unsigned char smem_raw[];
    TrainSmem &T = *reinterpret_cast<TrainSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    FwdSmem &S = T.f;
    const int row = threadIdx.x;
    load_tile(S.w1, blob + kBlobW1, sizeof(S.w1));
    load_tile(S.w2, blob + kBlobW2, sizeof(S.w2));
    load_tile(T.w2t, blob + kBlobW2T, sizeof(T.w2t));
    const float *f = reinterpret_cast<const float *>(blob + kBlobF32);
    for (int i = row; i < 193; i += blockDim.x) S.bias[i] = f[i];
    for (int i = row; i < 4 * 64 + 4; i += blockDim.x) T.gsmall[i] = 0.0f;
    // rows 64..127 of the weight-gradient A tiles stay zero
    for (int i = row; i < (int)(sizeof(T.adw2) / 16); i += blockDim.x) {
        reinterpret_cast<uint4 *>(T.adw2)[i] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(T.adw1)[i] = make_uint4(0, 0, 0, 0);
    }
    if (row == 0) {
        mbar_init(&S.mbar, 1);
        S.error = 0;
        T.loss = 0.0f;
    }
    if (row < 32) tmem_alloc(&S.tmem, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t lane_off = (uint32_t)((row & ~31) << 16);
    const float inv_n = 1.0f / (float)n;
    uint32_t phase = 0;
    bool first = true;
    float lsum = 0.0f;
    const int64_t ntile = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r = tile * 128 + row;
        const bool valid = r < n;
        float xi[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) xi[k] = valid ? x[r * kMlpIn + k] : 0.0f;
        write_a1_row(S, xi);
        // X^T for dW1, with input column 6 held at 1 for valid rows: its column
        // of dW1 = dZ1^T X is then sum_r dz1[r][j], the gradient of b1
#pragma unroll
        for (int k = 0; k < 16; ++k)
            st_bf16(T.bx, tile_off(k, row, 128), k < kMlpIn ? xi[k] : (k == kMlpIn && valid ? 1.0f : 0.0f));
        // forward; keep H1^T for dW2
        float z2[64];
        {
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (row == 0) {
                fence_after();
                mma_bf16(S.tmem + kTZ1, smem_desc(smem_u32(S.a1), 128, 256), smem_desc(smem_u32(S.w1), 128, 256),
                         idesc_bf16_f32(128, 64), false);
                commit(&S.mbar);
            }
            if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) { S.error = 1; break; }
            phase ^= 1u;
            fence_after();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[16];
                tmem_ld16(S.tmem + lane_off + kTZ1 + c * 16, v);
                uint32_t pk[8];
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int j = c * 16 + i;
                    const float h0 = silu(v[i] + S.bias[j]), h1 = silu(v[i + 1] + S.bias[j + 1]);
                    const __nv_bfloat162 hp = __floats2bfloat162_rn(h0, h1);
                    pk[i / 2] = *reinterpret_cast<const uint32_t *>(&hp);
                    st_bf16(T.bh1, tile_off(j, row, 128), valid ? h0 : 0.0f);
                    st_bf16(T.bh1, tile_off(j + 1, row, 128), valid ? h1 : 0.0f);
                }
                *reinterpret_cast<uint4 *>(S.a2 + tile_off(row, c * 16, 64)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4 *>(S.a2 + tile_off(row, c * 16 + 8, 64)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (row == 0) {
                fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_bf16(S.tmem + kTZ2, smem_desc(smem_u32(S.a2) + ks * 256, 128, 1024),
                             smem_desc(smem_u32(S.w2) + ks * 256, 128, 1024), idesc_bf16_f32(128, 64), ks > 0);
                commit(&S.mbar);
            }
            if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) { S.error = 1; break; }
            phase ^= 1u;
            fence_after();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[16];
                tmem_ld16(S.tmem + lane_off + kTZ2 + c * 16, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) z2[c * 16 + i] = v[i] + S.bias[64 + c * 16 + i];
            }
        }
        // output, loss and dL/dz2
        float yv = S.bias[192];
#pragma unroll
        for (int j = 0; j < 64; ++j) yv = fmaf(S.bias[128 + j], silu(z2[j]), yv);
        const float e = valid ? yv - target[r] : 0.0f;
        lsum += e * e;
        const float dy = 2.0f * e * inv_n;
        // sums over the tile's rows (db3, dw3, db2): reduced across the warp with
        // shuffles, then one shared-memory add per warp (the 128 rows of a tile
        // adding into the same 64 words would serialise)
        const bool lead = (row & 31) == 0;
        const float sdy = warp_sum(dy);
        if (lead) atomicAdd(&T.gsmall[192], sdy);
#pragma unroll
        for (int j8 = 0; j8 < 64; j8 += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                float d[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = j8 + i + h;
                    const float h2 = silu(z2[j]);
                    d[h] = dy * S.bias[128 + j] * silu_grad(z2[j]);
                    const float s3 = warp_sum(dy * h2), s2 = warp_sum(d[h]);
                    if (lead) {
                        atomicAdd(&T.gsmall[128 + j], s3);      // dw3
                        atomicAdd(&T.gsmall[64 + j], s2);       // db2
                    }
                    st_bf16(T.adw2, tile_off(j, row, 128), d[h]);
                }
                const __nv_bfloat162 dp = __floats2bfloat162_rn(d[0], d[1]);
                pk[i / 2] = *reinterpret_cast<const uint32_t *>(&dp);
            }
            *reinterpret_cast<uint4 *>(T.ad2 + tile_off(row, j8, 64)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        // dH1 = dZ2 W2 and dW2 += dZ2^T H1
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (row == 0) {
            fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(S.tmem + kTDH1, smem_desc(smem_u32(T.ad2) + ks * 256, 128, 1024),
                         smem_desc(smem_u32(T.w2t) + ks * 256, 128, 1024), idesc_bf16_f32(128, 64), ks > 0);
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(S.tmem + kTDW2, smem_desc(smem_u32(T.adw2) + ks * 256, 128, 2048),
                         smem_desc(smem_u32(T.bh1) + ks * 256, 128, 2048), idesc_bf16_f32(128, 64),
                         !first || ks > 0);
            commit(&S.mbar);
        }
        if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) { S.error = 1; break; }
        phase ^= 1u;
        fence_after();
        // dz1 = dH1 * silu'(z1), z1 re-read from TMEM
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float dh[16], z1[16];
            tmem_ld16(S.tmem + lane_off + kTDH1 + c * 16, dh);
            tmem_ld16(S.tmem + lane_off + kTZ1 + c * 16, z1);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = c * 16 + i;
                const float dz1 = valid ? dh[i] * silu_grad(z1[i] + S.bias[j]) : 0.0f;
                st_bf16(T.adw1, tile_off(j, row, 128), dz1);   // db1 comes with dW1
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (row == 0) {
            fence_after();
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(S.tmem + kTDW1, smem_desc(smem_u32(T.adw1) + ks * 256, 128, 2048),
                         smem_desc(smem_u32(T.bx) + ks * 256, 128, 2048), idesc_bf16_f32(128, 16),
                         !first || ks > 0);
            commit(&S.mbar);
        }
        if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) { S.error = 1; break; }
        phase ^= 1u;
        fence_after();
        first = false;
    }
    // flush the accumulated weight gradients (rows 0..63 of the TMEM tiles)
    fence_before();
    __syncthreads();
    fence_after();
    if (!S.error && !first) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(S.tmem + lane_off + kTDW2 + c * 16, v);
            if (row < 64) {
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(&grad[kMW2 + row * 64 + c * 16 + i], v[i]);
            }
        }
        float v[16];
        tmem_ld16(S.tmem + lane_off + kTDW1, v);
        if (row < 64) {
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) atomicAdd(&grad[kMW1 + row * kMlpIn + k], v[k]);
            atomicAdd(&grad[kMB1 + row], v[kMlpIn]);    // the column of ones
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((row & 31) == 0) atomicAdd(&T.loss, lsum);
    fence_before();
    __syncthreads();
    if (!S.error) {
        if (row < 64) {
            atomicAdd(&grad[kMB2 + row], T.gsmall[64 + row]);
            atomicAdd(&grad[kMW3 + row], T.gsmall[128 + row]);
        }
        if (row == 0) {
            atomicAdd(&grad[kMB3], T.gsmall[192]);
            atomicAdd(loss, T.loss * inv_n);
        }
    }
    if (row == 0 && S.error) atomicAdd(status + ENZO_ST_TIMEOUT, 1ull);
    if (row < 32) tmem_dealloc(S.tmem, 512);
}

__global__ void mlp_adam_kernel(float *__restrict__ m, float *__restrict__ mo, float *__restrict__ vo,
                                const float *__restrict__ g, int step, float lr, float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float gi = g[i];
    const float mi = b1 * mo[i] + (1.0f - b1) * gi;
    const float vi = b2 * vo[i] + (1.0f - b2) * gi * gi;
    mo[i] = mi;
    vo[i] = vi;
    const float mhat = mi / (1.0f - powf(b1, (float)step));
    const float vhat = vi / (1.0f - powf(b2, (float)step));
    m[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

// Riemann-invariant features of left/right states (same definition as the guess
// inside the sweep): x[i][0..5].
__global__ void mlp_features_kernel(const float *rl, const float *ul, const float *pl, const float *rr,
                                    const float *ur, const float *pr, float gamma, float *x, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v[6];
    mlp_features(rl[i], ul[i], pl[i], rr[i], ur[i], pr[i], gamma, v);
#pragma unroll
    for (int k = 0; k < 6; ++k) x[i * 6 + k] = v[k];
}

static int sms()
{
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s > 0 ? s : 1;
}

}  // namespace enzo

using namespace enzo;

extern "C" {

int enzo_mlp_pack(const float *master, void *blob, void *stream)
{
    if (!master || !blob || (reinterpret_cast<uintptr_t>(blob) & 15u)) return ENZO_ERR_ARG;
    mlp_pack_kernel<<<(64 * 64 + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, static_cast<unsigned char *>(blob));
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_mlp_forward(const void *blob, const float *x, float *y, int64_t n, unsigned long long *status,
                     void *stream)
{
    if (!blob || n < 0 || !status) return ENZO_ERR_ARG;
    if (n == 0) return ENZO_OK;
    if (!x || !y) return ENZO_ERR_ARG;
    const size_t smem = sizeof(FwdSmem) + 1024;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return ENZO_ERR_CUDA;
        attr = true;
    }
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)(tiles < (int64_t)sms() * 4 ? tiles : (int64_t)sms() * 4);
    mlp_forward_kernel<<<grid, 128, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const unsigned char *>(blob), x, y, n, status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_mlp_features(const float *rl, const float *ul, const float *pl, const float *rr, const float *ur,
                      const float *pr, double gamma, float *x, int64_t n, void *stream)
{
    if (n < 0 || !(gamma > 1.0)) return ENZO_ERR_ARG;
    if (n == 0) return ENZO_OK;
    if (!rl || !ul || !pl || !rr || !ur || !pr || !x) return ENZO_ERR_ARG;
    mlp_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        rl, ul, pl, rr, ur, pr, (float)gamma, x, n);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_mlp_train_step(float *master, float *adam_m, float *adam_v, int32_t step, const float *x,
                        const float *target, int64_t n, float lr, float *grad, float *loss, void *blob,
                        unsigned long long *status, void *stream)
{
    if (!master || !blob || !grad || !loss || !status || n <= 0 || !x || !target) return ENZO_ERR_ARG;
    if (lr > 0.0f && (!adam_m || !adam_v || step < 1)) return ENZO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(TrainSmem) + 1024;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return ENZO_ERR_CUDA;
        attr = true;
    }
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess) return ENZO_ERR_CUDA;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return ENZO_ERR_CUDA;
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)(tiles < (int64_t)sms() ? tiles : (int64_t)sms());
    mlp_train_kernel<<<grid, 128, smem, s>>>(static_cast<const unsigned char *>(blob), x, target, n, grad, loss,
                                              status);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    if (lr > 0.0f) {
        mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(master, adam_m, adam_v, grad, step, lr, 0.9f,
                                                                 0.999f, 1e-8f);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
        return enzo_mlp_pack(master, blob, stream);
    }
    return ENZO_OK;
}

}  // extern "C"
