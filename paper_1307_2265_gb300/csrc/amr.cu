// Hierarchy rebuild (paper Sec. 3.5, 3.6): cell flagging on the GPU and the
// clustering of flagged cells into new grids on the host.
//   * flag_kernel_fp64: the slope, shock and baryon-mass criteria of Sec. 3.6
//     per active cell, each ratio formed in FP64 as the paper writes it;
//   * flag_kernel: the same criteria from FP32 primitives staged once per 8^3
//     block, compared without division (the fast path of FP32 hierarchies);
//     this unit is built with --fmad=false and IEEE division, so each
//     operation rounds once in the order written and both kernels' flags are
//     exact functions of the fields;
//   * enzo_cluster_flags: Berger & Rigoutsos as Sec. 3.5 describes it, host
//     C++ over one grid's flags.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace enzo {

struct FlagArgs {
    const enzo_patch *patches;
    int npatch;
    const double *U[5];
    const int *prefix;
    uint8_t *flags;
    const int64_t *flag_off;
    float g1, s2, dp, ef;      // gamma - 1, 2 slope, shock_dp, shock_e (rounded to FP32)
    bool slope, shock;
    double mass;
    double g1d, sl, dpd, efd;  // the same thresholds in FP64 (flag_kernel_fp64)
};

// Primitive values of the cell at storage index idx (Sec. 2.1) in FP64, in the
// order the criteria's reference forms them: KE = 0.5 |m|^2 / rho, e = E - KE,
// p = (gamma - 1) e, u_ax = m_ax / rho.
struct Prim64 {
    double rho, E, e, p;
};

__device__ __forceinline__ Prim64 prim64(const FlagArgs &a, int64_t idx)
{
    Prim64 q;
    q.rho = a.U[0][idx];
    q.E = a.U[4][idx];
    const double m0 = a.U[1][idx], m1 = a.U[2][idx], m2 = a.U[3][idx];
    const double ke = 0.5 * ((m0 * m0 + m1 * m1) + m2 * m2) / q.rho;
    q.e = q.E - ke;
    q.p = a.g1d * q.e;
    return q;
}

// FP64 flags, one thread per active cell of an 8^3 block (the tile list of
// flag_kernel): slope |q_{i+1} - q_{i-1}| / (2 |q_i|) > slope for q = rho, E;
// shock |p_{i+1} - p_{i-1}| / min(p_{i+1}, p_{i-1}) > shock_dp with
// u_{i-1} - u_{i+1} > 0 and e_i / E_i > shock_e; mass rho dx^3 > mass.
// Neighbours come from the ghost zones, or wrap for periodic-flagged patches.
__global__ void __launch_bounds__(256) flag_kernel_fp64(const __grid_constant__ FlagArgs a)
{
    const int total = a.prefix[a.npatch];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lo = 0, hi = a.npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = a.patches[lo];
        const int n[3] = {P.n[0], P.n[1], P.n[2]};
        const int nt0 = (n[0] + kFlagTile - 1) / kFlagTile, nt1 = (n[1] + kFlagTile - 1) / kFlagTile;
        const int t = tile - a.prefix[lo];
        const int b0[3] = {(t % nt0) * kFlagTile, ((t / nt0) % nt1) * kFlagTile, (t / (nt0 * nt1)) * kFlagTile};
        const int64_t N0 = n[0] + 2 * P.ng, N1 = n[1] + 2 * P.ng;
        const bool wrap = (P.flags & ENZO_PATCH_PERIODIC) != 0;
        const double vol = P.dx[0] * P.dx[0] * P.dx[0];
        for (int c = threadIdx.x; c < kFlagTile * kFlagTile * kFlagTile; c += blockDim.x) {
            const int g[3] = {b0[0] + c % kFlagTile, b0[1] + (c / kFlagTile) % kFlagTile,
                              b0[2] + c / (kFlagTile * kFlagTile)};
            if (g[0] >= n[0] || g[1] >= n[1] || g[2] >= n[2]) continue;
            auto at = [&](int d, int s) {
                int h[3] = {g[0], g[1], g[2]};
                h[d] += s;
                if (wrap) h[d] = h[d] < 0 ? h[d] + n[d] : (h[d] >= n[d] ? h[d] - n[d] : h[d]);
                return P.off + (h[0] + P.ng) + N0 * ((h[1] + P.ng) + N1 * (int64_t)(h[2] + P.ng));
            };
            const int64_t i0 = at(0, 0);
            const Prim64 q0 = prim64(a, i0);
            uint8_t f = 0;
            for (int ax = 0; ax < 3; ++ax) {
                const int64_t im = at(ax, -1), ip = at(ax, 1);
                if (a.slope) {
                    const double rm = a.U[0][im], rp = a.U[0][ip], Em = a.U[4][im], Ep = a.U[4][ip];
                    if (fabs(rp - rm) / (2.0 * fabs(q0.rho)) > a.sl) f |= ENZO_FLAG_SLOPE;
                    if (fabs(Ep - Em) / (2.0 * fabs(q0.E)) > a.sl) f |= ENZO_FLAG_SLOPE;
                }
                if (a.shock) {
                    const Prim64 qm = prim64(a, im), qp = prim64(a, ip);
                    const double pmin = qm.p < qp.p ? qm.p : qp.p;
                    const double um = a.U[1 + ax][im] / qm.rho, up = a.U[1 + ax][ip] / qp.rho;
                    if (fabs(qp.p - qm.p) / pmin > a.dpd && um - up > 0.0 && q0.e / q0.E > a.efd)
                        f |= ENZO_FLAG_SHOCK;
                }
            }
            if (a.mass > 0.0 && q0.rho * vol > a.mass) f |= ENZO_FLAG_MASS;
            a.flags[a.flag_off[lo] + g[0] + (int64_t)n[0] * (g[1] + (int64_t)n[1] * g[2])] = f;
        }
    }
}

constexpr int kHalo = kFlagTile + 2;                 // staged block edge
constexpr int kStage = kHalo * kHalo * kHalo;        // staged cells per CTA

// One CTA per 8^3 block of active cells.  The block and its one-cell halo
// (ghost cells, or periodic images for ENZO_PATCH_PERIODIC patches) are staged
// in shared memory as FP32 primitives once: the conserved FP64 values are
// rounded toward zero to FP32 on the integer pipe, then 1/rho, KE = (|m|^2 / 2)
// (1/rho), e = E - KE, p = (gamma - 1) e and u = m (1/rho) follow in FP32 (each
// operation rounded once: this unit is built with --fmad=false and IEEE
// division).  The criteria then
// compare in FP32 without division: |q_{i+1} - q_{i-1}| > 2 slope |q_i| for
// q = rho, E; |p_{i+1} - p_{i-1}| > shock_dp min(p_{i+1}, p_{i-1}) with
// u_{i-1} - u_{i+1} > 0 and e_i > shock_e E_i.  The baryon mass test stays in
// FP64 (rho dx^3 > mass).
__global__ void __launch_bounds__(256) flag_kernel(const __grid_constant__ FlagArgs a)
{
    __shared__ float sr[kStage], sE[kStage], se[kStage], sp[kStage], su[3][kStage];
    const int total = a.prefix[a.npatch];
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lo = 0, hi = a.npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = a.patches[lo];
        const int n[3] = {P.n[0], P.n[1], P.n[2]};
        const int nt0 = (n[0] + kFlagTile - 1) / kFlagTile, nt1 = (n[1] + kFlagTile - 1) / kFlagTile;
        const int t = tile - a.prefix[lo];
        const int b0[3] = {(t % nt0) * kFlagTile, ((t / nt0) % nt1) * kFlagTile, (t / (nt0 * nt1)) * kFlagTile};
        const int64_t N0 = n[0] + 2 * P.ng, N1 = n[1] + 2 * P.ng;
        const bool wrap = (P.flags & ENZO_PATCH_PERIODIC) != 0;
        __syncthreads();                              // the previous tile's reads are done
        for (int c = threadIdx.x; c < kStage; c += blockDim.x) {
            const int h[3] = {c % kHalo, (c / kHalo) % kHalo, c / (kHalo * kHalo)};
            int g[3];
            bool need = true;
            for (int d = 0; d < 3; ++d) {
                g[d] = b0[d] + h[d] - 1;              // active index, -1 .. n
                if (g[d] > n[d]) need = false;        // past the block's last needed neighbour
                if (wrap) g[d] = g[d] < 0 ? g[d] + n[d] : (g[d] >= n[d] ? g[d] - n[d] : g[d]);
            }
            if (!need) continue;
            const int64_t idx = P.off + (g[0] + P.ng) + N0 * ((g[1] + P.ng) + N1 * (int64_t)(g[2] + P.ng));
            const float r = d2f_rz(a.U[0][idx]), m0 = d2f_rz(a.U[1][idx]), m1 = d2f_rz(a.U[2][idx]),
                        m2 = d2f_rz(a.U[3][idx]), E = d2f_rz(a.U[4][idx]);
            const float inv = 1.0f / r;
            const float ke = (0.5f * ((m0 * m0 + m1 * m1) + m2 * m2)) * inv;
            const float e = E - ke;
            sr[c] = r;
            sE[c] = E;
            se[c] = e;
            sp[c] = a.g1 * e;
            su[0][c] = m0 * inv;
            su[1][c] = m1 * inv;
            su[2][c] = m2 * inv;
        }
        __syncthreads();
        const double vol = P.dx[0] * P.dx[0] * P.dx[0];
        for (int c = threadIdx.x; c < kFlagTile * kFlagTile * kFlagTile; c += blockDim.x) {
            const int q[3] = {c % kFlagTile, (c / kFlagTile) % kFlagTile, c / (kFlagTile * kFlagTile)};
            const int g[3] = {b0[0] + q[0], b0[1] + q[1], b0[2] + q[2]};
            if (g[0] >= n[0] || g[1] >= n[1] || g[2] >= n[2]) continue;
            const int k0 = (q[0] + 1) + kHalo * ((q[1] + 1) + kHalo * (q[2] + 1));
            const int step[3] = {1, kHalo, kHalo * kHalo};
            uint8_t f = 0;
            for (int ax = 0; ax < 3; ++ax) {
                const int km = k0 - step[ax], kp = k0 + step[ax];
                if (a.slope) {
                    if (fabsf(sr[kp] - sr[km]) > a.s2 * fabsf(sr[k0])) f |= ENZO_FLAG_SLOPE;
                    if (fabsf(sE[kp] - sE[km]) > a.s2 * fabsf(sE[k0])) f |= ENZO_FLAG_SLOPE;
                }
                if (a.shock) {
                    const float pm = sp[km], pp = sp[kp];
                    const float pmin = pm < pp ? pm : pp;
                    if (fabsf(pp - pm) > a.dp * pmin && su[ax][km] - su[ax][kp] > 0.0f && se[k0] > a.ef * sE[k0])
                        f |= ENZO_FLAG_SHOCK;
                }
            }
            if (a.mass > 0.0) {
                const int64_t idx = P.off + (g[0] + P.ng) + N0 * ((g[1] + P.ng) + N1 * (int64_t)(g[2] + P.ng));
                if (a.U[0][idx] * vol > a.mass) f |= ENZO_FLAG_MASS;
            }
            a.flags[a.flag_off[lo] + g[0] + (int64_t)n[0] * (g[1] + (int64_t)n[1] * g[2])] = f;
        }
    }
}

static int sms()
{
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s > 0 ? s : 1;
}

// ---- clustering (host) ------------------------------------------------------

struct Region {
    int lo[3], hi[3];
};

class Clusterer {
public:
    Clusterer(const uint8_t *flags, const int32_t n[3], const enzo_cluster_params &cp)
        : nx_(n[0]), ny_(n[1]), nz_(n[2]), cp_(cp)
    {
        // the flags' bounding box, eight flags at a time over empty stretches;
        // everything after works inside it grown by the buffer (cells
        // elsewhere are never flagged)
        int lo[3] = {nx_, ny_, nz_}, hi[3] = {-1, -1, -1};
        for (int z = 0; z < nz_; ++z)
            for (int y = 0; y < ny_; ++y) {
                const uint8_t *row = flags + ((size_t)z * ny_ + y) * nx_;
                int first = -1, last = -1, x = 0;
                for (; x + 8 <= nx_; x += 8) {
                    uint64_t w;
                    memcpy(&w, row + x, 8);
                    if (!w) continue;
                    for (int i = 0; i < 8; ++i)
                        if (row[x + i]) {
                            if (first < 0) first = x + i;
                            last = x + i;
                        }
                }
                for (; x < nx_; ++x)
                    if (row[x]) {
                        if (first < 0) first = x;
                        last = x;
                    }
                if (first < 0) continue;
                if (first < lo[0]) lo[0] = first;
                if (last > hi[0]) hi[0] = last;
                if (y < lo[1]) lo[1] = y;
                if (y > hi[1]) hi[1] = y;
                if (z < lo[2]) lo[2] = z;
                if (z > hi[2]) hi[2] = z;
            }
        if (hi[0] < 0) {
            for (int d = 0; d < 3; ++d) box_.lo[d] = box_.hi[d] = bd_[d] = 0;
            return;
        }
        const int ext[3] = {nx_, ny_, nz_};
        for (int d = 0; d < 3; ++d) {
            box_.lo[d] = lo[d] - cp.buffer < 0 ? 0 : lo[d] - cp.buffer;
            box_.hi[d] = hi[d] + 1 + cp.buffer > ext[d] ? ext[d] : hi[d] + 1 + cp.buffer;
            bd_[d] = box_.hi[d] - box_.lo[d];
        }
        F_.assign((size_t)bd_[0] * bd_[1] * bd_[2], 0);
        for (int z = box_.lo[2]; z < box_.hi[2]; ++z)
            for (int y = box_.lo[1]; y < box_.hi[1]; ++y) {
                const uint8_t *row = flags + ((size_t)z * ny_ + y) * nx_;
                char *dst = row_of(y, z);
                for (int x = box_.lo[0]; x < box_.hi[0]; ++x) dst[x - box_.lo[0]] = row[x] != 0;
            }
        grow();
        const int k = cp.margin;
        if (k > 0)
            for (int z = box_.lo[2]; z < box_.hi[2]; ++z)
                for (int y = box_.lo[1]; y < box_.hi[1]; ++y) {
                    char *row = row_of(y, z);
                    for (int x = box_.lo[0]; x < box_.hi[0]; ++x)
                        if (x < k || x >= nx_ - k || y < k || y >= ny_ - k || z < k || z >= nz_ - k)
                            row[x - box_.lo[0]] = 0;
                }
    }

    void run(std::vector<Region> &out)
    {
        // depth first, the low part before the high part: a stack popped from
        // the back with the high part pushed first
        std::vector<Region> stack;
        if (box_.hi[0] > box_.lo[0]) stack.push_back(box_);
        while (!stack.empty()) {
            Region r = stack.back();
            stack.pop_back();
            long long cnt = 0;
            if (!scan(r, cnt)) continue;           // r is now the bounding box of its flags
            const long long vol = (long long)(r.hi[0] - r.lo[0]) * (r.hi[1] - r.lo[1]) * (r.hi[2] - r.lo[2]);
            if ((double)cnt >= cp_.efficiency * (double)vol || vol <= cp_.small_cells) {
                out.push_back(r);
                continue;
            }
            int ext[3], axes[3] = {0, 1, 2};
            for (int d = 0; d < 3; ++d) ext[d] = r.hi[d] - r.lo[d];
            // longest first, ties in axis order
            for (int i = 0; i < 3; ++i)
                for (int j = i + 1; j < 3; ++j)
                    if (ext[axes[j]] > ext[axes[i]] || (ext[axes[j]] == ext[axes[i]] && axes[j] < axes[i])) {
                        const int t = axes[i];
                        axes[i] = axes[j];
                        axes[j] = t;
                    }
            int cut_ax = -1, cut = 0;
            for (int k = 0; k < 3 && cut_ax < 0; ++k) {
                const int c = best_cut(axes[k]);
                if (c > 0) {
                    cut_ax = axes[k];
                    cut = c;
                }
            }
            if (cut_ax < 0) {
                cut_ax = axes[0];
                if (ext[cut_ax] < 2) {
                    out.push_back(r);
                    continue;
                }
                cut = ext[cut_ax] / 2;
            }
            Region low = r, high = r;
            low.hi[cut_ax] = r.lo[cut_ax] + cut;
            high.lo[cut_ax] = r.lo[cut_ax] + cut;
            stack.push_back(high);
            stack.push_back(low);
        }
    }

private:
    // Flags of the row (y, z) of the bounding box, indexed by x - box_.lo[0].
    char *row_of(int y, int z) { return &F_[((size_t)(z - box_.lo[2]) * bd_[1] + (y - box_.lo[1])) * bd_[0]]; }
    const char *row_of(int y, int z) const
    {
        return &F_[((size_t)(z - box_.lo[2]) * bd_[1] + (y - box_.lo[1])) * bd_[0]];
    }

    // Chebyshev growth by cp_.buffer cells: separable, x then y then z, one
    // cell per pass, inside box_ (which holds every cell the growth reaches).
    void grow()
    {
        const int *e = bd_;
        for (int ax = 0; ax < 3; ++ax)
            for (int it = 0; it < cp_.buffer; ++it) {
                const std::vector<char> G(F_);
                for (int z = 0; z < e[2]; ++z)
                    for (int y = 0; y < e[1]; ++y)
                        for (int x = 0; x < e[0]; ++x) {
                            if (!G[((size_t)z * e[1] + y) * e[0] + x]) continue;
                            const int c[3] = {x, y, z};
                            for (int s = -1; s <= 1; s += 2) {
                                int q[3] = {c[0], c[1], c[2]};
                                q[ax] += s;
                                if (q[ax] < 0 || q[ax] >= e[ax]) continue;
                                F_[((size_t)q[2] * e[1] + q[1]) * e[0] + q[0]] = 1;
                            }
                        }
            }
    }

    // One pass over region r: the count of its flags, their bounding box (r
    // shrinks to it) and the signature along each axis over that box; false
    // when r holds no flag.
    bool scan(Region &r, long long &cnt)
    {
        int lo[3] = {r.hi[0], r.hi[1], r.hi[2]}, hi[3] = {r.lo[0] - 1, r.lo[1] - 1, r.lo[2] - 1};
        for (int d = 0; d < 3; ++d) sig_[d].assign(r.hi[d] - r.lo[d], 0);
        cnt = 0;
        for (int z = r.lo[2]; z < r.hi[2]; ++z)
            for (int y = r.lo[1]; y < r.hi[1]; ++y) {
                const char *row = row_of(y, z);
                for (int x = r.lo[0]; x < r.hi[0]; ++x) {
                    if (!row[x - box_.lo[0]]) continue;
                    ++cnt;
                    sig_[0][x - r.lo[0]] += 1;
                    sig_[1][y - r.lo[1]] += 1;
                    sig_[2][z - r.lo[2]] += 1;
                    const int c[3] = {x, y, z};
                    for (int d = 0; d < 3; ++d) {
                        if (c[d] < lo[d]) lo[d] = c[d];
                        if (c[d] > hi[d]) hi[d] = c[d];
                    }
                }
            }
        if (cnt == 0) return false;
        for (int d = 0; d < 3; ++d) {
            // keep the signature entries inside the bounding box
            sig_[d].erase(sig_[d].begin() + (hi[d] + 1 - r.lo[d]), sig_[d].end());
            sig_[d].erase(sig_[d].begin(), sig_[d].begin() + (lo[d] - r.lo[d]));
            r.lo[d] = lo[d];
            r.hi[d] = hi[d] + 1;
        }
        return true;
    }

    // Cut position (cells in the low part) at the strongest inflection of the
    // signature along ax (from the last scan), or 0 when there is none.
    int best_cut(int ax) const
    {
        const std::vector<long long> &sig = sig_[ax];
        const int n = (int)sig.size();
        if (n < 4) return 0;
        // second difference D[j] at signature index j + 1
        std::vector<long long> D(n - 2);
        for (int j = 0; j < n - 2; ++j) D[j] = sig[j] - 2 * sig[j + 1] + sig[j + 2];
        long long best_s = -1;
        int best_dist = 0, best_c = 0;
        for (int j = 0; j + 1 < n - 2; ++j) {
            if (!((D[j] < 0 && D[j + 1] > 0) || (D[j] > 0 && D[j + 1] < 0))) continue;
            const long long strength = llabs(D[j + 1] - D[j]);
            const int c = j + 2;
            const int dist = abs(2 * c - n);
            if (strength > best_s || (strength == best_s && (dist < best_dist || (dist == best_dist && c < best_c)))) {
                best_s = strength;
                best_dist = dist;
                best_c = c;
            }
        }
        return best_c;
    }

    std::vector<long long> sig_[3];
    Region box_;       // the flags' bounding box grown by the buffer
    int bd_[3];        // its extents
    int nx_, ny_, nz_;
    enzo_cluster_params cp_;
    std::vector<char> F_;
};

}  // namespace enzo

using namespace enzo;

extern "C" {

int enzo_flag_cells(const enzo_patch_batch *b, const enzo_flag_params *fp, uint8_t *flags, const int64_t *flag_off)
{
    if (!b || !fp || b->npatch < 0) return ENZO_ERR_ARG;
    if (b->npatch == 0) return ENZO_OK;
    if (!b->patches || !b->status || !flags || !flag_off || !b->workspace) return ENZO_ERR_ARG;
    for (int f = 0; f < 5; ++f)
        if (!b->U[f]) return ENZO_ERR_ARG;
    if (b->ws_bytes < enzo_workspace_size(b->npatch)) return ENZO_ERR_WORKSPACE;
    if (!(fp->gamma > 1.0)) return ENZO_ERR_ARG;
    if (fp->precision != ENZO_FP64 && fp->precision != ENZO_FP32) return ENZO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    char *ws = static_cast<char *>(b->workspace);
    launch_tile_prefix(b->patches, b->npatch, b->field_len, kKindTiles8, 0, 0,
                       reinterpret_cast<int *>(ws + kWsPrefix), reinterpret_cast<unsigned *>(ws + kWsCounter),
                       nullptr, b->status, s);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    FlagArgs a;
    a.patches = b->patches;
    a.npatch = b->npatch;
    for (int f = 0; f < 5; ++f) a.U[f] = b->U[f];
    a.prefix = reinterpret_cast<const int *>(ws + kWsPrefix);
    a.flags = flags;
    a.flag_off = flag_off;
    a.g1 = (float)(fp->gamma - 1.0);
    a.s2 = (float)(2.0 * fp->slope);
    a.dp = (float)fp->shock_dp;
    a.ef = (float)fp->shock_e;
    a.slope = fp->slope > 0.0;
    a.shock = fp->shock_dp > 0.0;
    a.mass = fp->mass;
    a.g1d = fp->gamma - 1.0;
    a.sl = fp->slope;
    a.dpd = fp->shock_dp;
    a.efd = fp->shock_e;
    if (fp->precision == ENZO_FP64) flag_kernel_fp64<<<sms() * 6, 256, 0, s>>>(a);
    else flag_kernel<<<sms() * 6, 256, 0, s>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_cluster_flags(const uint8_t *flags, const int32_t n[3], const enzo_cluster_params *cp, enzo_box *boxes,
                       int32_t cap, int32_t *nbox)
{
    if (!flags || !n || !cp || !nbox || cap < 0 || (cap > 0 && !boxes)) return ENZO_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (n[d] < 1 || n[d] > 4096) return ENZO_ERR_ARG;
    if (cp->small_cells < 1 || cp->buffer < 0 || cp->margin < 0 || !(cp->efficiency >= 0.0) || !(cp->efficiency <= 1.0))
        return ENZO_ERR_ARG;
    std::vector<Region> out;
    Clusterer(flags, n, *cp).run(out);
    *nbox = (int32_t)out.size();
    if ((int64_t)out.size() > cap) return ENZO_ERR_RANGE;
    for (size_t i = 0; i < out.size(); ++i)
        for (int d = 0; d < 3; ++d) {
            boxes[i].lo[d] = out[i].lo[d];
            boxes[i].hi[d] = out[i].hi[d];
        }
    return ENZO_OK;
}

}  // extern "C"
