// Hierarchy rebuild (paper Sec. 3.5, 3.6): cell flagging on the GPU and the
// clustering of flagged cells into new grids on the host.
//   * flag_kernel: the slope, shock and baryon-mass criteria of Sec. 3.6 per
//     active cell, in FP64 (built with --fmad=false and IEEE division, so each
//     operation rounds once in the order written and the flags are exact
//     functions of the fields);
//   * enzo_cluster_flags: Berger & Rigoutsos as Sec. 3.5 describes it, host
//     C++ over one grid's flags.
#include <cstdint>
#include <cstdlib>
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
    double gamma, slope, shock_dp, shock_e, mass;
};

// Primitive pieces of one cell used by the criteria.
struct FlagCell {
    double rho, E, e, p, m[3];
};

__device__ __forceinline__ FlagCell flag_cell(const FlagArgs &a, int64_t idx)
{
    FlagCell c;
    c.rho = a.U[0][idx];
    c.m[0] = a.U[1][idx];
    c.m[1] = a.U[2][idx];
    c.m[2] = a.U[3][idx];
    c.E = a.U[4][idx];
    const double ke = 0.5 * ((c.m[0] * c.m[0] + c.m[1] * c.m[1]) + c.m[2] * c.m[2]) / c.rho;
    c.e = c.E - ke;
    c.p = (a.gamma - 1.0) * c.e;
    return c;
}

// One tile = kCflCells active cells of one patch (the CFL work list).
__global__ void __launch_bounds__(256) flag_kernel(const __grid_constant__ FlagArgs a)
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
        const int64_t N0 = n[0] + 2 * P.ng, N1 = n[1] + 2 * P.ng;
        const int64_t stride[3] = {1, N0, N0 * N1};
        const bool wrap = (P.flags & ENZO_PATCH_PERIODIC) != 0;
        const int64_t ncell = (int64_t)n[0] * n[1] * n[2];
        const int64_t first = (int64_t)(tile - a.prefix[lo]) * kCflCells;
        const double vol = P.dx[0] * P.dx[0] * P.dx[0];
        for (int t = threadIdx.x; t < kCflCells; t += blockDim.x) {
            const int64_t cell = first + t;
            if (cell >= ncell) break;
            const int64_t row = cell / n[0];
            const int c[3] = {(int)(cell - row * n[0]), (int)(row % n[1]), (int)(row / n[1])};
            int64_t base = P.off;
            for (int d = 0; d < 3; ++d) base += (int64_t)(c[d] + P.ng) * stride[d];
            const FlagCell z = flag_cell(a, base);
            uint8_t f = 0;
            for (int ax = 0; ax < 3; ++ax) {
                // neighbours along ax: ghost cells, or the periodic images
                int64_t im = base - stride[ax], ip = base + stride[ax];
                if (wrap) {
                    const int cm = c[ax] == 0 ? n[ax] - 1 : c[ax] - 1;
                    const int cp = c[ax] == n[ax] - 1 ? 0 : c[ax] + 1;
                    im = base + (int64_t)(cm - c[ax]) * stride[ax];
                    ip = base + (int64_t)(cp - c[ax]) * stride[ax];
                }
                const FlagCell zm = flag_cell(a, im), zp = flag_cell(a, ip);
                if (a.slope > 0.0) {
                    if (fabs(zp.rho - zm.rho) / (2.0 * fabs(z.rho)) > a.slope) f |= ENZO_FLAG_SLOPE;
                    if (fabs(zp.E - zm.E) / (2.0 * fabs(z.E)) > a.slope) f |= ENZO_FLAG_SLOPE;
                }
                if (a.shock_dp > 0.0) {
                    const double pmin = zm.p < zp.p ? zm.p : zp.p;
                    const double um = zm.m[ax] / zm.rho, up = zp.m[ax] / zp.rho;
                    if (fabs(zp.p - zm.p) / pmin > a.shock_dp && um - up > 0.0 && z.e / z.E > a.shock_e)
                        f |= ENZO_FLAG_SHOCK;
                }
            }
            if (a.mass > 0.0 && z.rho * vol > a.mass) f |= ENZO_FLAG_MASS;
            a.flags[a.flag_off[lo] + cell] = f;
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
        : nx_(n[0]), ny_(n[1]), nz_(n[2]), cp_(cp), F_((size_t)n[0] * n[1] * n[2])
    {
        for (size_t i = 0; i < F_.size(); ++i) F_[i] = flags[i] != 0;
        grow();
        const int k = cp.margin;
        if (k > 0)
            for (int z = 0; z < nz_; ++z)
                for (int y = 0; y < ny_; ++y)
                    for (int x = 0; x < nx_; ++x)
                        if (x < k || x >= nx_ - k || y < k || y >= ny_ - k || z < k || z >= nz_ - k)
                            F_[((size_t)z * ny_ + y) * nx_ + x] = 0;
    }

    void run(std::vector<Region> &out)
    {
        // depth first, the low part before the high part: a stack popped from
        // the back with the high part pushed first
        std::vector<Region> stack;
        stack.push_back(Region{{0, 0, 0}, {nx_, ny_, nz_}});
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
    // Chebyshev growth by cp_.buffer cells: separable, x then y then z.
    void grow()
    {
        const int n[3] = {nx_, ny_, nz_};
        for (int ax = 0; ax < 3; ++ax)
            for (int it = 0; it < cp_.buffer; ++it) {
                std::vector<char> G(F_);
                for (int z = 0; z < nz_; ++z)
                    for (int y = 0; y < ny_; ++y)
                        for (int x = 0; x < nx_; ++x) {
                            const int c[3] = {x, y, z};
                            if (!F_[((size_t)z * ny_ + y) * nx_ + x]) continue;
                            for (int s = -1; s <= 1; s += 2) {
                                int q[3] = {c[0], c[1], c[2]};
                                q[ax] += s;
                                if (q[ax] < 0 || q[ax] >= n[ax]) continue;
                                G[((size_t)q[2] * ny_ + q[1]) * nx_ + q[0]] = 1;
                            }
                        }
                F_.swap(G);
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
                const char *row = &F_[((size_t)z * ny_ + y) * nx_];
                for (int x = r.lo[0]; x < r.hi[0]; ++x) {
                    if (!row[x]) continue;
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
    cudaStream_t s = static_cast<cudaStream_t>(b->stream);
    char *ws = static_cast<char *>(b->workspace);
    launch_tile_prefix(b->patches, b->npatch, b->field_len, kKindCells, 0, 0, reinterpret_cast<int *>(ws + kWsPrefix),
                       reinterpret_cast<unsigned *>(ws + kWsCounter), nullptr, b->status, s);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    FlagArgs a;
    a.patches = b->patches;
    a.npatch = b->npatch;
    for (int f = 0; f < 5; ++f) a.U[f] = b->U[f];
    a.prefix = reinterpret_cast<const int *>(ws + kWsPrefix);
    a.flags = flags;
    a.flag_off = flag_off;
    a.gamma = fp->gamma;
    a.slope = fp->slope;
    a.shock_dp = fp->shock_dp;
    a.shock_e = fp->shock_e;
    a.mass = fp->mass;
    flag_kernel<<<sms() * 8, 256, 0, s>>>(a);
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
