// Static AMR hierarchy operations around the sweep (paper Sec. 3):
//   ghost fill of refined levels (parent interpolation by SecondOrderA,
//   Appendix A, after linear interpolation in time; then sibling copies),
//   flux correction at coarse-fine faces (Sec. 3.4) and projection (Sec. 3.3).
//   With dual energy (Sec. 4.1.1) the gas energy is a sixth field of each.
// FP64 throughout; built with --fmad=false so every operation rounds once in
// the order written.
#include <cstdint>

#include "internal.cuh"

namespace enzo {

constexpr double kEps = 1e-300;

__device__ __forceinline__ double minmod(double a, double b)
{
    const double aa = fabs(a), ab = fabs(b);
    const double m = aa < ab ? aa : ab;
    const double out = a > 0.0 ? m : (a < 0.0 ? -m : 0.0);
    return a * b < 0.0 ? 0.0 : out;
}

// SecondOrderA value of child (kz, ky, kx) of the centre of a 3x3x3 parent
// neighbourhood Q[z][y][x] (r = 2).  T = double: the FP64 arithmetic (the oracle's order);
// T = float: the same steps for the FP32 path (ghost values only feed the
// FP32 reconstruction; conservation is kept by flux correction).
template <class T>
__device__ __forceinline__ T minmod_t(T a, T b)
{
    const T aa = fabs(a), ab = fabs(b);
    const T m = aa < ab ? aa : ab;
    const T out = a > (T)0 ? m : (a < (T)0 ? -m : (T)0);
    return a * b < (T)0 ? (T)0 : out;
}

template <class T>
__device__ __forceinline__ T second_order_a(const T Q[3][3][3], int kz, int ky, int kx)
{
    const T Q0 = Q[1][1][1];
    T C[2][2][2];
#pragma unroll
    for (int sz = 0; sz < 2; ++sz)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy)
#pragma unroll
            for (int sx = 0; sx < 2; ++sx) {
                T acc = (T)0;
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) acc = acc + Q[sz + dz][sy + dy][sx + dx];
                C[sz][sy][sx] = acc * (T)0.125;
            }
    // diagonals: plus corners (z,y,x) = (1,1,1), (1,1,0), (1,0,1), (0,1,1)
    const T d0 = minmod_t(C[1][1][1] - Q0, Q0 - C[0][0][0]);
    const T d1 = minmod_t(C[1][1][0] - Q0, Q0 - C[0][0][1]);
    const T d2 = minmod_t(C[1][0][1] - Q0, Q0 - C[0][1][0]);
    const T d3 = minmod_t(C[0][1][1] - Q0, Q0 - C[1][0][0]);
    T a1 = d1, a2 = d2, a3 = d3;
    if (d0 == (T)0) {
        a1 = a2 = a3 = (T)0;
    } else {
        const T s = ((d1 + d2) + d3) / d0;
        if (s < (T)0 || s > (T)1) {
            const T sp = s < (T)0 ? (T)0 : (T)1;
            const T c1 = s < (T)0 ? (d1 / d0 < (T)0 ? (T)1 : (T)0) : (d1 / d0 > (T)0 ? (T)1 : (T)0);
            const T c2 = s < (T)0 ? (d2 / d0 < (T)0 ? (T)1 : (T)0) : (d2 / d0 > (T)0 ? (T)1 : (T)0);
            const T c3 = s < (T)0 ? (d3 / d0 < (T)0 ? (T)1 : (T)0) : (d3 / d0 > (T)0 ? (T)1 : (T)0);
            const T num = sp * d0 - ((((T)1 - c1) * d1 + ((T)1 - c2) * d2) + ((T)1 - c3) * d3);
            const T den = ((c1 * d1 + c2 * d2) + c3 * d3) + (sizeof(T) == 8 ? (T)kEps : (T)1e-37f);
            const T f = num / den;
            a1 = f * c1 * d1 + ((T)1 - c1) * d1;
            a2 = f * c2 * d2 + ((T)1 - c2) * d2;
            a3 = f * c3 * d3 + ((T)1 - c3) * d3;
        }
    }
    const T fx = a2 + a3, fy = a1 + a3, fz = a1 + a2;
    const T cx = kx ? (T)0.25 : (T)-0.25, cy = ky ? (T)0.25 : (T)-0.25, cz = kz ? (T)0.25 : (T)-0.25;
    return ((Q0 + cx * fx) + cy * fy) + cz * fz;
}

// float <-> double on the integer pipe (d2f_rz, f2d_exact: internal.cuh)
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return f2d_exact(x); }
template <class T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return d2f_rz(x); }

__device__ __forceinline__ int floordiv2(int g) { return g >= 0 ? g / 2 : -((1 - g) / 2); }

// Fields carried by the hierarchy operations: the five conserved ones, and the
// gas energy as a sixth when the batches have it (dual energy, Sec. 4.1.1).
constexpr int kMaxFields = 6;

struct InterpArgs {
    const enzo_patch *fine;
    const enzo_patch_link *flink;
    double *U[kMaxFields];
    const enzo_patch *par;
    const enzo_patch_link *plink;
    const double *Pn[kMaxFields];
    const double *Po[kMaxFields];
    int nf;
    double w;
    const enzo_copy_box *boxes;   // ghost regions no sibling covers (src unused)
    int nbox;
};

// Ghost cells of the listed boxes get the parent's SecondOrderA value (one CTA
// per box: boxes are the 3-cell-thick face, edge and corner slabs of a patch's
// ghost shell; cells that siblings cover are copied afterwards and not listed).
template <class T>
__global__ void __launch_bounds__(128) interp_ghosts_kernel(const __grid_constant__ InterpArgs a)
{
    for (int bi = blockIdx.x; bi < a.nbox; bi += gridDim.x) {
        const enzo_copy_box B = a.boxes[bi];
        const enzo_patch P = a.fine[B.dst];
        const enzo_patch_link L = a.flink[B.dst];
        if (L.parent < 0) continue;
        const enzo_patch PP = a.par[L.parent];
        const enzo_patch_link PL = a.plink[L.parent];
        const int e0 = B.hi[0] - B.lo[0], e1 = B.hi[1] - B.lo[1], e2 = B.hi[2] - B.lo[2];
        const int vol = e0 * e1 * e2, e01 = e0 * e1;
        const int N0 = P.n[0] + 2 * P.ng, N1 = P.n[1] + 2 * P.ng;
        const int M0 = PP.n[0] + 2 * PP.ng, M1 = PP.n[1] + 2 * PP.ng;
        const T w = (T)a.w;
        for (int c = threadIdx.x; c < vol; c += blockDim.x) {
            const int gz = c / e01, rem = c - gz * e01, gy = rem / e0;
            const int g[3] = {B.lo[0] + rem - gy * e0, B.lo[1] + gy, B.lo[2] + gz};
            int kid[3], ps[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int G = floordiv2(g[d]);
                kid[d] = g[d] - 2 * G;
                ps[d] = G - PL.origin[d] + PP.ng;
            }
            const int64_t dst = P.off + (g[0] - L.origin[0] + P.ng) +
                                (int64_t)N0 * ((g[1] - L.origin[1] + P.ng) + (int64_t)N1 * (g[2] - L.origin[2] + P.ng));
            const int64_t base = PP.off + (ps[0] - 1) + (int64_t)M0 * ((ps[1] - 1) + (int64_t)M1 * (ps[2] - 1));
            for (int f = 0; f < a.nf; ++f) {
                T Q[3][3][3];
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const int64_t idx = base + dx + (int64_t)M0 * (dy + (int64_t)M1 * dz);
                            const T o = from_d<T>(a.Po[f][idx]), n = from_d<T>(a.Pn[f][idx]);
                            Q[dz][dy][dx] = o + w * (n - o);
                        }
                a.U[f][dst] = to_d(second_order_a<T>(Q, kid[2], kid[1], kid[0]));
            }
        }
    }
}

// Ghost boxes copied from siblings: one CTA per box (boxes are the face, edge
// and corner slabs of a patch's ghost shell, 27 to a few thousand cells).
// Each thread loads the fields (five, six with the gas energy) of two cells
// before storing any, so that enough loads are in flight to cover HBM latency
// (sources are active cells, which this kernel never writes).
// The source patches may belong to another batch of the same level (a
// rebuild copying the old grids into the new ones).
struct CopyArgs {
    const enzo_patch *dpt, *spt;
    const enzo_patch_link *dlk, *slk;
    double *D[kMaxFields];
    const double *S[kMaxFields];
    int nf;
    const enzo_copy_box *boxes;
    int nbox;
};

__global__ void __launch_bounds__(128) copy_boxes_kernel(const __grid_constant__ CopyArgs a)
{
    for (int bi = blockIdx.x; bi < a.nbox; bi += gridDim.x) {
        const enzo_copy_box B = a.boxes[bi];
        const enzo_patch D = a.dpt[B.dst], S = a.spt[B.src];
        const enzo_patch_link DL = a.dlk[B.dst], SL = a.slk[B.src];
        const int e0 = B.hi[0] - B.lo[0], e1 = B.hi[1] - B.lo[1], e2 = B.hi[2] - B.lo[2];
        const int vol = e0 * e1 * e2, e01 = e0 * e1;
        const int D0 = D.n[0] + 2 * D.ng, D01 = D0 * (D.n[1] + 2 * D.ng);
        const int S0 = S.n[0] + 2 * S.ng, S01 = S0 * (S.n[1] + 2 * S.ng);
        // box origin inside each patch's ghosted block
        const int64_t dbase = D.off + (B.lo[0] - DL.origin[0] + D.ng) + (int64_t)D0 * (B.lo[1] - DL.origin[1] + D.ng) +
                              (int64_t)D01 * (B.lo[2] - DL.origin[2] + D.ng);
        const int64_t sbase = S.off + (B.lo[0] - SL.origin[0] + S.ng) + (int64_t)S0 * (B.lo[1] - SL.origin[1] + S.ng) +
                              (int64_t)S01 * (B.lo[2] - SL.origin[2] + S.ng);
        for (int c0 = 0; c0 < vol; c0 += 2 * blockDim.x) {
            int64_t di[2], si[2];
            double v[2][kMaxFields];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int c = c0 + threadIdx.x + k * blockDim.x;
                const int z = c / e01, rem = c - z * e01;
                const int y = rem / e0, x = rem - y * e0;
                di[k] = c < vol ? dbase + x + (int64_t)D0 * y + (int64_t)D01 * z : -1;
                si[k] = sbase + x + (int64_t)S0 * y + (int64_t)S01 * z;
                if (c < vol)
#pragma unroll
                    for (int f = 0; f < kMaxFields; ++f)
                        if (f < a.nf) v[k][f] = a.S[f][si[k]];
            }
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (di[k] >= 0)
#pragma unroll
                    for (int f = 0; f < kMaxFields; ++f)
                        if (f < a.nf) a.D[f][di[k]] = v[k][f];
        }
    }
}

struct FcArgs {
    const enzo_patch *cp;
    const enzo_patch_link *cl;
    double *U[kMaxFields];
    int nc;                   // register components per face (5, 6 with gas energy)
    const double *cfreg;
    const enzo_patch *fp;
    const enzo_patch_link *fl;
    const double *ffreg;
    const enzo_fc_face *faces;
    int nface;
    double dt_c;
    int increments;
};

__device__ __forceinline__ int64_t reg_all_block(const enzo_patch &P, int dir, int nc)
{
    int64_t o = 0;
    for (int d = 0; d < dir; ++d) {
        const int b1 = d == 0 ? 1 : 0, b2 = d == 2 ? 1 : 2;
        o += (int64_t)(P.n[d] + 1) * P.n[b1] * P.n[b2] * nc;
    }
    return o;
}
__device__ __forceinline__ int64_t reg_bnd_block(const enzo_patch &P, int dir, int nc)
{
    int64_t o = 0;
    for (int d = 0; d < dir; ++d) {
        const int b1 = d == 0 ? 1 : 0, b2 = d == 2 ? 1 : 2;
        o += (int64_t)2 * P.n[b1] * P.n[b2] * nc;
    }
    return o;
}

// One CTA per listed fine face part; threads over the coarse faces it covers.
__global__ void __launch_bounds__(128) flux_correct_kernel(const __grid_constant__ FcArgs a)
{
    for (int fi = blockIdx.x; fi < a.nface; fi += gridDim.x) {
        const enzo_fc_face F = a.faces[fi];
        const enzo_patch FP = a.fp[F.fine];
        const enzo_patch_link FL = a.fl[F.fine];
        const enzo_patch PP = a.cp[FL.parent];
        const enzo_patch_link PL = a.cl[FL.parent];
        const enzo_patch TP = a.cp[F.target];
        const enzo_patch_link TL = a.cl[F.target];
        const int d = F.dir, a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
        const int X = (FL.origin[d] + (F.side ? FP.n[d] : 0)) / 2;
        const int cell = F.side ? X : X - 1;
        const int fc = X - PL.origin[d];
        const int e1 = F.hi[0] - F.lo[0], e2 = F.hi[1] - F.lo[1];
        const int nc = a.nc;
        const double *creg = a.cfreg + PP.freg_all + reg_all_block(PP, d, nc);
        const double *freg = a.ffreg + FP.freg_bnd + reg_bnd_block(FP, d, nc);
        const int fna1 = FP.n[a1];
        const int T0 = TP.n[0] + 2 * TP.ng, T1 = TP.n[1] + 2 * TP.ng;
        // fields in pencil order (rho, m_n, m_t1, m_t2, E, then the gas energy)
        double *const Uf[kMaxFields] = {a.U[0], d == 0 ? a.U[1] : (d == 1 ? a.U[2] : a.U[3]),
                                        a1 == 0 ? a.U[1] : a.U[2], a2 == 1 ? a.U[2] : a.U[3], a.U[4], a.U[5]};
        for (int q = threadIdx.x; q < e1 * e2; q += blockDim.x) {
            const int q1 = F.lo[0] + q % e1, q2 = F.lo[1] + q / e1;
            const int c1 = FL.origin[a1] / 2 + q1, c2 = FL.origin[a2] / 2 + q2;
            const double *cf = creg + (((int64_t)(c2 - PL.origin[a2]) * PP.n[a1] + (c1 - PL.origin[a1])) *
                                           (PP.n[d] + 1) + fc) * nc;
            const double *f00 = freg + (((int64_t)(2 * q2) * fna1 + 2 * q1) * 2 + F.side) * nc;
            const double *f01 = freg + (((int64_t)(2 * q2) * fna1 + 2 * q1 + 1) * 2 + F.side) * nc;
            const double *f10 = freg + (((int64_t)(2 * q2 + 1) * fna1 + 2 * q1) * 2 + F.side) * nc;
            const double *f11 = freg + (((int64_t)(2 * q2 + 1) * fna1 + 2 * q1 + 1) * 2 + F.side) * nc;
            int g[3];
            g[d] = cell;
            g[a1] = c1;
            g[a2] = c2;
            const int64_t idx = TP.off + (g[0] - TL.origin[0] + TP.ng) +
                                (int64_t)T0 * ((g[1] - TL.origin[1] + TP.ng) + (int64_t)T1 * (g[2] - TL.origin[2] + TP.ng));
#pragma unroll
            for (int v = 0; v < kMaxFields; ++v) {
                if (v >= nc) break;
                double delta;
                if (a.increments) {
                    // registers hold applied increments (U units): the fine ones
                    // carry a factor dx_f / dx_c = 1/2 and the 4 faces a mean
                    delta = cf[v] - (((f00[v] + f01[v]) + f10[v]) + f11[v]) * 0.125;
                } else {
                    const double fine = (((f00[v] + f01[v]) + f10[v]) + f11[v]) * 0.25;
                    delta = (a.dt_c * cf[v] - fine) / TP.dx[d];
                }
                atomicAdd(&Uf[v][idx], F.side ? -delta : delta);
            }
        }
    }
}

struct ProjArgs {
    const enzo_patch *cp;
    const enzo_patch_link *cl;
    double *U[kMaxFields];
    const enzo_patch *fp;
    const enzo_patch_link *fl;
    const double *F[kMaxFields];
    int nf;
    int nfine;
};

// One CTA per fine patch: its covered coarse cells get the mean of their 8 children.
__global__ void __launch_bounds__(256) project_kernel(const __grid_constant__ ProjArgs a)
{
    for (int pi = blockIdx.x; pi < a.nfine; pi += gridDim.x) {
        const enzo_patch FP = a.fp[pi];
        const enzo_patch_link FL = a.fl[pi];
        if (FL.parent < 0) continue;
        const enzo_patch PP = a.cp[FL.parent];
        const enzo_patch_link PL = a.cl[FL.parent];
        const int m0 = FP.n[0] / 2, m1 = FP.n[1] / 2, m2 = FP.n[2] / 2;
        const int F0 = FP.n[0] + 2 * FP.ng, F1 = FP.n[1] + 2 * FP.ng;
        const int P0 = PP.n[0] + 2 * PP.ng, P1 = PP.n[1] + 2 * PP.ng;
        const int64_t vol = (int64_t)m0 * m1 * m2;
        for (int64_t c = threadIdx.x; c < vol; c += blockDim.x) {
            const int x = (int)(c % m0), y = (int)((c / m0) % m1), z = (int)(c / ((int64_t)m0 * m1));
            const int64_t pidx = PP.off + (FL.origin[0] / 2 + x - PL.origin[0] + PP.ng) +
                                 (int64_t)P0 * ((FL.origin[1] / 2 + y - PL.origin[1] + PP.ng) +
                                                (int64_t)P1 * (FL.origin[2] / 2 + z - PL.origin[2] + PP.ng));
            // all loads (8 per field) before the stores (coarse and fine fields
            // are distinct arrays, but the compiler cannot know that)
            double v[kMaxFields][8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
                const int64_t fidx = FP.off + (2 * x + kx + FP.ng) +
                                     (int64_t)F0 * ((2 * y + ky + FP.ng) + (int64_t)F1 * (2 * z + kz + FP.ng));
#pragma unroll
                for (int f = 0; f < kMaxFields; ++f)
                    if (f < a.nf) v[f][k] = a.F[f][fidx];
            }
#pragma unroll
            for (int f = 0; f < kMaxFields; ++f) {
                if (f >= a.nf) break;
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < 8; ++k) s = s + v[f][k];
                a.U[f][pidx] = s * 0.125;
            }
        }
    }
}

static int sm_count()
{
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s > 0 ? s : 1;
}

static bool batch_ok(const enzo_patch_batch *b)
{
    if (!b || b->npatch < 0) return false;
    if (b->npatch == 0) return true;
    if (!b->patches) return false;
    for (int f = 0; f < 5; ++f)
        if (!b->U[f]) return false;
    return true;
}

}  // namespace enzo

using namespace enzo;

extern "C" {

int enzo_ghost_fill_level(const enzo_patch_batch *fine, const enzo_patch_link *fine_links,
                          const enzo_patch_batch *parent_new, const enzo_patch_link *parent_links,
                          double *const parent_old_U[5], const double *parent_old_ge, double w,
                          const enzo_copy_box *interp_boxes, int32_t ninterp, const enzo_copy_box *copy_boxes,
                          int32_t ncopy, int32_t precision, int32_t r)
{
    if (r != 2 || !batch_ok(fine) || !batch_ok(parent_new) || !fine_links || !parent_links || !parent_old_U)
        return ENZO_ERR_ARG;
    // the gas energy goes with the level: fine, parent and the parent's old
    // state all carry it or none does
    const bool ge = fine->ge != nullptr;
    if ((parent_new->ge != nullptr) != ge || (ge && ninterp > 0 && !parent_old_ge) || (!ge && parent_old_ge))
        return ENZO_ERR_ARG;
    const int nf = ge ? 6 : 5;
    if (!(w >= 0.0) || !(w <= 1.0) || ninterp < 0 || ncopy < 0 || (ninterp > 0 && !interp_boxes) ||
        (ncopy > 0 && !copy_boxes))
        return ENZO_ERR_ARG;
    if (precision != ENZO_FP64 && precision != ENZO_FP32) return ENZO_ERR_ARG;
    if (fine->npatch == 0) return ENZO_OK;
    for (int f = 0; f < 5; ++f)
        if (!parent_old_U[f]) return ENZO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(fine->stream);
    if (ninterp > 0) {
        InterpArgs a;
        a.fine = fine->patches;
        a.flink = fine_links;
        for (int f = 0; f < 5; ++f) {
            a.U[f] = fine->U[f];
            a.Pn[f] = parent_new->U[f];
            a.Po[f] = parent_old_U[f];
        }
        a.U[5] = fine->ge;
        a.Pn[5] = parent_new->ge;
        a.Po[5] = parent_old_ge;
        a.nf = nf;
        a.par = parent_new->patches;
        a.plink = parent_links;
        a.w = w;
        a.boxes = interp_boxes;
        a.nbox = ninterp;
        // one CTA per box (boxes are short; a grid-stride over a resident grid
        // measured slower)
        const int grid = ninterp < sm_count() * 16 ? ninterp : sm_count() * 16;
        if (precision == ENZO_FP64) interp_ghosts_kernel<double><<<grid, 128, 0, s>>>(a);
        else interp_ghosts_kernel<float><<<grid, 128, 0, s>>>(a);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    }
    if (ncopy > 0) {
        CopyArgs c;
        c.dpt = c.spt = fine->patches;
        c.dlk = c.slk = fine_links;
        for (int f = 0; f < 5; ++f) {
            c.D[f] = fine->U[f];
            c.S[f] = fine->U[f];
        }
        c.D[5] = fine->ge;
        c.S[5] = fine->ge;
        c.nf = nf;
        c.boxes = copy_boxes;
        c.nbox = ncopy;
        copy_boxes_kernel<<<ncopy, 128, 0, s>>>(c);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return ENZO_ERR_CUDA;
    }
    return ENZO_OK;
}

int enzo_copy_level(const enzo_patch_batch *dst, const enzo_patch_link *dst_links, const enzo_patch_batch *src,
                    const enzo_patch_link *src_links, const enzo_copy_box *boxes, int32_t nbox)
{
    if (!batch_ok(dst) || !batch_ok(src) || !dst_links || !src_links || nbox < 0 || (nbox > 0 && !boxes))
        return ENZO_ERR_ARG;
    if ((dst->ge != nullptr) != (src->ge != nullptr)) return ENZO_ERR_ARG;
    if (nbox == 0) return ENZO_OK;
    CopyArgs c;
    c.dpt = dst->patches;
    c.spt = src->patches;
    c.dlk = dst_links;
    c.slk = src_links;
    for (int f = 0; f < 5; ++f) {
        c.D[f] = dst->U[f];
        c.S[f] = src->U[f];
    }
    c.D[5] = dst->ge;
    c.S[5] = src->ge;
    c.nf = dst->ge ? 6 : 5;
    c.boxes = boxes;
    c.nbox = nbox;
    copy_boxes_kernel<<<nbox < sm_count() * 16 ? nbox : sm_count() * 16, 128, 0,
                        static_cast<cudaStream_t>(dst->stream)>>>(c);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_flux_correct(const enzo_patch_batch *coarse, const enzo_patch_link *coarse_links,
                      const enzo_patch_batch *fine, const enzo_patch_link *fine_links, const enzo_fc_face *faces,
                      int32_t nface, double dt_coarse, int32_t r, int32_t increments)
{
    if (r != 2 || !batch_ok(coarse) || !batch_ok(fine) || !coarse_links || !fine_links) return ENZO_ERR_ARG;
    if (nface < 0 || (nface > 0 && !faces) || !(dt_coarse >= 0.0)) return ENZO_ERR_ARG;
    if ((coarse->ge != nullptr) != (fine->ge != nullptr)) return ENZO_ERR_ARG;
    if (nface == 0) return ENZO_OK;
    if (!coarse->freg || !fine->freg) return ENZO_ERR_ARG;
    FcArgs a;
    a.cp = coarse->patches;
    a.cl = coarse_links;
    for (int f = 0; f < 5; ++f) a.U[f] = coarse->U[f];
    a.U[5] = coarse->ge;
    a.nc = coarse->ge ? 6 : 5;
    a.cfreg = coarse->freg;
    a.fp = fine->patches;
    a.fl = fine_links;
    a.ffreg = fine->freg;
    a.faces = faces;
    a.nface = nface;
    a.dt_c = dt_coarse;
    a.increments = increments ? 1 : 0;
    flux_correct_kernel<<<nface < sm_count() * 16 ? nface : sm_count() * 16, 128, 0,
                          static_cast<cudaStream_t>(coarse->stream)>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

int enzo_project(const enzo_patch_batch *coarse, const enzo_patch_link *coarse_links, const enzo_patch_batch *fine,
                 const enzo_patch_link *fine_links, int32_t r)
{
    if (r != 2 || !batch_ok(coarse) || !batch_ok(fine) || !coarse_links || !fine_links) return ENZO_ERR_ARG;
    if ((coarse->ge != nullptr) != (fine->ge != nullptr)) return ENZO_ERR_ARG;
    if (fine->npatch == 0) return ENZO_OK;
    ProjArgs a;
    a.cp = coarse->patches;
    a.cl = coarse_links;
    for (int f = 0; f < 5; ++f) {
        a.U[f] = coarse->U[f];
        a.F[f] = fine->U[f];
    }
    a.U[5] = coarse->ge;
    a.F[5] = fine->ge;
    a.nf = coarse->ge ? 6 : 5;
    a.fp = fine->patches;
    a.fl = fine_links;
    a.nfine = fine->npatch;
    project_kernel<<<fine->npatch, 256, 0,
                     static_cast<cudaStream_t>(coarse->stream)>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ENZO_OK : ENZO_ERR_CUDA;
}

}  // extern "C"
