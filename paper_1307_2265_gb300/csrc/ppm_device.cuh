// Device code of the split PPM sweep, templated on the arithmetic type.
//
// R = double: the FP64 path.  Its translation unit is compiled with
// --fmad=false and IEEE division/square root, and every formula keeps the
// association written here, so results are reproducible operation by
// operation.
// R = float: the FP32 path (fast reciprocal/sqrt, FMA contraction allowed);
// conserved variables stay FP64 in memory and are updated in FP64, and the
// internal energy E - KE is recovered in FP64 where E - KE < eta * E
// (high-Mach cells).
//
// Method (paper Sec. 4.1 and 4.1.2, reconstruction formulas of CW84 that the
// paper defers to):
//   primitives rho, u_n, p, u_t1, u_t2 from the conserved state (Sec. 2.1);
//   limited slopes and interface values q_{j+1/2}; monotone parabola per zone
//   (q_L, q_R, Delta q, q6); averages over the u-c, u, u+c domains of
//   dependence; characteristic left/right states (reference wave plus beta
//   corrections); two-shock Riemann solve with Newton iteration on p* (or the
//   HLL / HLLC approximate solvers on the traced states); fluxes;
//   U_j += dt/dx (F_{j-1/2} - F_{j+1/2}); HLL re-flux of cells whose density
//   would drop to <= 0.  The Newton start is the plain two-shock guess or, in
//   the FP32 path, a small network evaluated on the tensor cores
//   (LearnedGuess).
//
// Thread layout: one thread marches one pencil from one end to the other,
// holding a sliding window of zones in registers: reading cell k it finishes
// the slope of zone k-1, the interface value at (k-2)+1/2, the parabola and
// both edge states of zone k-2, the Riemann problem at (k-3)+1/2, decides
// whether cell k-3 needs the fallback, and writes cell k-4.  Threads of a
// warp take neighbouring pencils, which for y and z sweeps are neighbouring
// x positions (coalesced loads and stores).
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "internal.cuh"
#include "mlp_layout.cuh"
#include "tc05.cuh"

// Cache prefetch of the march: a position's five fields are requested this
// many steps before their load (0: off).
#ifndef ENZO_PREFETCH_AHEAD
#define ENZO_PREFETCH_AHEAD 2
#endif
#ifndef ENZO_NEWTON_HEAD
#define ENZO_NEWTON_HEAD 3   // FP32 Newton: evaluations done as straight-line code before the loop
#endif
#ifdef ENZO_PREFETCH_TO_L2
#define ENZO_PREFETCH(p) asm volatile("prefetch.global.L2 [%0];" ::"l"(p))
#else
#define ENZO_PREFETCH(p) asm volatile("prefetch.global.L1 [%0];" ::"l"(p))
#endif

namespace enzo {

template <class R>
struct Consts {
    R gamma, gm1, gm1inv, gp1o2g, rho_floor, p_floor, tol, step_tol, eta_eke;
    int nmax;
};

template <class R>
__device__ __forceinline__ Consts<R> make_consts(const MethodParams &m)
{
    Consts<R> k;
    k.gamma = (R)m.gamma;
    k.gm1 = (R)(m.gamma - 1.0);
    k.gm1inv = (R)(1.0 / (m.gamma - 1.0));
    k.gp1o2g = (R)((m.gamma + 1.0) / (2.0 * m.gamma));
    k.rho_floor = (R)m.rho_floor;
    k.p_floor = (R)m.p_floor;
    k.tol = (R)m.newton_tol;
    k.step_tol = sizeof(R) == 8 ? (R)0 : (R)4e-7;
    k.eta_eke = (R)0.05;
    k.nmax = m.newton_max;
    return k;
}

template <class R>
struct Zone {
    R r, u, p, t1, t2, c;
};

__device__ __forceinline__ double div6(double x) { return x / 6.0; }
__device__ __forceinline__ float div6(float x) { return x * (1.0f / 6.0f); }

// Load of a field value by the march (and the update's read of a cell's old
// value where no ring holds it).  An x pencil's thread reads its own row, one
// cache line per 16 positions, and the lines of a warp's 32 rows and five
// fields outgrow L1 before they are used up: x loads ask L1 to keep their
// lines (evict_last).  y and z sweeps read each line once per warp.  A cell is
// read this way only before its own thread writes it.
template <int DIR>
__device__ __forceinline__ double ld_march(const double *p)
{
    if constexpr (DIR == 0) {
        double v;
        asm volatile("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    } else {
        return __ldg(p);
    }
}

// Primitive state of one cell from its conserved values (Sec. 2.1), with floors.
template <class R, bool COUNT>
__device__ __forceinline__ Zone<R> prim(double rho64, double mn64, double m164, double m264,
                                        double E64, const Consts<R> &k, Counters &cnt);

template <>
__device__ __forceinline__ Zone<double> prim<double, true>(double rho, double mn, double m1,
                                                           double m2, double E,
                                                           const Consts<double> &k,
                                                           Counters &cnt)
{
    Zone<double> z;
    if (!(rho >= k.rho_floor)) { rho = k.rho_floor; cnt.rare(ENZO_ST_RHO_FLOOR); }
    double ke = 0.5 * ((mn * mn + m1 * m1) + m2 * m2) / rho;
    double p = k.gm1 * (E - ke);
    if (!(p >= k.p_floor)) { p = k.p_floor; cnt.rare(ENZO_ST_P_FLOOR); }
    z.r = rho;
    z.u = mn / rho;
    z.p = p;
    z.t1 = m1 / rho;
    z.t2 = m2 / rho;
    z.c = sqrt(k.gamma * p / rho);
    return z;
}

template <>
__device__ __forceinline__ Zone<double> prim<double, false>(double rho, double mn, double m1,
                                                            double m2, double E,
                                                            const Consts<double> &k,
                                                            Counters &cnt)
{
    Counters quiet;
    return prim<double, true>(rho, mn, m1, m2, E, k, quiet);
}

template <bool COUNT>
__device__ __forceinline__ Zone<float> prim_f(double rho64, double mn64, double m164,
                                              double m264, double E64, const Consts<float> &k,
                                              Counters &cnt)
{
    Zone<float> z;
    float rho = d2f_rz(rho64);
    if (!(rho >= k.rho_floor)) { rho = k.rho_floor; rho64 = f2d_exact(rho); if (COUNT) cnt.rare(ENZO_ST_RHO_FLOOR); }
    const float inv = 1.0f / rho;
    const float mn = d2f_rz(mn64), m1 = d2f_rz(m164), m2 = d2f_rz(m264), E = d2f_rz(E64);
    const float ke = 0.5f * ((mn * mn + m1 * m1) + m2 * m2) * inv;
    float e = E - ke;
    if (e < k.eta_eke * E) {
        // high-Mach cell: the internal energy is a small difference of two
        // large numbers, so it is recovered in FP64
        const double ke64 = 0.5 * ((mn64 * mn64 + m164 * m164) + m264 * m264) / rho64;
        e = (float)(E64 - ke64);
        if (COUNT) cnt.rare(ENZO_ST_FP64_EKE);
    }
    float p = k.gm1 * e;
    if (!(p >= k.p_floor)) { p = k.p_floor; if (COUNT) cnt.rare(ENZO_ST_P_FLOOR); }
    z.r = rho;
    z.u = mn * inv;
    z.p = p;
    z.t1 = m1 * inv;
    z.t2 = m2 * inv;
    z.c = sqrtf(k.gamma * p * inv);
    return z;
}

template <>
__device__ __forceinline__ Zone<float> prim<float, true>(double rho, double mn, double m1,
                                                         double m2, double E,
                                                         const Consts<float> &k, Counters &cnt)
{
    return prim_f<true>(rho, mn, m1, m2, E, k, cnt);
}

template <>
__device__ __forceinline__ Zone<float> prim<float, false>(double rho, double mn, double m1,
                                                          double m2, double E,
                                                          const Consts<float> &k, Counters &cnt)
{
    return prim_f<false>(rho, mn, m1, m2, E, k, cnt);
}

// Primitive state with the dual-energy option (Sec. 4.1.1): the pressure comes
// from the gas energy ge where E - KE < 1e-3 E, else from E - KE; eps = ge / rho
// is the specific gas energy, carried like a transverse velocity.  The choice is
// taken in FP64 in both precisions.  FP64: the same arithmetic as prim<double>.
template <bool COUNT>
__device__ __forceinline__ Zone<double> prim_dual(double rho, double mn, double m1, double m2, double E,
                                                  double ge, const Consts<double> &k, Counters &cnt,
                                                  double &eps)
{
    Zone<double> z;
    if (!(rho >= k.rho_floor)) { rho = k.rho_floor; if (COUNT) cnt.rare(ENZO_ST_RHO_FLOOR); }
    const double ke = 0.5 * ((mn * mn + m1 * m1) + m2 * m2) / rho;
    double p;
    if (E - ke < 1e-3 * E) {
        p = k.gm1 * ge;
        if (COUNT) cnt.gep++;
    } else {
        p = k.gm1 * (E - ke);
    }
    if (!(p >= k.p_floor)) { p = k.p_floor; if (COUNT) cnt.rare(ENZO_ST_P_FLOOR); }
    z.r = rho;
    z.u = mn / rho;
    z.p = p;
    z.t1 = m1 / rho;
    z.t2 = m2 / rho;
    z.c = sqrt(k.gamma * p / rho);
    eps = ge / rho;
    return z;
}

// FP32: as prim_f; a zone whose FP32 internal energy is below 5% of E (the only
// zones where E - KE can fall under 1e-3 E) recovers E - KE in FP64 and takes
// the gas-energy pressure where that is below 1e-3 E.
template <bool COUNT>
__device__ __forceinline__ Zone<float> prim_dual(double rho64, double mn64, double m164, double m264,
                                                 double E64, double ge64, const Consts<float> &k,
                                                 Counters &cnt, float &eps)
{
    Zone<float> z;
    float rho = d2f_rz(rho64);
    if (!(rho >= k.rho_floor)) { rho = k.rho_floor; rho64 = f2d_exact(rho); if (COUNT) cnt.rare(ENZO_ST_RHO_FLOOR); }
    const float inv = 1.0f / rho;
    const float mn = d2f_rz(mn64), m1 = d2f_rz(m164), m2 = d2f_rz(m264), E = d2f_rz(E64);
    const float ke = 0.5f * ((mn * mn + m1 * m1) + m2 * m2) * inv;
    float e = E - ke;
    if (e < k.eta_eke * E) {
        const double ke64 = 0.5 * ((mn64 * mn64 + m164 * m164) + m264 * m264) / rho64;
        if (E64 - ke64 < 1e-3 * E64) {
            e = d2f_rz(ge64);
            if (COUNT) cnt.gep++;
        } else {
            e = (float)(E64 - ke64);
        }
        if (COUNT) cnt.rare(ENZO_ST_FP64_EKE);
    }
    float p = k.gm1 * e;
    if (!(p >= k.p_floor)) { p = k.p_floor; if (COUNT) cnt.rare(ENZO_ST_P_FLOOR); }
    z.r = rho;
    z.u = mn * inv;
    z.p = p;
    z.t1 = m1 * inv;
    z.t2 = m2 * inv;
    z.c = sqrtf(k.gamma * p * inv);
    eps = d2f_rz(ge64) * inv;
    return z;
}

template <class R>
__device__ __forceinline__ R zv(const Zone<R> &z, int v)
{
    return v == 0 ? z.r : v == 1 ? z.u : v == 2 ? z.p : v == 3 ? z.t1 : z.t2;
}

// Limited slope of zone j (CW84 1.7-1.8).
template <class R>
__device__ __forceinline__ R limited_slope(R qm, R q0, R qp)
{
    const R dl = q0 - qm;
    const R dr = qp - q0;
    const R dc = (R)0.5 * (qp - qm);
    R r = (R)0;
    if (dl * dr > (R)0) {
        const R a = fabs(dc), b = (R)2 * fabs(dl), e = (R)2 * fabs(dr);
        R m = a < b ? a : b;
        m = m < e ? m : e;
        r = dc >= (R)0 ? m : -m;
    }
    return r;
}

// Monotone parabola of a zone (CW84 1.10): edges ql, qr in, (qL, Delta q, q6) out.
template <class R>
__device__ __forceinline__ void parabola(R qs, R ql, R qr, R &oL, R &oR, R &d, R &q6)
{
    if ((qr - qs) * (qs - ql) <= (R)0) {
        ql = qs;
        qr = qs;
    } else {
        const R dd = qr - ql;
        const R qq6 = (R)6 * (qs - (R)0.5 * (ql + qr));
        if (dd * qq6 > dd * dd) ql = (R)3 * qs - (R)2 * qr;
        else if (-(dd * dd) > dd * qq6) qr = (R)3 * qs - (R)2 * ql;
    }
    oL = ql;
    oR = qr;
    d = qr - ql;
    q6 = (R)6 * (qs - (R)0.5 * (ql + qr));
}

// Averages of the zone parabola over the fraction sig of the zone adjacent to
// its right / left edge (CW84 1.12).
template <class R>
__device__ __forceinline__ R avg_right(R qR, R d, R q6, R sig)
{
    return qR - ((R)0.5 * sig) * (d - ((R)1 - sig * (R)(2.0 / 3.0)) * q6);
}
template <class R>
__device__ __forceinline__ R avg_left(R qL, R d, R q6, R sig)
{
    return qL + ((R)0.5 * sig) * (d + ((R)1 - sig * (R)(2.0 / 3.0)) * q6);
}

// Characteristic state at one edge of a zone (CW84 3.6/3.7, Sec. 4.1).
// SIDE = +1: left state of the interface at the zone's right edge (waves with
// lambda > 0 reach it); SIDE = -1: right state at the zone's left edge.
// Wave order: 0 = u-c, 1 = u, 2 = u+c.  The reference state is the fastest wave
// moving toward the edge (u+c or u-c) averaged over its domain, else the edge
// value; the others enter through beta corrections of the linearised
// Lagrangian characteristic relations dp +- C du = 0, dp + C^2 d(1/rho) = 0.
template <class R, int SIDE>
__device__ __forceinline__ void trace_exact(const R qL[5], const R qR[5], const R d[5], const R q6[5],
                                            R u, R c, R dtdx, const Consts<R> &k, R out[5])
{
    const R lam0 = u - c, lam1 = u, lam2 = u + c;
    const bool r0 = SIDE > 0 ? lam0 > (R)0 : lam0 < (R)0;
    const bool r1 = SIDE > 0 ? lam1 > (R)0 : lam1 < (R)0;
    const bool r2 = SIDE > 0 ? lam2 > (R)0 : lam2 < (R)0;
    const R s0 = SIDE > 0 ? lam0 * dtdx : -lam0 * dtdx;
    const R s1 = SIDE > 0 ? lam1 * dtdx : -lam1 * dtdx;
    const R s2 = SIDE > 0 ? lam2 * dtdx : -lam2 * dtdx;
#define ENZO_I(SIG, V) (SIDE > 0 ? avg_right<R>(qR[V], d[V], q6[V], SIG) : avg_left<R>(qL[V], d[V], q6[V], SIG))
    const bool rref = SIDE > 0 ? r2 : r0;
    const R sref = SIDE > 0 ? s2 : s0;
    const R *edge = SIDE > 0 ? qR : qL;
    R rho_ref, u_ref, p_ref;
    if (rref) {
        rho_ref = ENZO_I(sref, 0);
        u_ref = ENZO_I(sref, 1);
        p_ref = ENZO_I(sref, 2);
    } else {
        rho_ref = edge[0];
        u_ref = edge[1];
        p_ref = edge[2];
    }
    if (!(rho_ref > k.rho_floor)) rho_ref = k.rho_floor;
    if (!(p_ref > k.p_floor)) p_ref = k.p_floor;
    const R C = sqrt(k.gamma * p_ref * rho_ref);
    R bp = (R)0, bm = (R)0, b0 = (R)0;
    if (r2) bp = -((R)0.5 / C) * ((u_ref - ENZO_I(s2, 1)) + (p_ref - ENZO_I(s2, 2)) / C);
    if (r0) bm = ((R)0.5 / C) * ((u_ref - ENZO_I(s0, 1)) - (p_ref - ENZO_I(s0, 2)) / C);
    if (r1) b0 = (p_ref - ENZO_I(s1, 2)) / (C * C) + (R)1 / rho_ref - (R)1 / ENZO_I(s1, 0);
    R p = p_ref + (C * C) * (bp + bm);
    const R un = u_ref + C * (bp - bm);
    const R tau = (R)1 / rho_ref - ((bp + bm) + b0);
    R rho = (R)1 / tau;
    if (!(rho > k.rho_floor)) rho = k.rho_floor;
    if (!(p > k.p_floor)) p = k.p_floor;
    out[0] = rho;
    out[1] = un;
    out[2] = p;
    out[3] = r1 ? ENZO_I(s1, 3) : edge[3];
    out[4] = r1 ? ENZO_I(s1, 4) : edge[4];
#undef ENZO_I
}

// The same characteristic state in FP32, arranged for fewer operations (the
// FP32 path is bound by instruction issue).  Written for SIDE = +1 with
// sg = +1, and mirrored through sg = -1:
//   * a wave's domain fraction is sigma = max(sg lambda dt/dx, 0), so a wave
//     moving away from the edge averages to the edge value itself;
//   * the reference is the average over the fastest wave toward the edge
//     (u + sg c), so that wave's own beta, which measures the difference of
//     the reference and its own average, vanishes identically and is not
//     formed; the slow acoustic wave (u - sg c) and the entropy wave (u)
//     give beta_s = sg (1/2C) [(u_ref - I_s(u)) - sg (p_ref - I_s(p)) / C]
//     and beta_0 = (p_ref - I_0(p)) / C^2 + 1/rho_ref - 1/I_0(rho), each only
//     where its wave reaches the edge;
//   * p = p_ref + C^2 beta_s, u = u_ref - sg C beta_s,
//     1/rho = 1/rho_ref - (beta_s + beta_0), with 1/C from one reciprocal
//     square root of C^2 = gamma p_ref rho_ref.
template <int SIDE>
__device__ __forceinline__ void trace_f(const float qL[5], const float qR[5], const float d[5],
                                        const float q6[5], float u, float c, float dtdx,
                                        const Consts<float> &k, float out[5])
{
    constexpr float sg = SIDE > 0 ? 1.0f : -1.0f;
    const float *edge = SIDE > 0 ? qR : qL;
    const float sdt = sg * dtdx;
    const float sf = fmaxf((u + sg * c) * sdt, 0.0f);   // fastest wave toward the edge
    const float s0 = fmaxf(u * sdt, 0.0f);              // entropy wave
    const float ss = fmaxf((u - sg * c) * sdt, 0.0f);   // slow acoustic wave
    // average over a fraction s next to the edge: edge - sg (s/2) (d - sg (1 - 2s/3) q6)
    const float af = -sg * 0.5f * sf, bf = -sg * fmaf(-2.0f / 3.0f, sf, 1.0f);
    const float a0 = -sg * 0.5f * s0, b0c = -sg * fmaf(-2.0f / 3.0f, s0, 1.0f);
    const float as = -sg * 0.5f * ss, bs = -sg * fmaf(-2.0f / 3.0f, ss, 1.0f);
#define ENZO_AVG(A, B, V) fmaf((A), fmaf((B), q6[V], d[V]), edge[V])
    float rho_ref = ENZO_AVG(af, bf, 0);
    const float u_ref = ENZO_AVG(af, bf, 1);
    float p_ref = ENZO_AVG(af, bf, 2);
    rho_ref = rho_ref > k.rho_floor ? rho_ref : k.rho_floor;
    p_ref = p_ref > k.p_floor ? p_ref : k.p_floor;
    const float C2 = k.gamma * p_ref * rho_ref;
    const float iC = rsqrtf(C2);
    const float C = C2 * iC;
    const float irho = 1.0f / rho_ref;
    float bsl = 0.0f, b0 = 0.0f;
    if (ss > 0.0f) {
        const float du = u_ref - ENZO_AVG(as, bs, 1), dp = p_ref - ENZO_AVG(as, bs, 2);
        bsl = (sg * 0.5f * iC) * fmaf(-sg * dp, iC, du);
    }
    if (s0 > 0.0f) {
        const float dp = p_ref - ENZO_AVG(a0, b0c, 2);
        b0 = fmaf(dp, iC * iC, irho) - 1.0f / ENZO_AVG(a0, b0c, 0);
    }
    float p = fmaf(C2, bsl, p_ref);
    const float un = fmaf(-sg * C, bsl, u_ref);
    float rho = 1.0f / (irho - (bsl + b0));
    out[0] = rho > k.rho_floor ? rho : k.rho_floor;
    out[1] = un;
    out[2] = p > k.p_floor ? p : k.p_floor;
    out[3] = ENZO_AVG(a0, b0c, 3);
    out[4] = ENZO_AVG(a0, b0c, 4);
#undef ENZO_AVG
}

template <class R, int SIDE>
__device__ __forceinline__ void trace(const R qL[5], const R qR[5], const R d[5], const R q6[5],
                                      R u, R c, R dtdx, const Consts<R> &k, R out[5])
{
    if constexpr (std::is_same<R, float>::value) trace_f<SIDE>(qL, qR, d, q6, u, c, dtdx, k, out);
    else trace_exact<R, SIDE>(qL, qR, d, q6, u, c, dtdx, k, out);
}

// A passive variable (eps of the dual-energy option) traced to one edge of its
// zone as trace() takes the transverse velocities: the average over the domain
// of the u wave where that wave reaches the edge, else the edge value.
template <class R, int SIDE>
__device__ __forceinline__ R trace_passive(R qL, R qR, R d, R q6, R u, R dtdx)
{
    const bool r1 = SIDE > 0 ? u > (R)0 : u < (R)0;
    const R s1 = SIDE > 0 ? u * dtdx : -u * dtdx;
    if (!r1) return SIDE > 0 ? qR : qL;
    return SIDE > 0 ? avg_right<R>(qR, d, q6, s1) : avg_left<R>(qL, d, q6, s1);
}

// Lagrangian shock speed W and |dp/du| of the shock curve Z = 2W^3/(W^2+C^2).
template <class R>
__device__ __forceinline__ void shock_side(R ps, R p, R C, const Consts<R> &k, R &W, R &Z)
{
    R rad = (R)1 + k.gp1o2g * (ps / p - (R)1);
    if (rad < (R)1e-6) rad = (R)1e-6;
    W = C * sqrt(rad);
    Z = (R)2 * W * W * W / (W * W + C * C);
}

template <class R>
__device__ __forceinline__ R plain_guess(R rl, R ul, R pl, R rr, R ur, R pr, const Consts<R> &k)
{
    const R CL = sqrt(k.gamma * pl * rl);
    const R CR = sqrt(k.gamma * pr * rr);
    const R p0 = (CR * pl + CL * pr + CL * CR * (ul - ur)) / (CL + CR);
    return p0 > k.p_floor ? p0 : k.p_floor;
}

// Newton iteration on f(p*) = u*_R - u*_L = 0 (two-shock, Sec. 4.1.2).  Stops
// when |f| <= tol (|u_L| + |u_R| + c_L + c_R), when the update no longer moves
// p*, or (FP32 only) when the update is below a few ulp of p*.
template <class R>
__device__ __forceinline__ int newton(R rl, R ul, R pl, R rr, R ur, R pr, R p0,
                                      const Consts<R> &k, R &pstar, bool &conv)
{
    const R CL = sqrt(k.gamma * pl * rl);
    const R CR = sqrt(k.gamma * pr * rr);
    const R uscale = (fabs(ul) + fabs(ur)) + (sqrt(k.gamma * pl / rl) + sqrt(k.gamma * pr / rr));
    R ps = p0 > k.p_floor ? p0 : k.p_floor;
    conv = false;
    int it;
    for (it = 0; it < k.nmax; ++it) {
        R WL, ZL, WR, ZR;
        shock_side(ps, pl, CL, k, WL, ZL);
        shock_side(ps, pr, CR, k, WR, ZR);
        const R usL = ul - (ps - pl) / WL;
        const R usR = ur + (ps - pr) / WR;
        const R f = usR - usL;
        if (fabs(f) <= k.tol * uscale) { conv = true; break; }
        R pn = ps - ZL * ZR * f / (ZL + ZR);
        if (!(pn > k.p_floor)) pn = k.p_floor;
        if (pn == ps) { conv = true; break; }
        if (sizeof(R) == 4 && fabs(pn - ps) <= k.step_tol * pn) { ps = pn; conv = true; ++it; break; }
        ps = pn;
    }
    pstar = ps;
    return it;
}

template <class R>
struct RiemannOut {
    R rho, u, p, ustar, pstar;
    int iters;
    bool conv;
};

// FP32 two-shock solve (Sec. 4.1.2): the method of riemann_exact below,
// arranged for the FP32 pipe.  With rad_s = 1 + (gamma+1)/(2 gamma)(p*/p_s - 1)
// and r_s = rad_s^{-1/2}: W_s = C_s sqrt(rad_s), so 1/W_s = r_s / C_s, and
// Z_s = 2 W_s^3 / (W_s^2 + C_s^2) = 2 C_s rad_s^{3/2} / (1 + rad_s), so
// 1/Z_s = (r_s / (2 C_s)) (1 + r_s^2).  One reciprocal square root per side
// and iteration therefore gives the star velocities u*_L = u_L - (p* - p_L)/W_L,
// u*_R = u_R + (p* - p_R)/W_R and the Newton step f / (1/Z_L + 1/Z_R), and
// u* = (Z_L u*_L + Z_R u*_R)/(Z_L + Z_R) = (u*_L/Z_R + u*_R/Z_L)/(1/Z_L + 1/Z_R).
// The loop keeps the side quantities of the iterate it accepts, so the star
// state needs no second evaluation: it stops when |f| meets the tolerance, or
// when the next step is below step_tol p* (the iterate is then within that
// step of the root).  A learned start that reaches the iteration cap restarts
// once from the plain guess inside the same loop.  The upwind side alone is
// sampled.
__device__ __forceinline__ RiemannOut<float> riemann_f(float rl, float ul, float pl, float rr, float ur, float pr,
                                                      float pguess, const Consts<float> &k, Counters &cnt)
{
    const float C2L = k.gamma * pl * rl, C2R = k.gamma * pr * rr;
    const float iCL = rsqrtf(C2L), iCR = rsqrtf(C2R);
    const float ipl = 1.0f / pl, ipr = 1.0f / pr;
    float plain, ftol;
    {
        const float CL = C2L * iCL, CR = C2R * iCR;
        // |u*_R - u*_L| <= tol (|u_L| + |u_R| + c_L + c_R), c = C / rho
        ftol = k.tol * ((fabsf(ul) + fabsf(ur)) + (CL / rl + CR / rr));
        plain = (CR * pl + CL * pr + CL * CR * (ul - ur)) / (CL + CR);
        plain = plain > k.p_floor ? plain : k.p_floor;
    }
    float ps = pguess > 0.0f ? (pguess > k.p_floor ? pguess : k.p_floor) : plain;
    float rsL, rsR, usL, usR, izL, izR;
    int it = 0, lim = k.nmax;
    bool conv = false, restarted = pguess <= 0.0f;
#if ENZO_NEWTON_HEAD > 0
    // the first ENZO_NEWTON_HEAD evaluations as straight-line code: each lane
    // keeps its accepted iterate once it has converged, so the steps after
    // that re-evaluate the same p* and change nothing
#pragma unroll
    for (int h = 0; h < ENZO_NEWTON_HEAD; ++h) {
        const float radL = fmaxf(fmaf(k.gp1o2g, fmaf(ps, ipl, -1.0f), 1.0f), 1e-6f);
        const float radR = fmaxf(fmaf(k.gp1o2g, fmaf(ps, ipr, -1.0f), 1.0f), 1e-6f);
        rsL = rsqrtf(radL);
        rsR = rsqrtf(radR);
        const float iWL = rsL * iCL, iWR = rsR * iCR;
        usL = fmaf(pl - ps, iWL, ul);
        usR = fmaf(ps - pr, iWR, ur);
        izL = iWL * fmaf(0.5f * rsL, rsL, 0.5f);
        izR = iWR * fmaf(0.5f * rsR, rsR, 0.5f);
        const float f = usR - usL;
        float pn = ps - f / (izL + izR);
        pn = pn > k.p_floor ? pn : k.p_floor;
        const bool fconv = fabsf(f) <= ftol;
        const bool sconv = fabsf(pn - ps) <= k.step_tol * pn;
        if (!conv) {
            if (fconv) conv = true;
            else {
                ++it;
                if (sconv) conv = true;
                else ps = pn;
            }
        }
    }
    if (!conv)
#endif
    for (;;) {
        if (it >= lim) {
            // a learned start that does not converge restarts once from the plain guess
            if (restarted) break;
            restarted = true;
            cnt.restarts++;
            ps = plain;
            lim += k.nmax;
        }
        const float radL = fmaxf(fmaf(k.gp1o2g, fmaf(ps, ipl, -1.0f), 1.0f), 1e-6f);
        const float radR = fmaxf(fmaf(k.gp1o2g, fmaf(ps, ipr, -1.0f), 1.0f), 1e-6f);
        rsL = rsqrtf(radL);
        rsR = rsqrtf(radR);
        const float iWL = rsL * iCL, iWR = rsR * iCR;
        usL = fmaf(pl - ps, iWL, ul);
        usR = fmaf(ps - pr, iWR, ur);
        izL = iWL * fmaf(0.5f * rsL, rsL, 0.5f);
        izR = iWR * fmaf(0.5f * rsR, rsR, 0.5f);
        const float f = usR - usL;
        if (fabsf(f) <= ftol) { conv = true; break; }
        float pn = ps - f / (izL + izR);
        pn = pn > k.p_floor ? pn : k.p_floor;
        ++it;
        if (fabsf(pn - ps) <= k.step_tol * pn) { conv = true; break; }
        ps = pn;
    }
    RiemannOut<float> o;
    o.iters = it;
    o.conv = conv;
    const float us = (usL * izR + usR * izL) / (izL + izR);
    o.ustar = us;
    o.pstar = ps;
    // sample x/t = 0 on the side upwind of the contact: sg = +1 left, -1 right;
    // w is the weight of the star state (0 outside the wave, 1 inside, linear in
    // the head/tail speed fraction across a transonic rarefaction)
    const bool left = us >= 0.0f;
    const float sg = left ? 1.0f : -1.0f;
    const float r_s = left ? rl : rr, u_s = left ? ul : ur, p_s = left ? pl : pr;
    const float iW = left ? rsL * iCL : rsR * iCR;              // 1 / W
    const float ir_s = 1.0f / r_s;
    float rs_st = 1.0f / fmaf(p_s - ps, iW * iW, ir_s);          // 1/rho* = 1/rho - (p* - p)/W^2
    rs_st = rs_st > k.rho_floor ? rs_st : k.rho_floor;
    const float Sshock = u_s - sg * ir_s / iW;                   // shock speed u -+ W / rho
    const float c_s = sqrtf(k.gamma * p_s * ir_s);
    const float c_st = sqrtf(k.gamma * ps / rs_st);
    const float Sh = u_s - sg * c_s;
    const float St = us - sg * c_st;
    const float fr = -Sh / (St - Sh);
    const float w_rare = sg * Sh >= 0.0f ? 0.0f : (sg * St <= 0.0f ? 1.0f : fr);
    const float w_shock = sg * Sshock >= 0.0f ? 0.0f : 1.0f;
    const float w = ps > p_s ? w_shock : w_rare;
    o.rho = fmaf(w, rs_st - r_s, r_s);
    o.u = fmaf(w, us - u_s, u_s);
    o.p = fmaf(w, ps - p_s, p_s);
    return o;
}

// Two-shock solve and sampling of the self-similar solution at x/t = 0.
template <class R>
__device__ __forceinline__ RiemannOut<R> riemann_exact(R rl, R ul, R pl, R rr, R ur, R pr, R pguess,
                                                       const Consts<R> &k, Counters &cnt)
{
    RiemannOut<R> o;
    R ps;
    bool conv;
    int it;
    if (pguess > (R)0) {
        it = newton(rl, ul, pl, rr, ur, pr, pguess, k, ps, conv);
        if (!conv) {
            cnt.restarts++;
            it += newton(rl, ul, pl, rr, ur, pr, plain_guess(rl, ul, pl, rr, ur, pr, k), k, ps, conv);
        }
    } else {
        it = newton(rl, ul, pl, rr, ur, pr, plain_guess(rl, ul, pl, rr, ur, pr, k), k, ps, conv);
    }
    o.iters = it;
    o.conv = conv;
    const R CL = sqrt(k.gamma * pl * rl);
    const R CR = sqrt(k.gamma * pr * rr);
    R WL, ZL, WR, ZR;
    shock_side(ps, pl, CL, k, WL, ZL);
    shock_side(ps, pr, CR, k, WR, ZR);
    const R usL = ul - (ps - pl) / WL;
    const R usR = ur + (ps - pr) / WR;
    const R us = (ZL * usL + ZR * usR) / (ZL + ZR);
    R rsL = (R)1 / ((R)1 / rl - (ps - pl) / (WL * WL));
    R rsR = (R)1 / ((R)1 / rr - (ps - pr) / (WR * WR));
    if (!(rsL > k.rho_floor)) rsL = k.rho_floor;
    if (!(rsR > k.rho_floor)) rsR = k.rho_floor;
    o.ustar = us;
    o.pstar = ps;
    R rho, u, p;
    if (us >= (R)0) {
        if (ps > pl) {
            const R S = ul - WL / rl;
            if (S >= (R)0) { rho = rl; u = ul; p = pl; }
            else { rho = rsL; u = us; p = ps; }
        } else {
            const R cl = sqrt(k.gamma * pl / rl);
            const R cs = sqrt(k.gamma * ps / rsL);
            const R Sh = ul - cl;
            const R St = us - cs;
            if (Sh >= (R)0) { rho = rl; u = ul; p = pl; }
            else if (St <= (R)0) { rho = rsL; u = us; p = ps; }
            else {
                const R f = -Sh / (St - Sh);
                rho = rl + f * (rsL - rl);
                u = ul + f * (us - ul);
                p = pl + f * (ps - pl);
            }
        }
    } else {
        if (ps > pr) {
            const R S = ur + WR / rr;
            if (S <= (R)0) { rho = rr; u = ur; p = pr; }
            else { rho = rsR; u = us; p = ps; }
        } else {
            const R cr = sqrt(k.gamma * pr / rr);
            const R cs = sqrt(k.gamma * ps / rsR);
            const R Sh = ur + cr;
            const R St = us + cs;
            if (Sh <= (R)0) { rho = rr; u = ur; p = pr; }
            else if (St >= (R)0) { rho = rsR; u = us; p = ps; }
            else {
                const R f = Sh / (Sh - St);
                rho = rr + f * (rsR - rr);
                u = ur + f * (us - ur);
                p = pr + f * (ps - pr);
            }
        }
    }
    o.rho = rho;
    o.u = u;
    o.p = p;
    return o;
}

template <class R>
__device__ __forceinline__ RiemannOut<R> riemann(R rl, R ul, R pl, R rr, R ur, R pr, R pguess,
                                                 const Consts<R> &k, Counters &cnt)
{
    if constexpr (std::is_same<R, float>::value) return riemann_f(rl, ul, pl, rr, ur, pr, pguess, k, cnt);
    else return riemann_exact<R>(rl, ul, pl, rr, ur, pr, pguess, k, cnt);
}

// Physical flux of the split 1-D equations (Sec. 4.1): mass, normal momentum,
// transverse momenta, total energy.
template <class R>
__device__ __forceinline__ void phys_flux(R rho, R u, R p, R t1, R t2, const Consts<R> &k, R F[5])
{
    const R mflux = rho * u;
    F[0] = mflux;
    F[1] = mflux * u + p;
    F[2] = mflux * t1;
    F[3] = mflux * t2;
    const R eint = p * k.gm1inv;
    const R ke = (R)0.5 * rho * ((u * u + t1 * t1) + t2 * t2);
    F[4] = u * ((eint + ke) + p);
}

// HLL flux with Davis wave-speed bounds from first-order zone states (fallback).
template <class R>
__device__ __forceinline__ void hll_flux(const Zone<R> &L, const Zone<R> &Rz, const Consts<R> &k,
                                         R F[5])
{
    const R cl = sqrt(k.gamma * L.p / L.r), cr = sqrt(k.gamma * Rz.p / Rz.r);
    const R SL = L.u - cl < Rz.u - cr ? L.u - cl : Rz.u - cr;
    const R SR = L.u + cl > Rz.u + cr ? L.u + cl : Rz.u + cr;
    R FL[5], FR[5];
    phys_flux(L.r, L.u, L.p, L.t1, L.t2, k, FL);
    phys_flux(Rz.r, Rz.u, Rz.p, Rz.t1, Rz.t2, k, FR);
    if (SL >= (R)0) {
        _Pragma("unroll") for (int c = 0; c < 5; ++c) F[c] = FL[c];
        return;
    }
    if (SR <= (R)0) {
        _Pragma("unroll") for (int c = 0; c < 5; ++c) F[c] = FR[c];
        return;
    }
    const R UL[5] = {L.r, L.r * L.u, L.r * L.t1, L.r * L.t2,
                     L.p * k.gm1inv + (R)0.5 * L.r * ((L.u * L.u + L.t1 * L.t1) + L.t2 * L.t2)};
    const R UR[5] = {Rz.r, Rz.r * Rz.u, Rz.r * Rz.t1, Rz.r * Rz.t2,
                     Rz.p * k.gm1inv + (R)0.5 * Rz.r * ((Rz.u * Rz.u + Rz.t1 * Rz.t1) + Rz.t2 * Rz.t2)};
    _Pragma("unroll") for (int c = 0; c < 5; ++c)
        F[c] = (SR * FL[c] - SL * FR[c] + SL * SR * (UR[c] - UL[c])) / (SR - SL);
}

// HLL flux of two primitive states (r, u, p, t1, t2) as the interface flux
// (the approximate solver of Sec. 4.1.2 used on the traced states).
template <class R>
__device__ __forceinline__ void hll_states(const R l[5], const R r[5], const Consts<R> &k, R F[5])
{
    const Zone<R> zl{l[0], l[1], l[2], l[3], l[4], (R)0}, zr{r[0], r[1], r[2], r[3], r[4], (R)0};
    hll_flux<R>(zl, zr, k, F);
}

// HLLC flux of two primitive states: the Davis bounds SL, SR of hll_flux, the
// contact speed S* = (pR - pL + rL uL (SL - uL) - rR uR (SR - uR)) /
// (rL (SL - uL) - rR (SR - uR)), and on the upwind side of the contact the star
// state rK (SK - uK)/(SK - S*) [1, S*, t1K, t2K, EK/rK + (S* - uK)(S* + pK/(rK (SK - uK)))]
// with flux FK + SK (U*K - UK) (Sec. 4.1.2 names HLLC; Toro's three-wave form).
template <class R>
__device__ __forceinline__ void hllc_states(const R l[5], const R r[5], const Consts<R> &k, R F[5])
{
    const R rl = l[0], ul = l[1], pl = l[2], rr = r[0], ur = r[1], pr = r[2];
    const R cl = sqrt(k.gamma * pl / rl), cr = sqrt(k.gamma * pr / rr);
    const R SL = ul - cl < ur - cr ? ul - cl : ur - cr;
    const R SR = ul + cl > ur + cr ? ul + cl : ur + cr;
    R FL[5], FR[5];
    phys_flux(rl, ul, pl, l[3], l[4], k, FL);
    phys_flux(rr, ur, pr, r[3], r[4], k, FR);
    if (SL >= (R)0) {
        _Pragma("unroll") for (int c = 0; c < 5; ++c) F[c] = FL[c];
        return;
    }
    if (SR <= (R)0) {
        _Pragma("unroll") for (int c = 0; c < 5; ++c) F[c] = FR[c];
        return;
    }
    const R ml = rl * (SL - ul), mr = rr * (SR - ur);
    const R Ss = ((pr - pl) + ul * ml - ur * mr) / (ml - mr);
    const bool left = Ss >= (R)0;
    const R rk = left ? rl : rr, uk = left ? ul : ur, pk = left ? pl : pr;
    const R t1 = left ? l[3] : r[3], t2 = left ? l[4] : r[4], S = left ? SL : SR, m = left ? ml : mr;
    const R E = pk * k.gm1inv + (R)0.5 * rk * ((uk * uk + t1 * t1) + t2 * t2);
    const R UK[5] = {rk, rk * uk, rk * t1, rk * t2, E};
    const R chi = m / (S - Ss);
    const R Us[5] = {chi, chi * Ss, chi * t1, chi * t2, chi * (E / rk + (Ss - uk) * (Ss + pk / m))};
    _Pragma("unroll") for (int c = 0; c < 5; ++c) F[c] = (left ? FL[c] : FR[c]) + S * (Us[c] - UK[c]);
}

// Pencil addressing: storage index of pencil position s (0 .. L-1).
struct Pencil {
    int64_t base, sd;
    int L, ng, n;
    __device__ __forceinline__ int64_t at(int s) const { return base + (int64_t)s * sd; }
};

// Face contribution to the FP64 conservative update.  FP64 path: the flux
// itself (the update is U + dt/dx (F_m - F_p), as in the oracle).  FP32 path:
// G = dt/dx * F rounded once in FP32 and widened exactly to FP64; a cell then
// gets (U + G_m) - G_p in FP64, so each face's contribution enters its two
// cells with opposite signs exactly and the totals change only by FP64 rounding.
template <class R>
struct Face {
    double g[5];
};

__device__ __forceinline__ double cell_update(double U, double dtdx64, double Fm, double Fp)
{
    return U + dtdx64 * (Fm - Fp);
}

// Starting guess for Newton: the plain acoustic guess (inside riemann()).
struct PlainGuess {
    static constexpr int kDepth = 0;   // the guess of an interface is known at once
    template <class R>
    __device__ __forceinline__ R operator()(R, R, R, R, R, R) { return (R)-1; }
};

// Learned guess evaluated on the tensor cores for the 128 interfaces the CTA's
// pencils reach at the same march step (one per thread = one MMA row).
// Operands, as the sweep keeps them: both layers' weights pre-scaled by 1/2 (so
// the accumulators hold h = z/2, the argument SiLU needs) and both biases folded
// into the products through an input column held at 1 (column 6 of the 16
// feature columns; column 64 of the 80 activation columns).  (Adding layer 2's
// bias in FP16 before the SiLU instead, with K = 64, measured slower.)
// No-swizzle K-major tiles need 16-byte alignment; 128 is kept.
struct alignas(128) GuessSmem {
    unsigned char w1[64 * 16 * 2];   // B of layer 1: 64 units x 16 inputs
    unsigned char w2[64 * 80 * 2];   // B of layer 2: 64 units x (64 + 16) inputs
    unsigned char a1[128 * 16 * 2];  // A of layer 1: features
    unsigned char a2[128 * 80 * 2];  // A of layer 2: layer-1 activations
    float4 ring[2][128][3];          // per thread: traced states (sL, sR) of two march steps
    __half2 w3h[32];                 // output unit weights as FP16 pairs (w3_2i, w3_2i+1)
    float b3;
    int err;
    uint64_t mbar;
    uint32_t tmem;
};

// SiLU of two accumulator values in FP16 (h = z/2; z sigmoid(z) = h + h tanh(h)),
// then their terms of the output unit's dot product added into acc.
__device__ __forceinline__ __half2 silu_dot_f16x2(float h0, float h1, __half2 w, __half2 acc)
{
    const __half2 h = __floats2half2_rn(h0, h1);
    uint32_t tb;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(tb) : "r"(*reinterpret_cast<const uint32_t *>(&h)));
    const __half2 sl = __hfma2(h, *reinterpret_cast<const __half2 *>(&tb), h);
    return __hfma2(w, sl, acc);
}

// SiLU of two accumulator values holding h = z/2: z sigmoid(z) = h + h tanh(h).
__device__ __forceinline__ uint32_t silu_half_bf16x2(float h0, float h1)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(h0, h1);
    const uint32_t hb = *reinterpret_cast<const uint32_t *>(&h);
    uint32_t tb;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(tb) : "r"(hb));
    const __nv_bfloat162 o = __hfma2(h, *reinterpret_cast<const __nv_bfloat162 *>(&tb), h);
    return *reinterpret_cast<const uint32_t *>(&o);
}

__device__ __forceinline__ unsigned short bf16_half_bits(unsigned short b)
{
    const float f = __bfloat162float(__ushort_as_bfloat16(b)) * 0.5f;
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// Software-pipelined evaluation: each call of pipe() takes the states of the
// CTA's newest interfaces and returns the guesses of the interfaces of two calls
// back.  In one call the threads (i) wait for the products issued by the
// previous call, (ii) finish layer 2 of the interface two calls back (SiLU and
// the output unit), (iii) finish layer 1 of the interface one call back (SiLU
// into the layer-2 operand), (iv) write the new features; one barrier (which
// also votes whether any new interface passes the gate); then one thread issues
// layer 1 of the new interfaces and layer 2 of the previous ones.  The products
// run while the threads do the next march step's reconstruction, so no call
// waits on the tensor core in the steady state.
struct LearnedGuess {
    static constexpr int kDepth = 2;
    GuessSmem *S;
    uint32_t phase;
    bool ok;
    bool committed;      // products issued by the previous call (CTA-uniform)
    bool any1, any2;     // layer 1 / layer 2 in flight for the interfaces 1 / 2 calls back
    bool need1, need2;   // this thread's interface 1 / 2 calls back passed the gate
    float s1, s2;        // log2 sqrt(pL pR) of those interfaces
    float gamma, rsqg;   // gamma and 1/sqrt(gamma)
    float gate, gate2g;  // jump-strength gate (< 0: always) and gate^2 gamma

    __device__ void setup(unsigned char *raw, const void *blob, float g, double gate_)
    {
        S = reinterpret_cast<GuessSmem *>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
        const unsigned char *b = static_cast<const unsigned char *>(blob);
        const float *bvec = reinterpret_cast<const float *>(b + kBlobF32);   // b1, b2, w3, b3
        // layer 1: inputs 0..5 from the blob (already 16-column tiles), column 6 = b1
        for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
            const int n = i >> 4, k = i & 15;
            const uint32_t off = tc::tile_off(n, k, 16);
            unsigned short v;
            if (k == 6) v = __bfloat16_as_ushort(__float2bfloat16_rn(0.5f * bvec[n]));
            else v = bf16_half_bits(*reinterpret_cast<const unsigned short *>(b + kBlobW1 + off));
            *reinterpret_cast<unsigned short *>(S->w1 + off) = v;
        }
        // layer 2: 64 input columns re-tiled from K = 64 to K = 80, column 64 = b2
        for (int i = threadIdx.x; i < 64 * 80; i += blockDim.x) {
            const int n = i / 80, k = i - 80 * (i / 80);
            unsigned short v = 0;
            if (k < 64) v = bf16_half_bits(*reinterpret_cast<const unsigned short *>(b + kBlobW2 + tc::tile_off(n, k, 64)));
            else if (k == 64) v = __bfloat16_as_ushort(__float2bfloat16_rn(0.5f * bvec[64 + n]));
            *reinterpret_cast<unsigned short *>(S->w2 + tc::tile_off(n, k, 80)) = v;
        }
        // constant columns 64..79 of the activations: 1, 0, ..., 0
        for (int i = threadIdx.x; i < 128 * 16; i += blockDim.x) {
            const int r = i >> 4, k = 64 + (i & 15);
            *reinterpret_cast<unsigned short *>(S->a2 + tc::tile_off(r, k, 80)) = k == 64 ? 0x3F80u : 0u;
        }
        for (int i = threadIdx.x; i < 32; i += blockDim.x) S->w3h[i] = __floats2half2_rn(bvec[128 + 2 * i], bvec[129 + 2 * i]);
        if (threadIdx.x == 0) {
            S->b3 = bvec[192];
            S->err = 0;
            tc::mbar_init(&S->mbar, 1);
        }
        if (threadIdx.x < 32) tc::tmem_alloc(&S->tmem, 128);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        phase = 0;
        ok = true;
        committed = any1 = any2 = need1 = need2 = false;
        s1 = s2 = 0.0f;
        gamma = g;
        rsqg = rsqrtf(g);
        gate = (float)gate_;
        gate2g = gate * gate * g;
    }

    __device__ void teardown()
    {
        // products still in flight (only after a failed wait: pencils drain
        // the pipeline) get one more bounded wait before TMEM is released
        if (committed) tc::mbar_wait(&S->mbar, phase);
        tc::fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tc::tmem_dealloc(S->tmem, 128);
    }

    // Every thread of the CTA calls this at the same march step; valid: this
    // thread has a new interface.  Returns the learned p* of its interface of
    // two calls back, or -1 (plain guess: below the gate, none, or failure).
    __device__ float pipe(bool valid, float rl, float ul, float pl, float rr, float ur, float pr)
    {
        if (!ok) return -1.0f;
        const int row = threadIdx.x;
        const uint32_t lane = (uint32_t)((row & ~31) << 16);
        bool timeout = false;
        if (committed) {
            timeout = !tc::mbar_wait(&S->mbar, phase);
            phase ^= 1u;
            tc::fence_after();
        }
        float p0 = -1.0f;
        if (any2) {
            // output unit of the interface two calls back: SiLU and the dot
            // product in packed FP16, one partial sum per 16 units, summed in FP32
            float y = S->b3;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[16];
                tc::tmem_ld16(S->tmem + lane + 64 + c * 16, v);
                __half2 acc = __float2half2_rn(0.0f);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc = silu_dot_f16x2(v[2 * i], v[2 * i + 1], S->w3h[c * 8 + i], acc);
                const float2 a = __half22float2(acc);
                y += a.x + a.y;
            }

            if (need2) p0 = exp2f(fmaf(y, 1.44269504f, s2));   // sqrt(p_L p_R) e^y
        }
        if (any1) {
            // layer-1 activations of the interface one call back
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[16];
                tc::tmem_ld16(S->tmem + lane + c * 16, v);
                uint4 lo, hi;
                lo.x = silu_half_bf16x2(v[0], v[1]);
                lo.y = silu_half_bf16x2(v[2], v[3]);
                lo.z = silu_half_bf16x2(v[4], v[5]);
                lo.w = silu_half_bf16x2(v[6], v[7]);
                hi.x = silu_half_bf16x2(v[8], v[9]);
                hi.y = silu_half_bf16x2(v[10], v[11]);
                hi.z = silu_half_bf16x2(v[12], v[13]);
                hi.w = silu_half_bf16x2(v[14], v[15]);
                *reinterpret_cast<uint4 *>(S->a2 + tc::tile_off(row, c * 16, 80)) = lo;
                *reinterpret_cast<uint4 *>(S->a2 + tc::tile_off(row, c * 16 + 8, 80)) = hi;
            }
        }
        // features of the new interface (column 6 carries the bias)
        const float psum = pl + pr, du = ul - ur;
        const bool need = valid && (gate < 0.0f || fabsf(pl - pr) > gate * psum || du * du * (rl + rr) > gate2g * psum);
        // the features of mlp_features from four base-2 logarithms: with
        // l = log2 of rho_L, rho_R, p_L, p_R, ln(rho_L/rho_ref) = (ln 2 / 2)(l_rL - l_rR),
        // ln(p_L/p_ref) likewise, and 1/c_ref = 2^(-(l_pL + l_pR - l_rL - l_rR)/4) / sqrt(gamma)
        float x[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float lgp = 0.0f;                       // log2 sqrt(p_L p_R)
        if (need) {
            const float lrl = __log2f(rl), lrr = __log2f(rr), lpl = __log2f(pl), lpr = __log2f(pr);
            constexpr float hln2 = 0.34657359f;   // ln 2 / 2
            const float a = hln2 * (lrl - lrr), b = hln2 * (lpl - lpr);
            lgp = 0.5f * (lpl + lpr);
            const float icref = exp2f(0.25f * ((lrl + lrr) - (lpl + lpr))) * rsqg;
            const float du2 = 0.5f * du * icref;
            x[0] = a;
            x[1] = du2;
            x[2] = b;
            x[3] = -a;
            x[4] = -du2;
            x[5] = -b;
        }
        {
            uint4 lo;
            const __nv_bfloat162 x01 = __floats2bfloat162_rn(x[0], x[1]);
            const __nv_bfloat162 x23 = __floats2bfloat162_rn(x[2], x[3]);
            const __nv_bfloat162 x45 = __floats2bfloat162_rn(x[4], x[5]);
            lo.x = *reinterpret_cast<const uint32_t *>(&x01);
            lo.y = *reinterpret_cast<const uint32_t *>(&x23);
            lo.z = *reinterpret_cast<const uint32_t *>(&x45);
            lo.w = 0x3F80u;   // column 6 = 1, column 7 = 0
            *reinterpret_cast<uint4 *>(S->a1 + tc::tile_off(row, 0, 16)) = lo;
            *reinterpret_cast<uint4 *>(S->a1 + tc::tile_off(row, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
        }
        if (timeout) S->err = 1;
        tc::fence_async_smem();
        tc::fence_before();
        const bool anynew = __syncthreads_or(need) != 0;
        if (S->err) {
            ok = false;
            return -1.0f;
        }
        if (row == 0 && (anynew || any1)) {
            tc::fence_after();
            if (anynew)
                tc::mma_bf16(S->tmem, tc::smem_desc(tc::smem_u32(S->a1), 128, 256),
                             tc::smem_desc(tc::smem_u32(S->w1), 128, 256), tc::idesc_bf16_f32(128, 64), false);
            if (any1) {
#pragma unroll
                for (int ks = 0; ks < 5; ++ks)
                    tc::mma_bf16(S->tmem + 64, tc::smem_desc(tc::smem_u32(S->a2) + ks * 256, 128, 1280),
                                 tc::smem_desc(tc::smem_u32(S->w2) + ks * 256, 128, 1280),
                                 tc::idesc_bf16_f32(128, 64), ks > 0);
            }
            tc::commit(&S->mbar);
        }
        committed = anynew || any1;
        any2 = any1;
        any1 = anynew;
        need2 = need1;
        need1 = need;
        s2 = s1;
        s1 = lgp;
        return p0;
    }
};

// EXT: 0 the default kernels; 1 with the reconstruction options (steepening,
// flattening, diffusive flux); 2 with those and dual energy.
template <class R, bool WRAP, int DIR, bool REG = false, int EXT = 0>
struct Marcher {
    static constexpr int A1 = DIR == 0 ? 1 : 0;
    static constexpr int A2 = DIR == 2 ? 1 : 2;
    const SweepArgs &a;
    Pencil pc;
    Consts<R> k;
    bool active;          // false: a stand-in pencil that only keeps the CTA in step
    unsigned log_key;     // pencil identity for the interface-state log
    double *reg_all;      // this pencil's all-face flux register row, or nullptr
    double *reg_bnd;      // this pencil's boundary-face register pair, or nullptr
    double dt64;
    // WRAP: the initial state of the first three active cells (and their eps
    // with dual energy), which the trailing ghost positions reuse after the
    // pencil has updated those cells.  FP32 keeps them in shared memory (the
    // kernel's per-thread slots, stride kSave), FP64 in registers.
    float *wsave;
    static constexpr int kSave = EXT == 2 ? 7 : 6;   // r, u, p, t1, t2, c (and eps with dual energy)
    // Plain FP32 march: the raw FP64 values (rho, m_n, m_t1, m_t2, E) of the
    // last kRingSlots positions, in shared memory ([slot][field] x blockDim.x,
    // this thread's column), so the update of a cell four steps after its load
    // and the fallback test read them there instead of going back to L2.  In y
    // and z sweeps the ring also holds the kStage positions ahead of the march,
    // copied in asynchronously (cp.async) while the march works on earlier
    // ones: positions k-4 .. k+kStage at step k.
    double *uring;
    static constexpr int kRingSlots = DIR == 0 ? 5 : 8;
    static constexpr int kStage = 3;
    // Learned march (y and z): no room for the update's ring beside the
    // network's shared memory, only for the loads: positions k..k+2, staged
    // two steps ahead, after the network's shared memory.
    static constexpr int kLearnedSlots = 3;
    template <int SLOTS = kRingSlots>
    __device__ __forceinline__ double &ring(int s, int f) const
    {
        return uring[((s % SLOTS) * 5 + f) * (int)blockDim.x];
    }
    Zone<R> c0, c1, c2;
    R ce0, ce1, ce2;

    __device__ __forceinline__ void save(int t, const Zone<R> &z, R e)
    {
        if constexpr (sizeof(R) == 4) {
            float *o = wsave + t * kSave * blockDim.x;
            const float v[7] = {z.r, z.u, z.p, z.t1, z.t2, z.c, e};
            _Pragma("unroll") for (int i = 0; i < kSave; ++i) o[i * blockDim.x] = v[i];
        } else {
            if (t == 0) { c0 = z; ce0 = e; }
            else if (t == 1) { c1 = z; ce1 = e; }
            else { c2 = z; ce2 = e; }
        }
    }
    __device__ __forceinline__ Zone<R> saved(int t, R &e) const
    {
        if constexpr (sizeof(R) == 4) {
            const float *o = wsave + t * kSave * blockDim.x;
            e = EXT == 2 ? o[6 * blockDim.x] : 0.0f;
            return Zone<R>{o[0], o[blockDim.x], o[2 * blockDim.x], o[3 * blockDim.x], o[4 * blockDim.x],
                           o[5 * blockDim.x]};
        } else {
            e = t == 0 ? ce0 : (t == 1 ? ce1 : ce2);
            return t == 0 ? c0 : (t == 1 ? c1 : c2);
        }
    }

    // Dual energy: gas-energy flux and interface velocity of one face.
    struct GeFace {
        R F, uf;
    };
    // Dual energy: the last updated cell, whose resynchronisation waits for the
    // new E of its right neighbour (Sec. 4.1.1 compares E - KE with the largest
    // E of the cell and its two neighbours along the sweep).
    struct GePending {
        int64_t idx;        // < 0: none yet
        double ge, e, E;    // advected gas energy, E - KE and E after the update
        double Eleft;       // E of its left neighbour (the ghost's for the first cell)
        bool ok;            // rho > 0 after the update
    };
    GePending gpend;

    // Write the pending cell's gas energy once the E of its right neighbour is known.
    __device__ __forceinline__ void ge_commit(double Eright)
    {
        double emax = gpend.Eleft;
        if (gpend.E > emax) emax = gpend.E;
        if (Eright > emax) emax = Eright;
        const double g = gpend.ok && gpend.e > 0.1 * emax ? gpend.e : gpend.ge;
        if (active) a.ge[gpend.idx] = g;
    }

    __device__ __forceinline__ const double *F(int f) const { return a.U[f]; }

    // Storage index of pencil position s (the stored cell or its periodic
    // image); -1 for a trailing wrapped ghost, whose zone is a saved one.
    __device__ __forceinline__ int64_t index_of(int s) const
    {
        if (WRAP) {
            const int j = s - pc.ng;
            if (j >= pc.n) return -1;
            return pc.at(pc.ng + (j < 0 ? (pc.n - ((-j) % pc.n)) % pc.n : j));
        }
        return pc.at(s);
    }

    // Ask the memory system for the five fields of pencil position s ahead of
    // their load (a cache prefetch: no registers are held), so that the load
    // a few march steps later hits the cache instead of waiting for HBM.
    __device__ __forceinline__ void warm(int s) const
    {
        // x pencils walk their own rows, which the cache lines they already
        // loaded cover 16 positions at a time
        if (ENZO_PREFETCH_AHEAD == 0 || DIR == 0 || s >= pc.L) return;
        const int64_t idx = index_of(s);
        if (idx < 0) return;
        ENZO_PREFETCH(a.U[0] + idx);
        ENZO_PREFETCH(a.U[1] + idx);
        ENZO_PREFETCH(a.U[2] + idx);
        ENZO_PREFETCH(a.U[3] + idx);
        ENZO_PREFETCH(a.U[4] + idx);
    }

    // Start the asynchronous copy of pencil position s's five raw values into
    // its slot of a SLOTS-slot ring (nothing for a trailing wrapped ghost or
    // past the pencil's end), as one commit group of this thread.  A warp's 32
    // copies of one field are 32 consecutive doubles in y and z sweeps.
    template <int SLOTS = kRingSlots>
    __device__ __forceinline__ void stage(int s) const
    {
        if (s < pc.L) {
            const int64_t idx = index_of(s);
            if (idx >= 0) {
                const double *src[5] = {a.U[0] + idx, a.U[1 + DIR] + idx, a.U[1 + A1] + idx, a.U[1 + A2] + idx,
                                        a.U[4] + idx};
                _Pragma("unroll") for (int f = 0; f < 5; ++f)
                {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(&ring<SLOTS>(s, f));
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src[f]) : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // Zone at pencil position s from its ring slot, once its copy has landed
    // (the AHEAD groups committed after it may still be in flight).
    template <int SLOTS = kRingSlots, int AHEAD = kStage>
    __device__ __forceinline__ Zone<R> zone_staged(int s, Counters &cnt)
    {
        if (index_of(s) < 0) {
            R e;
            return saved((s - pc.ng - pc.n) % pc.n, e);
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(AHEAD) : "memory");
        return prim<R, true>(ring<SLOTS>(s, 0), ring<SLOTS>(s, 1), ring<SLOTS>(s, 2), ring<SLOTS>(s, 3),
                             ring<SLOTS>(s, 4), k, cnt);
    }

    // Zone at pencil position s, its raw values also kept in the ring.
    __device__ __forceinline__ Zone<R> zone_keep(int s, Counters &cnt)
    {
        const int64_t idx = index_of(s);
        if (idx < 0) {
            R e;
            return saved((s - pc.ng - pc.n) % pc.n, e);
        }
        const double v0 = ld_march<DIR>(a.U[0] + idx), v1 = ld_march<DIR>(a.U[1 + DIR] + idx),
                     v2 = ld_march<DIR>(a.U[1 + A1] + idx), v3 = ld_march<DIR>(a.U[1 + A2] + idx),
                     v4 = ld_march<DIR>(a.U[4] + idx);
        ring(s, 0) = v0;
        ring(s, 1) = v1;
        ring(s, 2) = v2;
        ring(s, 3) = v3;
        ring(s, 4) = v4;
        return prim<R, true>(v0, v1, v2, v3, v4, k, cnt);
    }

    // Zone at pencil position s, before any update of this sweep.
    template <bool COUNT>
    __device__ __forceinline__ Zone<R> zone(int s, Counters &cnt)
    {
        int64_t idx;
        if (WRAP) {
            const int j = s - pc.ng;
            if (j >= pc.n) {
                // trailing ghost: image of active cell (j - n) mod n, which this
                // pencil may already have updated, so its initial state is kept
                R e;
                return saved((j - pc.n) % pc.n, e);
            }
            const int jj = j < 0 ? (pc.n - ((-j) % pc.n)) % pc.n : j;
            idx = pc.at(pc.ng + jj);
        } else {
            idx = pc.at(s);
        }
        // read-only (non-coherent) path: within one sweep a cell is read by the
        // thread of its own pencil before that thread writes it, never after
        return prim<R, COUNT>(ld_march<DIR>(a.U[0] + idx), ld_march<DIR>(a.U[1 + DIR] + idx),
                              ld_march<DIR>(a.U[1 + A1] + idx), ld_march<DIR>(a.U[1 + A2] + idx),
                              ld_march<DIR>(a.U[4] + idx), k, cnt);
    }

    // Zone at pencil position s with the dual-energy pressure choice, and its
    // eps = ge / rho (EXT kernels with a gas-energy field only).
    template <bool COUNT>
    __device__ __forceinline__ Zone<R> zone_dual(int s, Counters &cnt, R &eps)
    {
        int64_t idx;
        if (WRAP) {
            const int j = s - pc.ng;
            if (j >= pc.n) {
                return saved((j - pc.n) % pc.n, eps);
            }
            const int jj = j < 0 ? (pc.n - ((-j) % pc.n)) % pc.n : j;
            idx = pc.at(pc.ng + jj);
        } else {
            idx = pc.at(s);
        }
        return prim_dual<COUNT>(__ldg(a.U[0] + idx), __ldg(a.U[1 + DIR] + idx), __ldg(a.U[1 + A1] + idx),
                                __ldg(a.U[1 + A2] + idx), __ldg(a.U[4] + idx), __ldg(a.ge + idx), k, cnt, eps);
    }

    // Fallback mode 2 (EXT kernels): does the Godunov update of cell s with face
    // fluxes Fm, Fp leave rho <= 0 or a non-positive internal energy (tested as
    // 2 rho E - |m|^2 <= 0)?  Decided in FP64 on the exact update the cell would
    // get: the FP64 flux difference, or the FP32 path's widened increments.
    __device__ __forceinline__ bool fails_full(int s, const R Fm[5], const R Fp[5], R dtdx, double dtdx64) const
    {
        const int64_t idx = pc.at(s);
        const int map[5] = {0, 1 + DIR, 1 + A1, 1 + A2, 4};
        double u[5];
        _Pragma("unroll") for (int v = 0; v < 5; ++v)
        {
            const double U = a.U[map[v]][idx];
            if (sizeof(R) == 8) u[v] = cell_update(U, dtdx64, (double)Fm[v], (double)Fp[v]);
            else u[v] = (U + f2d_exact((float)(dtdx * Fm[v]))) - f2d_exact((float)(dtdx * Fp[v]));
        }
        return fails_state(u);
    }

    // FP32 screen of fallback mode 2: the zone's conserved state rebuilt from its
    // primitives plus the two faces' FP32 increments.  True only when rho and
    // E keep at least 1e-3 of their old values and the internal energy at
    // least 1e-2 of E, far beyond the FP32 rounding of the estimate; a floored
    // zone never passes (its primitives are not its conserved state).
    __device__ __forceinline__ bool clearly_ok(const Zone<R> &z, const R Fm[5], const R Fp[5], R dtdx) const
    {
        if (!(z.r > (R)4 * k.rho_floor) || !(z.p > (R)4 * k.p_floor)) return false;
        const R E0 = z.p * k.gm1inv + (R)0.5 * z.r * ((z.u * z.u + z.t1 * z.t1) + z.t2 * z.t2);
        const R rn = z.r + dtdx * (Fm[0] - Fp[0]);
        const R m0 = z.r * z.u + dtdx * (Fm[1] - Fp[1]);
        const R m1 = z.r * z.t1 + dtdx * (Fm[2] - Fp[2]);
        const R m2 = z.r * z.t2 + dtdx * (Fm[3] - Fp[3]);
        const R En = E0 + dtdx * (Fm[4] - Fp[4]);
        if (!(rn > (R)1e-3 * z.r) || !(En > (R)1e-3 * E0)) return false;
        const R twoRE = (R)2 * rn * En;
        return twoRE - ((m0 * m0 + m1 * m1) + m2 * m2) > (R)1e-2 * twoRE;
    }

    static __device__ __forceinline__ bool fails_state(const double u[5])
    {
        if (!(u[0] > 0.0)) return true;
        const double m2 = (u[1] * u[1] + u[2] * u[2]) + u[3] * u[3];
        return !((2.0 * u[0]) * u[4] - m2 > 0.0);
    }

    // Density of cell s at the start of the sweep (raw, no floor).
    template <bool RING = false>
    __device__ __forceinline__ double rho_old(int s) const
    {
        if constexpr (RING) return ring(s, 0);
        else return a.U[0][pc.at(s)];
    }

    // Write the final state of active cell s given its two face terms.  With
    // dual energy (gm, gp non-null) also the gas energy: its flux difference
    // and the source -p (u_{s+1/2} - u_{s-1/2}) dt/dx with the zone pressure pz;
    // the cell then becomes the pending one, and the previous pending cell,
    // whose right neighbour this is, is resynchronised and written.
    template <bool RING = false>
    __device__ __forceinline__ void update(int s, const R Fm[5], const R Fp[5], double dtdx64,
                                           const double Gm[5], const double Gp[5], bool fb,
                                           Counters &cnt, const GeFace *gm = nullptr,
                                           const GeFace *gp = nullptr, R pz = (R)0, R dtdx = (R)0)
    {
        const int64_t idx = pc.at(s);
        double u[5];
        const int map[5] = {0, 1 + DIR, 1 + A1, 1 + A2, 4};
        _Pragma("unroll") for (int v = 0; v < 5; ++v)
        {
            const double U = RING ? ring(s, v) : ld_march<DIR>(a.U[map[v]] + idx);
            if (sizeof(R) == 8) u[v] = cell_update(U, dtdx64, (double)Fm[v], (double)Fp[v]);
            else u[v] = (U + Gm[v]) - Gp[v];
        }
        double gnew = 0.0;
        const bool dual = EXT == 2 && gm != nullptr;
        if (dual) {
            const double g0 = a.ge[idx];
            if (sizeof(R) == 8) {
                gnew = (g0 + dtdx64 * ((double)gm->F - (double)gp->F)) -
                       dtdx64 * (double)pz * ((double)gp->uf - (double)gm->uf);
            } else {
                const double g_m = f2d_exact((float)(dtdx * gm->F));
                const double g_p = f2d_exact((float)(dtdx * gp->F));
                const double src = f2d_exact((float)(dtdx * pz * (gp->uf - gm->uf)));
                gnew = ((g0 + g_m) - g_p) - src;
            }
            double enew = 0.0;
            const bool ok = u[0] > 0.0;
            if (ok) {
                if (sizeof(R) == 8) {
                    const double ke = 0.5 * ((u[1] * u[1] + u[2] * u[2]) + u[3] * u[3]) / u[0];
                    enew = u[4] - ke;
                } else {
                    // FP32 path: KE in FP32 off the FP64 pipe; E - KE is only
                    // taken where it exceeds 0.1 E, so its error stays below
                    // 1e-6 of it
                    const float r = d2f_rz(u[0]), m0 = d2f_rz(u[1]), m1 = d2f_rz(u[2]), m2 = d2f_rz(u[3]);
                    enew = u[4] - f2d_exact((R)0.5 * ((m0 * m0 + m1 * m1) + m2 * m2) / r);
                }
            }
            if (gpend.idx >= 0) {
                ge_commit(u[4]);
                gpend.Eleft = gpend.E;
            }
            gpend.idx = idx;
            gpend.ge = gnew;
            gpend.e = enew;
            gpend.E = u[4];
            gpend.ok = ok;
        }
        if (!active) return;
        if (fb && (EXT && a.mp.fallback == 2 ? fails_state(u) : !(u[0] > 0.0))) cnt.rare(ENZO_ST_NEG_AFTER);
        if (u[0] != u[0] || u[4] != u[4]) cnt.rare(ENZO_ST_NAN);
        _Pragma("unroll") for (int v = 0; v < 5; ++v) const_cast<double *>(a.U[map[v]])[idx] = u[v];
    }

    __device__ __forceinline__ void widen(const R Fv[5], R dtdx, double G[5]) const
    {
        if (sizeof(R) == 4) {
            _Pragma("unroll") for (int v = 0; v < 5; ++v) G[v] = f2d_exact((float)(dtdx * Fv[v]));
        }
    }

    __device__ __forceinline__ void log_states(int kk, const R sl[5], const R sr[5])
    {
        const unsigned h = (log_key * 2654435761u) ^ ((unsigned)kk * 40503u);
        if (!active || (h % (unsigned)a.log_stride) != 0u) return;
        const unsigned long long slot = atomicAdd(a.log_count, 1ull);
        if ((long long)slot >= a.log_cap) return;
        float *o = a.log + 6 * slot;
        o[0] = (float)sl[0]; o[1] = (float)sl[1]; o[2] = (float)sl[2];
        o[3] = (float)sr[0]; o[4] = (float)sr[1]; o[5] = (float)sr[2];
    }

    // Flux register entries of face f (left of active cell f; f = n is the
    // right face of the last cell) once its final flux is known.  FP64 path:
    // the flux F (all faces) and dt F summed over steps (boundary faces).  FP32
    // path: the increment G = dt/dx F exactly as the cells applied it, and its
    // sum, so a flux correction cancels the applied coarse increment exactly.
    // With dual energy (EXT == 2) a face has a sixth entry, the gas-energy
    // flux gF (FP32 path: its applied increment gG); the -p div v source is a
    // zone term and has none.
    static constexpr int NC = EXT == 2 ? 6 : 5;
    __device__ __forceinline__ void record(int f, const R Fv[5], const double G[5], R gF = (R)0, double gG = 0.0)
    {
        if (!REG) return;
        if (reg_all) {
            _Pragma("unroll") for (int v = 0; v < 5; ++v) reg_all[f * NC + v] = sizeof(R) == 8 ? (double)Fv[v] : G[v];
            if constexpr (EXT == 2) reg_all[f * NC + 5] = sizeof(R) == 8 ? (double)gF : gG;
        }
        if (reg_bnd && (f == 0 || f == pc.n)) {
            double *o = reg_bnd + (f == 0 ? 0 : NC);
            _Pragma("unroll") for (int v = 0; v < 5; ++v) o[v] = o[v] + (sizeof(R) == 8 ? dt64 * (double)Fv[v] : G[v]);
            if constexpr (EXT == 2) o[5] = o[5] + (sizeof(R) == 8 ? dt64 * (double)gF : gG);
        }
    }

    // Optional reconstruction dissipation of zone j (CW84; optional in
    // Sec. 4.1) on its unlimited edge values el/er, in the order the monotone
    // parabola then takes them: contact steepening of the density, then
    // flattening of all five variables.  Zones j-2..j+2 are zj2m (density and
    // pressure only), zj1m, zj, zj1p, zj2p; dm1 / dp1 are the limited density
    // slopes of zones j-1 / j+1.  Detectors and weights as in the oracle:
    // steepening where the density has an inflection across a jump of at least
    // 1% that is a contact, not a shock; flattening where the flow compresses
    // across a pressure jump above 33%, weighted by the ratio of the 2-zone and
    // 4-zone pressure differences.  With dual energy (elx, erx non-null) the
    // edges of eps (zone value qx) are flattened with the same weight.
    __device__ __forceinline__ void dissipate(const MethodParams &mp, const Zone<R> &zj1m, const Zone<R> &zj,
                                              const Zone<R> &zj1p, const Zone<R> &zj2p, R rj2m, R pj2m, R dm1,
                                              R dp1, R el[5], R er[5], R qx = (R)0, R *elx = nullptr,
                                              R *erx = nullptr) const
    {
        if (mp.options & ENZO_OPT_STEEPEN) {
            const R Dm = (zj.r - (R)2 * zj1m.r) + rj2m;
            const R Dp = (zj2p.r - (R)2 * zj1p.r) + zj.r;
            const R dr = zj1p.r - zj1m.r;
            const R rmin = zj1p.r < zj1m.r ? zj1p.r : zj1m.r;
            const R pmin = zj1p.p < zj1m.p ? zj1p.p : zj1m.p;
            R et = (R)0;
            const bool contact = fabs(zj1p.p - zj1m.p) / pmin <= (R)0.1 * k.gamma * (fabs(dr) / rmin);
            if (Dm * Dp < (R)0 && fabs(dr) >= (R)0.01 * rmin && contact) et = -(Dp - Dm) / ((R)6 * dr);
            R e = (R)20 * (et - (R)0.05);
            e = e < (R)0 ? (R)0 : (e > (R)1 ? (R)1 : e);
            if (e > (R)0) {
                el[0] = el[0] * ((R)1 - e) + (zj1m.r + (R)0.5 * dm1) * e;
                er[0] = er[0] * ((R)1 - e) + (zj1p.r - (R)0.5 * dp1) * e;
            }
        }
        if (mp.options & ENZO_OPT_FLATTEN) {
            const R dp1p = zj1p.p - zj1m.p, dp2p = zj2p.p - pj2m;
            const R pmin = zj1p.p < zj1m.p ? zj1p.p : zj1m.p;
            if (zj1m.u - zj1p.u > (R)0 && fabs(dp1p) > (R)0.33 * pmin) {
                R f = (R)1;
                if (dp2p != (R)0) {
                    f = (R)10 * (dp1p / dp2p - (R)0.75);
                    f = f < (R)0 ? (R)0 : (f > (R)1 ? (R)1 : f);
                }
                if (f > (R)0) {
                    _Pragma("unroll") for (int v = 0; v < 5; ++v)
                    {
                        const R q = zv(zj, v);
                        el[v] = f * q + ((R)1 - f) * el[v];
                        er[v] = f * q + ((R)1 - f) * er[v];
                    }
                    if (elx) {
                        *elx = f * qx + ((R)1 - f) * *elx;
                        *erx = f * qx + ((R)1 - f) * *erx;
                    }
                }
            }
        }
    }

    // Diffusive flux at the interface between zones a (left) and b (right):
    // 0.1 max(0, u_a - u_b) times the jump of the conserved state rebuilt from
    // the zone primitives (CW84; optional in Sec. 4.1).  With dual energy
    // (Fx non-null) the gas-energy flux too, rho eps being its conserved value.
    __device__ __forceinline__ void diffuse(const Zone<R> &za, const Zone<R> &zb, R F[5], R ea = (R)0,
                                            R eb = (R)0, R *Fx = nullptr) const
    {
        const R du = za.u - zb.u;
        if (!(du > (R)0)) return;
        const R nu = (R)0.1 * du;
        R Ua[5], Ub[5];
        const Zone<R> *zs[2] = {&za, &zb};
        _Pragma("unroll") for (int z = 0; z < 2; ++z)
        {
            R *Uz = z ? Ub : Ua;
            const Zone<R> &q = *zs[z];
            Uz[0] = q.r;
            Uz[1] = q.r * q.u;
            Uz[2] = q.r * q.t1;
            Uz[3] = q.r * q.t2;
            Uz[4] = q.p / k.gm1 + (R)0.5 * q.r * ((q.u * q.u + q.t1 * q.t1) + q.t2 * q.t2);
        }
        _Pragma("unroll") for (int v = 0; v < 5; ++v) F[v] = F[v] + nu * (Ua[v] - Ub[v]);
        if (Fx) *Fx = *Fx + nu * (za.r * ea - zb.r * eb);
    }

    // One pencil with the plain guess: a sliding window over the zones; march
    // step kk loads zone kk and solves interface (kk-3)+1/2.
    template <class GS>
    __device__ void run(R dtdx, double dtdx64, const MethodParams &mp, Counters &cnt, GS &guess)
    {
        constexpr bool RING = sizeof(R) == 4 && EXT == 0;   // the shared-memory ring of raw values
        const int L = pc.L;
        const bool fb = mp.fallback != 0;
        Zone<R> zm2, zm1, z0;                 // zones k-2, k-1, k
        R dprev[5], qfprev[5], sLprev[5];
        R Fgprev[5], Fuprev2[5];
        double Gprev2[5];                     // FP32 path: widened face term of Fuprev2
        R rho3 = (R)0, rho2 = (R)0, rho1 = (R)0, rho0 = (R)0;   // FP32: raw densities of cells k-3..k
        bool badprev = false;
        _Pragma("unroll") for (int v = 0; v < 5; ++v)
        {
            dprev[v] = qfprev[v] = sLprev[v] = Fgprev[v] = Fuprev2[v] = (R)0;
            Gprev2[v] = 0.0;
        }
        z0 = zm1 = zm2 = Zone<R>{};
        // EXT (steepening, flattening, diffusive flux): zone k-3, density and
        // pressure of zone k-4, and the density slope of zone k-3
        Zone<R> zm3{};
        R r4 = (R)0, p4 = (R)0, ds3 = (R)0;
        // EXT with dual energy: eps of zones k-3..k; for eps the slope of zone
        // k-2, the interface value at (k-3)+1/2 and the left state traced there;
        // the gas-energy face terms, Godunov at (k-4)+1/2 and final at (k-5)+1/2
        const bool dual = EXT == 2 && a.ge != nullptr;
        R e3 = (R)0, e2 = (R)0, e1 = (R)0, e0 = (R)0;
        R dep = (R)0, qfep = (R)0, sLep = (R)0;
        GeFace gg{(R)0, (R)0}, gfin2{(R)0, (R)0};
        // E at the start of the sweep of the ghosts beside the first and last
        // active cells (their periodic images when the pencil wraps: the last
        // active cell is not yet updated here, the first one will be by the end)
        double Eghost_right = 0.0;
        if (dual) {
            gpend.idx = -1;
            gpend.Eleft = a.U[4][WRAP ? pc.at(pc.ng + pc.n - 1) : pc.at(pc.ng - 1)];
            Eghost_right = a.U[4][WRAP ? pc.at(pc.ng) : pc.at(pc.ng + pc.n)];
        }
        if constexpr (RING && DIR != 0)
            for (int q = 0; q < kStage; ++q) stage(q);
        for (int kk = 0; kk < L; ++kk) {
            if constexpr (EXT) {
                r4 = zm3.r;
                p4 = zm3.p;
                zm3 = zm2;
                e3 = e2;
                e2 = e1;
                e1 = e0;
            }
            zm2 = zm1;
            zm1 = z0;
            if (dual) {
                z0 = zone_dual<true>(kk, cnt, e0);
            } else {
                if constexpr (RING && DIR != 0) {
                    stage(kk + kStage);
                    z0 = zone_staged(kk, cnt);
                } else if constexpr (RING) {
                    z0 = zone_keep(kk, cnt);
                } else {
                    warm(kk + ENZO_PREFETCH_AHEAD);
                    z0 = zone<true>(kk, cnt);
                }
            }
            if (WRAP) {
                const int j = kk - pc.ng;
                if (j >= 0 && j < 3) save(j, z0, e0);
            }
            if (sizeof(R) == 4) {
                rho3 = rho2;
                rho2 = rho1;
                rho1 = rho0;
                rho0 = z0.r;
            }
            if (kk < 2) continue;
            R dcur[5];
            _Pragma("unroll") for (int v = 0; v < 5; ++v) dcur[v] = limited_slope<R>(zv(zm2, v), zv(zm1, v), zv(z0, v));
            const R dce = dual ? limited_slope<R>(e2, e1, e0) : (R)0;
            if (kk >= 3) {
                R qfcur[5];
                _Pragma("unroll") for (int v = 0; v < 5; ++v)
                    qfcur[v] = (R)0.5 * (zv(zm2, v) + zv(zm1, v)) - div6(dcur[v] - dprev[v]);
                const R qfce = dual ? (R)0.5 * (e2 + e1) - div6(dce - dep) : (R)0;
                if (kk >= 4) {
                    R sRe = (R)0, sLen = (R)0;   // eps traced to the left / right edge of zone kk-2
                    // parabola of zone kk-2 (its edges: qfprev on the left, qfcur on the right)
                    R pL[5], pR[5], pd[5], p6[5];
                    if constexpr (EXT) {
                        R el[5], er[5];
                        _Pragma("unroll") for (int v = 0; v < 5; ++v)
                        {
                            el[v] = qfprev[v];
                            er[v] = qfcur[v];
                        }
                        R ele = qfep, ere = qfce;
                        dissipate(mp, zm3, zm2, zm1, z0, r4, p4, ds3, dcur[0], el, er, e2, dual ? &ele : nullptr,
                                  dual ? &ere : nullptr);
                        _Pragma("unroll") for (int v = 0; v < 5; ++v) parabola<R>(zv(zm2, v), el[v], er[v], pL[v], pR[v], pd[v], p6[v]);
                        if (dual) {
                            R eL, eR, ed, e6;
                            parabola<R>(e2, ele, ere, eL, eR, ed, e6);
                            sRe = trace_passive<R, -1>(eL, eR, ed, e6, zm2.u, dtdx);
                            sLen = trace_passive<R, +1>(eL, eR, ed, e6, zm2.u, dtdx);
                        }
                    } else {
                        _Pragma("unroll") for (int v = 0; v < 5; ++v) parabola<R>(zv(zm2, v), qfprev[v], qfcur[v], pL[v], pR[v], pd[v], p6[v]);
                    }
                    R sR[5], sLnew[5];
                    trace<R, -1>(pL, pR, pd, p6, zm2.u, zm2.c, dtdx, k, sR);
                    trace<R, +1>(pL, pR, pd, p6, zm2.u, zm2.c, dtdx, k, sLnew);
                    if (kk >= 5) {
                        // Riemann problem at interface (kk-3)+1/2
                        if (a.log) log_states(kk, sLprev, sR);
                        R Fg[5];
                        GeFace gcur{(R)0, (R)0};
                        if (mp.solver == ENZO_SOLVER_TWOSHOCK) {
                            const R p0 = guess(sLprev[0], sLprev[1], sLprev[2], sR[0], sR[1], sR[2]);
                            const RiemannOut<R> o = riemann<R>(sLprev[0], sLprev[1], sLprev[2], sR[0], sR[1],
                                                               sR[2], p0, k, cnt);
                            if (active) {
                                if (p0 > (R)0) cnt.guesses++;
                                cnt.iters += (unsigned)o.iters;
                                if (!o.conv) cnt.rare(ENZO_ST_NEWTON_NONCONV);
                            }
                            const R t1 = o.ustar >= (R)0 ? sLprev[3] : sR[3];
                            const R t2 = o.ustar >= (R)0 ? sLprev[4] : sR[4];
                            phys_flux<R>(o.rho, o.u, o.p, t1, t2, k, Fg);
                            if (dual) {
                                gcur.F = Fg[0] * (o.ustar >= (R)0 ? sLep : sRe);
                                gcur.uf = o.u;
                            }
                        } else if (mp.solver == ENZO_SOLVER_HLLC) {
                            hllc_states<R>(sLprev, sR, k, Fg);
                        } else {
                            hll_states<R>(sLprev, sR, k, Fg);
                        }
                        if constexpr (EXT) {
                            if (mp.options & ENZO_OPT_DIFFUSE) diffuse(zm3, zm2, Fg, e3, e2, dual ? &gcur.F : nullptr);
                        }
                        if (kk >= 6) {
                            // cell c = kk-3: does the Godunov update leave rho > 0?
                            const int c = kk - 3;
                            bool bad = false;
                            if (fb) {
                                if (EXT && mp.fallback == 2) {
                                    // FP32: a screen on the zone's own primitives with wide
                                    // margins; only unclear cells take the exact FP64 test
                                    // (always with dual energy: the zone pressure may come
                                    // from the gas energy, not from E)
                                    bad = (sizeof(R) == 8 || dual || !clearly_ok(zm3, Fgprev, Fg, dtdx))
                                              ? fails_full(c, Fgprev, Fg, dtdx, dtdx64) : false;
                                } else if (sizeof(R) == 8) {
                                    bad = !(cell_update(rho_old<RING>(c), dtdx64, (double)Fgprev[0], (double)Fg[0]) > 0.0);
                                } else {
                                    // FP32 screen; cells near zero are decided in FP64
                                    const R rt = rho3 + dtdx * (Fgprev[0] - Fg[0]);
                                    if (!(rt > (R)1e-3 * rho3)) {
                                        const double g0 = f2d_exact((float)(dtdx * Fgprev[0]));
                                        const double g1 = f2d_exact((float)(dtdx * Fg[0]));
                                        bad = !((rho_old<RING>(c) + g0) - g1 > 0.0);
                                    }
                                }
                                if (bad && active) cnt.rare(ENZO_ST_HLL_CELLS);
                            }
                            // final flux at face (kk-4)+1/2
                            R Fu1[5];
                            GeFace gfin = gg;
                            if (badprev || bad) fallback_face(kk - 4, dual, Fu1, gfin);
                            else {
                                _Pragma("unroll") for (int v = 0; v < 5; ++v) Fu1[v] = Fgprev[v];
                            }
                            double G1[5];
                            widen(Fu1, dtdx, G1);
                            if constexpr (REG && EXT == 2)
                                record(kk - 6, Fu1, G1, gfin.F, sizeof(R) == 4 ? f2d_exact((float)(dtdx * gfin.F)) : 0.0);
                            else record(kk - 6, Fu1, G1);
                            if (kk >= 7)
                                update<RING>(kk - 4, Fuprev2, Fu1, dtdx64, Gprev2, G1, fb, cnt,
                                             dual ? &gfin2 : nullptr, &gfin, p4, dtdx);
                            gfin2 = gfin;
                            _Pragma("unroll") for (int v = 0; v < 5; ++v)
                            {
                                Fuprev2[v] = Fu1[v];
                                Gprev2[v] = G1[v];
                            }
                            badprev = bad;
                        }
                        _Pragma("unroll") for (int v = 0; v < 5; ++v) Fgprev[v] = Fg[v];
                        gg = gcur;
                    }
                    _Pragma("unroll") for (int v = 0; v < 5; ++v) sLprev[v] = sLnew[v];
                    sLep = sLen;
                }
                _Pragma("unroll") for (int v = 0; v < 5; ++v) qfprev[v] = qfcur[v];
                qfep = qfce;
            }
            if constexpr (EXT) ds3 = dprev[0];
            _Pragma("unroll") for (int v = 0; v < 5; ++v) dprev[v] = dcur[v];
            dep = dce;
        }
        // last active cell L-4: its right face (L-4)+1/2 borders a ghost zone
        R Fu1[5];
        GeFace gfin = gg;
        if (badprev) fallback_face(L - 4, dual, Fu1, gfin);
        else {
            _Pragma("unroll") for (int v = 0; v < 5; ++v) Fu1[v] = Fgprev[v];
        }
        double G1[5];
        widen(Fu1, dtdx, G1);
        if constexpr (REG && EXT == 2)
            record(pc.n, Fu1, G1, gfin.F, sizeof(R) == 4 ? f2d_exact((float)(dtdx * gfin.F)) : 0.0);
        else record(pc.n, Fu1, G1);
        // the pressure of zone L-4 is the last window's zone k-3
        update<RING>(L - 4, Fuprev2, Fu1, dtdx64, Gprev2, G1, fb, cnt, dual ? &gfin2 : nullptr, &gfin, zm3.p, dtdx);
        if (dual) ge_commit(Eghost_right);
    }

    // HLL re-flux (Sec. 4.1.2) of the face between zones s and s+1 from their
    // zone states; with dual energy also its gas-energy flux (the HLL mass flux
    // times the upwind zone eps) and interface velocity (the mean zone velocity).
    __device__ __forceinline__ void fallback_face(int s, bool dual, R Fu[5], GeFace &g)
    {
        Counters quiet;
        if (dual) {
            R ea, eb;
            const Zone<R> za = zone_dual<false>(s, quiet, ea);
            const Zone<R> zb = zone_dual<false>(s + 1, quiet, eb);
            hll_flux<R>(za, zb, k, Fu);
            g.F = Fu[0] * (Fu[0] >= (R)0 ? ea : eb);
            g.uf = (R)0.5 * (za.u + zb.u);
        } else {
            const Zone<R> za = zone<false>(s, quiet);
            const Zone<R> zb = zone<false>(s + 1, quiet);
            hll_flux<R>(za, zb, k, Fu);
        }
    }

    // One pencil with the pipelined learned guess.  March step kk loads zone kk
    // and traces the states of interface (kk-3)+1/2; the Riemann solve, flux and
    // update of interface jj = kk - D follow (D = 2: the traced states wait two
    // steps in a shared-memory ring while the tensor core evaluates the
    // network, and the pencil takes D extra drain steps).
    template <class GS>
    __device__ void run_piped(R dtdx, double dtdx64, const MethodParams &mp, Counters &cnt, GS &guess)
    {
        constexpr int D = GS::kDepth;
        static_assert(D == 2, "the state ring holds two steps");
        float4 *ring = guess.S->ring[0][threadIdx.x];
        const int ring_stride = kSweepThreads * 3;     // float4 between the two slots
        const int L = pc.L;
        if (!__any_sync(0xffffffffu, active)) {
            // a warp of stand-in rows only takes part in the network's hand-off
            // (one call per march step, as the marching warps make)
            for (int kk = 5; kk < L + D; ++kk) guess.pipe(false, 1.0f, 0.0f, 1.0f, 1.0f, 0.0f, 1.0f);
            return;
        }
        const bool fb = mp.fallback != 0;
        Zone<R> zm2, zm1, z0;                 // zones k-2, k-1, k
        R dprev[5], qfprev[5], sLprev[5];
        R Fgprev[5], Fuprev2[5];
        double Gprev2[5];                     // FP32 path: widened face term of Fuprev2
        R rh[6];                              // FP32: raw densities of cells kk..kk-5
        bool qh1 = false, qh2 = false;        // the ring slots hold states of interfaces 1 / 2 steps back
        bool badprev = false;
        _Pragma("unroll") for (int v = 0; v < 5; ++v)
        {
            dprev[v] = qfprev[v] = sLprev[v] = Fgprev[v] = Fuprev2[v] = (R)0;
            Gprev2[v] = 0.0;
        }
        _Pragma("unroll") for (int i = 0; i < 6; ++i) rh[i] = (R)0;
        z0 = zm1 = zm2 = Zone<R>{};
        if constexpr (DIR != 0)
            for (int q = 0; q < kLearnedSlots - 1; ++q) stage<kLearnedSlots>(q);
        for (int kk = 0; kk < L + D; ++kk) {
            bool have = false;                // states of interface (kk-3)+1/2 traced this step
            R sLi[5], sRi[5];
            if (kk < L) {
                zm2 = zm1;
                zm1 = z0;
                if constexpr (DIR != 0) {
                    stage<kLearnedSlots>(kk + kLearnedSlots - 1);
                    z0 = zone_staged<kLearnedSlots, kLearnedSlots - 1>(kk, cnt);
                } else {
                    warm(kk + ENZO_PREFETCH_AHEAD);
                    z0 = zone<true>(kk, cnt);
                }
                if (WRAP) {
                    const int j = kk - pc.ng;
                    if (j >= 0 && j < 3) save(j, z0, (R)0);
                }
            }
            if (sizeof(R) == 4) {
                _Pragma("unroll") for (int i = 5; i > 0; --i) rh[i] = rh[i - 1];
                rh[0] = kk < L ? z0.r : (R)0;
            }
            if (kk < L && kk >= 2) {
                R dcur[5];
                _Pragma("unroll") for (int v = 0; v < 5; ++v) dcur[v] = limited_slope<R>(zv(zm2, v), zv(zm1, v), zv(z0, v));
                if (kk >= 3) {
                    R qfcur[5];
                    _Pragma("unroll") for (int v = 0; v < 5; ++v)
                        qfcur[v] = (R)0.5 * (zv(zm2, v) + zv(zm1, v)) - div6(dcur[v] - dprev[v]);
                    if (kk >= 4) {
                        // parabola of zone kk-2 (its edges: qfprev on the left, qfcur on the right)
                        R pL[5], pR[5], pd[5], p6[5];
                        _Pragma("unroll") for (int v = 0; v < 5; ++v) parabola<R>(zv(zm2, v), qfprev[v], qfcur[v], pL[v], pR[v], pd[v], p6[v]);
                        R sR[5], sLnew[5];
                        trace<R, -1>(pL, pR, pd, p6, zm2.u, zm2.c, dtdx, k, sR);
                        trace<R, +1>(pL, pR, pd, p6, zm2.u, zm2.c, dtdx, k, sLnew);
                        if (kk >= 5) {
                            // interface (kk-3)+1/2: left state from zone kk-3, right from kk-2
                            if (a.log) log_states(kk, sLprev, sR);
                            have = true;
                            _Pragma("unroll") for (int v = 0; v < 5; ++v)
                            {
                                sLi[v] = sLprev[v];
                                sRi[v] = sR[v];
                            }
                        }
                        _Pragma("unroll") for (int v = 0; v < 5; ++v) sLprev[v] = sLnew[v];
                    }
                    _Pragma("unroll") for (int v = 0; v < 5; ++v) qfprev[v] = qfcur[v];
                }
                _Pragma("unroll") for (int v = 0; v < 5; ++v) dprev[v] = dcur[v];
            }
            if (!have) {
                _Pragma("unroll") for (int v = 0; v < 5; ++v) sLi[v] = sRi[v] = (R)1;
            }
            // interface jj = kk - D: its states (from the ring slot of step kk - 2,
            // which then takes this step's states) and its starting guess;
            // every thread of the CTA reaches the guess at the same kk
            const R p0 = kk >= 5 ? (R)guess.pipe(have, (float)sLi[0], (float)sLi[1], (float)sLi[2], (float)sRi[0],
                                                 (float)sRi[1], (float)sRi[2])
                                 : (R)-1;
            const bool hj = qh2;
            qh2 = qh1;
            qh1 = have;
            float4 *slot = ring + (kk & 1) * ring_stride;
            R sL[5], sRj[5];
            {
                const float4 a0 = slot[0], a1 = slot[1], a2 = slot[2];
                sL[0] = a0.x; sL[1] = a0.y; sL[2] = a0.z; sL[3] = a0.w; sL[4] = a1.x;
                sRj[0] = a1.y; sRj[1] = a1.z; sRj[2] = a1.w; sRj[3] = a2.x; sRj[4] = a2.y;
                slot[0] = make_float4(sLi[0], sLi[1], sLi[2], sLi[3]);
                slot[1] = make_float4(sLi[4], sRi[0], sRi[1], sRi[2]);
                slot[2] = make_float4(sRi[3], sRi[4], 0.0f, 0.0f);
            }
            if (!hj) continue;
            const int jj = kk - D;            // Riemann problem at interface (jj-3)+1/2
            const RiemannOut<R> o = riemann<R>(sL[0], sL[1], sL[2], sRj[0], sRj[1], sRj[2], p0, k, cnt);
            if (active) {
                if (p0 > (R)0) cnt.guesses++;
                cnt.iters += (unsigned)o.iters;
                if (!o.conv) cnt.rare(ENZO_ST_NEWTON_NONCONV);
            }
            const R t1 = o.ustar >= (R)0 ? sL[3] : sRj[3];
            const R t2 = o.ustar >= (R)0 ? sL[4] : sRj[4];
            R Fg[5];
            phys_flux<R>(o.rho, o.u, o.p, t1, t2, k, Fg);
            if (jj >= 6) {
                // cell c = jj-3: does the Godunov update leave rho > 0?
                const int c = jj - 3;
                bool bad = false;
                if (fb) {
                    if (sizeof(R) == 8) {
                        bad = !(cell_update(rho_old(c), dtdx64, (double)Fgprev[0], (double)Fg[0]) > 0.0);
                    } else {
                        // FP32 screen; cells near zero are decided in FP64
                        const R rc = rh[3 + D];
                        const R rt = rc + dtdx * (Fgprev[0] - Fg[0]);
                        if (!(rt > (R)1e-3 * rc)) {
                            const double g0 = f2d_exact((float)(dtdx * Fgprev[0]));
                            const double g1 = f2d_exact((float)(dtdx * Fg[0]));
                            bad = !((rho_old(c) + g0) - g1 > 0.0);
                        }
                    }
                    if (bad && active) cnt.rare(ENZO_ST_HLL_CELLS);
                }
                // final flux at face (jj-4)+1/2
                R Fu1[5];
                if (badprev || bad) {
                    Counters quiet;
                    const Zone<R> za = zone<false>(jj - 4, quiet);
                    const Zone<R> zb = zone<false>(jj - 3, quiet);
                    hll_flux<R>(za, zb, k, Fu1);
                } else {
                    _Pragma("unroll") for (int v = 0; v < 5; ++v) Fu1[v] = Fgprev[v];
                }
                double G1[5];
                widen(Fu1, dtdx, G1);
                record(jj - 6, Fu1, G1);
                if (jj >= 7) update(jj - 4, Fuprev2, Fu1, dtdx64, Gprev2, G1, fb, cnt);
                _Pragma("unroll") for (int v = 0; v < 5; ++v)
                {
                    Fuprev2[v] = Fu1[v];
                    Gprev2[v] = G1[v];
                }
                badprev = bad;
            }
            _Pragma("unroll") for (int v = 0; v < 5; ++v) Fgprev[v] = Fg[v];
        }
        // last active cell L-4: its right face (L-4)+1/2 borders a ghost zone
        R Fu1[5];
        if (badprev) {
            Counters quiet;
            const Zone<R> za = zone<false>(L - 4, quiet);
            const Zone<R> zb = zone<false>(L - 3, quiet);
            hll_flux<R>(za, zb, k, Fu1);
        } else {
            _Pragma("unroll") for (int v = 0; v < 5; ++v) Fu1[v] = Fgprev[v];
        }
        double G1[5];
        widen(Fu1, dtdx, G1);
        record(pc.n, Fu1, G1);
        update(L - 4, Fuprev2, Fu1, dtdx64, Gprev2, G1, fb, cnt);
    }
};

__device__ __forceinline__ void warp_flush(unsigned long long *status, unsigned long long v, int word)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(status + word, v);
}

// Dynamic shared memory of a plain (not learned) sweep kernel: the FP32
// default kernels keep the raw values of their last five positions there, and
// in y and z sweeps three more staged ahead.  The x sweep keeps the ring at
// five: it depends on L1 keeping its rows' cache lines, and L1 gets what
// shared memory leaves (with eight slots the x sweep took 20.9 ms instead of
// 11.9 on the 4000-patch level).
template <class R, int THREADS, int EXT, int DIR>
__host__ __device__ constexpr int ring_bytes()
{
    return (sizeof(R) == 4 && EXT == 0) ? (DIR == 0 ? 5 : 8) * 5 * THREADS * (int)sizeof(double) : 0;
}

// Learned kernels: the network's shared memory (aligned to 128 bytes inside
// the dynamic block), then in y and z sweeps the staged loads' ring.
__host__ __device__ constexpr size_t learned_ring_offset() { return (sizeof(GuessSmem) + 127 + 127) & ~size_t(127); }
template <int DIR>
__host__ __device__ constexpr size_t learned_smem_bytes()
{
    return learned_ring_offset() + (DIR != 0 ? 3 * 5 * kSweepThreads * sizeof(double) : 0);
}

// Persistent sweep kernel: CTAs take (patch, 128-pencil tile) work items from a
// device counter until the batch is exhausted.  DIR is the sweep axis.
#ifndef ENZO_SWEEP_MIN_BLOCKS_FP32
#define ENZO_SWEEP_MIN_BLOCKS_FP32 4   // 128 registers per thread: 16 warps per SM
#endif
#ifndef ENZO_LEARNED_CTAS
#define ENZO_LEARNED_CTAS 3            // learned guess: CTAs per SM (TMEM holds 4 x 128 columns)
#endif
#ifndef ENZO_SWEEP_MIN_BLOCKS_DUAL
#define ENZO_SWEEP_MIN_BLOCKS_DUAL 3   // dual energy (FP32): 168 registers per thread
#endif
// LEARNED: the CTA evaluates the learned Newton guess on the tensor cores at
// every interface step, so all 128 threads march in step (threads without a
// pencil march a stand-in copy of the tile's first pencil and write nothing).
// REG: the batch has flux registers (hierarchy levels); the per-pencil register
// rows are then tracked, otherwise the recording compiles away.
template <class R, int DIR, bool LEARNED, int THREADS = kSweepThreads, bool REG = false, int EXT = 0>
__global__ void __launch_bounds__(THREADS, LEARNED ? ENZO_LEARNED_CTAS : (sizeof(R) == 4 ? (EXT == 2 ? ENZO_SWEEP_MIN_BLOCKS_DUAL : ENZO_SWEEP_MIN_BLOCKS_FP32 * 128 / THREADS) : 2))
    ppm_sweep_kernel(const __grid_constant__ SweepArgs a)
{
    constexpr int A1 = DIR == 0 ? 1 : 0, A2 = DIR == 2 ? 1 : 2;
    __shared__ int s_tile;
    // FP32: per-thread slots for the wrapped pencils' first three cells
    __shared__ float s_wrap[sizeof(R) == 4 ? 3 * (EXT == 2 ? 7 : 6) * THREADS : 1];
    extern __shared__ __align__(16) unsigned char dsmem[];
    // plain FP32 default kernels: the ring of raw values in dynamic shared memory
    double *uring = nullptr;
    if constexpr (ring_bytes<R, THREADS, EXT, DIR>() > 0 && !LEARNED) uring = reinterpret_cast<double *>(dsmem) + threadIdx.x;
    if constexpr (LEARNED && DIR != 0) uring = reinterpret_cast<double *>(dsmem + learned_ring_offset()) + threadIdx.x;
    Counters cnt;
    cnt.st = a.status;
    const Consts<R> k = make_consts<R>(a.mp);
    const double dt = a.dt_ptr ? *a.dt_ptr : a.dt;
    const int total = a.prefix[a.npatch];
    unsigned long long interfaces = 0;
    typename std::conditional<LEARNED, LearnedGuess, PlainGuess>::type guess;
    if constexpr (LEARNED) guess.setup(dsmem, a.mp.mlp, (float)a.mp.gamma, a.mp.mlp_gate);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.tile_counter, 1u);
        __syncthreads();
        const int tile = s_tile;
        __syncthreads();
        if (tile >= total) break;
        int lo = 0, hi = a.npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const enzo_patch P = a.patches[lo];
        int rlo[3], rhi[3];
        sweep_ranges(P, DIR, a.cover_mask, rlo, rhi);
        const int cnt1 = rhi[A1] - rlo[A1], cnt2 = rhi[A2] - rlo[A2];
        const int pen0 = (tile - a.prefix[lo]) * THREADS;
        const int pen = pen0 + (int)threadIdx.x;
        const bool valid = pen < cnt1 * cnt2;
        if (!LEARNED && !valid) continue;
        const int pe = valid ? pen : pen0;
        const int i1 = rlo[A1] + pe % cnt1, i2 = rlo[A2] + pe / cnt1;
        const int64_t N0 = P.n[0] + 2 * P.ng, N1 = P.n[1] + 2 * P.ng;
        const int64_t stride[3] = {1, N0, N0 * N1};
        Pencil pc;
        pc.base = P.off + (int64_t)i1 * stride[A1] + (int64_t)i2 * stride[A2];
        pc.sd = stride[DIR];
        pc.L = P.n[DIR] + 2 * P.ng;
        pc.ng = P.ng;
        pc.n = P.n[DIR];
        const double dtdx64 = dt / P.dx[DIR];
        const R dtdx = (R)dtdx64;
        if (valid) interfaces += (unsigned long long)(P.n[DIR] + 1);
        const unsigned key = (unsigned)lo * 7919u + (unsigned)pe;
        // flux register rows of this pencil (active transverse position only)
        double *reg_all = nullptr, *reg_bnd = nullptr;
        if (REG) {
            const int j1 = i1 - P.ng, j2 = i2 - P.ng;
            const int na1 = P.n[A1], na2 = P.n[A2];
            if (a.freg && valid && j1 >= 0 && j1 < na1 && j2 >= 0 && j2 < na2) {
                // components per face: five, six with dual energy
                constexpr int NC = EXT == 2 ? 6 : 5;
                int64_t oall = 0, obnd = 0;
                for (int d = 0; d < DIR; ++d) {
                    const int b1 = d == 0 ? 1 : 0, b2 = d == 2 ? 1 : 2;
                    oall += (int64_t)(P.n[d] + 1) * P.n[b1] * P.n[b2] * NC;
                    obnd += (int64_t)2 * P.n[b1] * P.n[b2] * NC;
                }
                const int64_t row = (int64_t)j2 * na1 + j1;
                if (P.freg_all >= 0) reg_all = a.freg + P.freg_all + oall + row * (P.n[DIR] + 1) * NC;
                if (P.freg_bnd >= 0) reg_bnd = a.freg + P.freg_bnd + obnd + row * 2 * NC;
            }
        }
        // a stand-in row counts none of its rare events (floors, FP64 E - KE)
        cnt.st = valid ? a.status : nullptr;
        if (P.flags & ENZO_PATCH_PERIODIC) {
            Marcher<R, true, DIR, REG, EXT> m{a, pc, k, valid, key, reg_all, reg_bnd, dt, s_wrap + threadIdx.x, uring};
            if constexpr (LEARNED) m.run_piped(dtdx, dtdx64, a.mp, cnt, guess);
            else m.run(dtdx, dtdx64, a.mp, cnt, guess);
        } else {
            Marcher<R, false, DIR, REG, EXT> m{a, pc, k, valid, key, reg_all, reg_bnd, dt, s_wrap + threadIdx.x, uring};
            if constexpr (LEARNED) m.run_piped(dtdx, dtdx64, a.mp, cnt, guess);
            else m.run(dtdx, dtdx64, a.mp, cnt, guess);
        }
    }
    if constexpr (LEARNED) {
        if (threadIdx.x == 0 && !guess.ok) atomicAdd(a.status + ENZO_ST_TIMEOUT, 1ull);
        guess.teardown();
    }
    warp_flush(a.status, interfaces, ENZO_ST_INTERFACES);
    warp_flush(a.status, cnt.iters, ENZO_ST_NEWTON_ITERS);
    warp_flush(a.status, cnt.restarts, ENZO_ST_GUESS_RESTARTS);
    warp_flush(a.status, cnt.guesses, ENZO_ST_GUESS_CALLS);
    if constexpr (EXT == 2) warp_flush(a.status, cnt.gep, ENZO_ST_GE_PRESSURE);
}

// CFL rate of Sec. 9 per active cell, max-reduced into *rate_bits.  A tile is
// kCflTile active cells of one patch; one thread finds the tile's patch and
// the block walks the tile's cells with 32-bit index arithmetic.
constexpr int kCflTile = kCflCells;

template <class R>
__global__ void __launch_bounds__(256) cfl_kernel(const __grid_constant__ CflArgs a)
{
    __shared__ double s_max[8];
    __shared__ int s_patch;
    const int total = a.prefix[a.npatch];
    double best = 0.0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = a.npatch;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (a.prefix[mid] <= tile) lo = mid; else hi = mid;
            }
            s_patch = lo;
        }
        __syncthreads();
        const int pi = s_patch;
        __syncthreads();
        const enzo_patch P = a.patches[pi];
        const int nx = P.n[0], ny = P.n[1];
        const int64_t ncell = (int64_t)nx * ny * P.n[2];
        const int64_t first = (int64_t)(tile - a.prefix[pi]) * kCflTile;
        const int64_t N0 = nx + 2 * P.ng, N1 = ny + 2 * P.ng;
        const double idx0 = 1.0 / P.dx[0], idx1 = 1.0 / P.dx[1], idx2 = 1.0 / P.dx[2];
        for (int t = threadIdx.x; t < kCflTile; t += blockDim.x) {
            const int64_t cell = first + t;
            if (cell >= ncell) break;
            const int64_t row = cell / nx;
            const int i = (int)(cell - row * nx);
            const int j = (int)(row % ny);
            const int kz = (int)(row / ny);
            const int64_t idx = P.off + (i + P.ng) + N0 * ((j + P.ng) + N1 * (int64_t)(kz + P.ng));
            if (sizeof(R) == 8) {
                double rho = a.U[0][idx];
                if (!(rho >= a.rho_floor)) rho = a.rho_floor;
                const double mx = a.U[1][idx], my = a.U[2][idx], mz = a.U[3][idx];
                const double ke = 0.5 * ((mx * mx + my * my) + mz * mz) / rho;
                double p = (a.gamma - 1.0) * (a.U[4][idx] - ke);
                if (!(p >= a.p_floor)) p = a.p_floor;
                const double c = sqrt(a.gamma * p / rho);
                const double r = ((c + fabs(mx / rho)) / P.dx[0] + (c + fabs(my / rho)) / P.dx[1]) +
                                 (c + fabs(mz / rho)) / P.dx[2];
                best = r > best ? r : best;
            } else {
                Counters quiet;
                Consts<float> k;
                k.gamma = (float)a.gamma;
                k.gm1 = (float)(a.gamma - 1.0);
                k.rho_floor = (float)a.rho_floor;
                k.p_floor = (float)a.p_floor;
                k.eta_eke = 0.05f;
                const Zone<float> z = prim_f<false>(a.U[0][idx], a.U[1][idx], a.U[2][idx], a.U[3][idx],
                                                    a.U[4][idx], k, quiet);
                const float r = ((z.c + fabsf(z.u)) * (float)idx0 + (z.c + fabsf(z.t1)) * (float)idx1) +
                                (z.c + fabsf(z.t2)) * (float)idx2;
                best = (double)r > best ? (double)r : best;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_down_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_max[w] > m ? s_max[w] : m;
        if (m > 0.0) atomicMax(a.rate_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// Standalone Riemann problems (one thread per interface).
template <class R>
__global__ void __launch_bounds__(256) riemann_kernel(const __grid_constant__ RiemannArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const Consts<R> k = make_consts<R>(a.mp);
    const R *rl = (const R *)a.rl, *ul = (const R *)a.ul, *pl = (const R *)a.pl;
    const R *rr = (const R *)a.rr, *ur = (const R *)a.ur, *pr = (const R *)a.pr;
    const R g = a.pguess ? ((const R *)a.pguess)[i] : (R)-1;
    Counters cnt;
    const RiemannOut<R> o = riemann<R>(rl[i], ul[i], pl[i], rr[i], ur[i], pr[i], g, k, cnt);
    if (a.pstar) ((R *)a.pstar)[i] = o.pstar;
    if (a.ustar) ((R *)a.ustar)[i] = o.ustar;
    if (a.rho) ((R *)a.rho)[i] = o.rho;
    if (a.u) ((R *)a.u)[i] = o.u;
    if (a.p) ((R *)a.p)[i] = o.p;
    if (a.iters) a.iters[i] = o.conv ? o.iters : -o.iters;
}

// Allow a plain kernel's ring (with its static shared memory the total can pass
// the 48 KB default), once per device.
template <class R, int DIR, int THREADS, bool REG>
cudaError_t ring_prepare(int dev)
{
    constexpr int bytes = ring_bytes<R, THREADS, 0, DIR>();
    if (bytes == 0) return cudaSuccess;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) dev = 0;
    if (done[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(ppm_sweep_kernel<R, DIR, false, THREADS, REG>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <class R>
int sweep_grid_for(int device)
{
    static int cached[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (cached[device]) return cached[device];
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ring_prepare<R, 0, kSweepThreads, false>(device);
    ring_prepare<R, 1, kSweepThreads, false>(device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ppm_sweep_kernel<R, 1, false>, kSweepThreads,
                                                  ring_bytes<R, kSweepThreads, 0, 1>());
    if (sms < 1) sms = 1;
    if (per < 1) per = 1;
    cached[device] = sms * per;
    return cached[device];
}

template <class R, int THREADS>
int tiled_grid(int device)
{
    static int cached[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (cached[device]) return cached[device];
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ring_prepare<R, 1, THREADS, false>(device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ppm_sweep_kernel<R, 1, false, THREADS>, THREADS,
                                                  ring_bytes<R, THREADS, 0, 1>());
    cached[device] = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    return cached[device];
}

template <class R, int THREADS>
cudaError_t launch_tiled(const SweepArgs &a, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const int grid = tiled_grid<R, THREADS>(dev);
    cudaError_t e = cudaSuccess;
    switch (a.dir) {
    case 0:
        e = ring_prepare<R, 0, THREADS, false>(dev);
        if (e == cudaSuccess)
            ppm_sweep_kernel<R, 0, false, THREADS><<<grid, THREADS, ring_bytes<R, THREADS, 0, 0>(), s>>>(a);
        break;
    case 1:
        e = ring_prepare<R, 1, THREADS, false>(dev);
        if (e == cudaSuccess)
            ppm_sweep_kernel<R, 1, false, THREADS><<<grid, THREADS, ring_bytes<R, THREADS, 0, 1>(), s>>>(a);
        break;
    default:
        e = ring_prepare<R, 2, THREADS, false>(dev);
        if (e == cudaSuccess)
            ppm_sweep_kernel<R, 2, false, THREADS><<<grid, THREADS, ring_bytes<R, THREADS, 0, 2>(), s>>>(a);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_sweep_dir(const SweepArgs &a, int grid, cudaStream_t s)
{
    if (a.mp.options & ENZO_OPT_DUAL) {
        // dual energy has its own instantiations too (with and without flux
        // registers), so the option kernels without it keep their registers;
        // their persistent grid follows their own occupancy
        static int cached[2][64] = {{0}};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64) dev = 0;
        const int withreg = a.freg ? 1 : 0;
        if (!cached[withreg][dev]) {
            int sms = 0, per = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (withreg)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, ppm_sweep_kernel<R, 0, false, kSweepThreads, true, 2>, kSweepThreads, 0);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, ppm_sweep_kernel<R, 0, false, kSweepThreads, false, 2>, kSweepThreads, 0);
            cached[withreg][dev] = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        }
        grid = cached[withreg][dev];
        if (a.freg) {
            switch (a.dir) {
            case 0: ppm_sweep_kernel<R, 0, false, kSweepThreads, true, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
            case 1: ppm_sweep_kernel<R, 1, false, kSweepThreads, true, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
            default: ppm_sweep_kernel<R, 2, false, kSweepThreads, true, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
            }
            return cudaGetLastError();
        }
        switch (a.dir) {
        case 0: ppm_sweep_kernel<R, 0, false, kSweepThreads, false, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
        case 1: ppm_sweep_kernel<R, 1, false, kSweepThreads, false, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
        default: ppm_sweep_kernel<R, 2, false, kSweepThreads, false, 2><<<grid, kSweepThreads, 0, s>>>(a); break;
        }
        return cudaGetLastError();
    }
    if (a.mp.options || a.mp.fallback == 2) {
        // the reconstruction options (and fallback mode 2) have their own
        // instantiations, so the default kernels stay as they are
        if (a.freg) {
            switch (a.dir) {
            case 0: ppm_sweep_kernel<R, 0, false, kSweepThreads, true, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            case 1: ppm_sweep_kernel<R, 1, false, kSweepThreads, true, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            default: ppm_sweep_kernel<R, 2, false, kSweepThreads, true, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            }
        } else {
            switch (a.dir) {
            case 0: ppm_sweep_kernel<R, 0, false, kSweepThreads, false, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            case 1: ppm_sweep_kernel<R, 1, false, kSweepThreads, false, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            default: ppm_sweep_kernel<R, 2, false, kSweepThreads, false, 1><<<grid, kSweepThreads, 0, s>>>(a); break;
            }
        }
        return cudaGetLastError();
    }
    constexpr int sx = ring_bytes<R, kSweepThreads, 0, 0>(), syz = ring_bytes<R, kSweepThreads, 0, 1>();
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaError_t e = cudaSuccess;
        if (a.freg) {
            if (e == cudaSuccess) e = ring_prepare<R, 0, kSweepThreads, true>(dev);
            if (e == cudaSuccess) e = ring_prepare<R, 1, kSweepThreads, true>(dev);
            if (e == cudaSuccess) e = ring_prepare<R, 2, kSweepThreads, true>(dev);
        } else {
            if (e == cudaSuccess) e = ring_prepare<R, 0, kSweepThreads, false>(dev);
            if (e == cudaSuccess) e = ring_prepare<R, 1, kSweepThreads, false>(dev);
            if (e == cudaSuccess) e = ring_prepare<R, 2, kSweepThreads, false>(dev);
        }
        if (e != cudaSuccess) return e;
    }
    if (a.freg) {
        switch (a.dir) {
        case 0: ppm_sweep_kernel<R, 0, false, kSweepThreads, true><<<grid, kSweepThreads, sx, s>>>(a); break;
        case 1: ppm_sweep_kernel<R, 1, false, kSweepThreads, true><<<grid, kSweepThreads, syz, s>>>(a); break;
        default: ppm_sweep_kernel<R, 2, false, kSweepThreads, true><<<grid, kSweepThreads, syz, s>>>(a); break;
        }
        return cudaGetLastError();
    }
    switch (a.dir) {
    case 0: ppm_sweep_kernel<R, 0, false><<<grid, kSweepThreads, sx, s>>>(a); break;
    case 1: ppm_sweep_kernel<R, 1, false><<<grid, kSweepThreads, syz, s>>>(a); break;
    default: ppm_sweep_kernel<R, 2, false><<<grid, kSweepThreads, syz, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace enzo
