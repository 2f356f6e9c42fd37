/*
 * ppm_oracle.c -- plain, slow, FP64 CPU oracle for the directionally split,
 * direct-Eulerian PPM hydrodynamics sweep of the Enzo method paper.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header or constant with the CUDA library; the two meet only through the
 * seeded inputs both are given.
 *
 * What it follows (paper sections; CW84 = Colella & Woodward 1984, which the
 * paper defers to for the reconstruction formulas):
 *   Sec. 2.1      conserved variables, total energy density E = e + rho v^2/2,
 *                 ideal-gas EOS e = p/(gamma-1).
 *   Sec. 3        patches with 3 ghost layers, Dirichlet ghost zones filled once
 *                 per step; periodic external boundary (Sec. 3.1, case 4).
 *   Sec. 4.1      split 1-D conservative equations and their Eulerian difference
 *                 form (mass, momentum, energy); parabolic interpolant q(x) with
 *                 Delta q and q6; interface values + monotonicity (CW84 1.6-1.10);
 *                 averages over the u-c, u, u+c domains of dependence and the
 *                 characteristic left/right states (CW84 1.12, 3.6, 3.7);
 *                 operator splitting with transverse velocities advected.
 *   Sec. 4.1.2    two-shock Riemann solver (Newton iteration on p*), HLL, and
 *                 the HLL fallback for cells that go to negative density.
 *   Sec. 9        hydro CFL timestep, harmonic form over axes, min over level.
 *
 * Readings where the paper is silent or garbled:
 *   - update sign: U_j += dt/dx (F_{j-1/2} - F_{j+1/2}), momentum uses rho^n v^n
 *     (the printed difference equations carry a flipped sign and rho^{n+1}).
 *   - E is the total energy DENSITY; specific values appear only in fluxes.
 *   - floors: rho >= rho_floor, p >= p_floor on cell primitives, traced
 *     states, Newton iterates and star states.
 *   - characteristic reference state is the u+c (left) / u-c (right) domain
 *     average when that wave moves toward the interface, else the edge value;
 *     the Lagrangian sound speed C is taken from the reference state.
 *   - Newton stops when the residual |u*_R - u*_L| <= tol (|u_L|+|u_R|+c_L+c_R)
 *     or p* stops moving; capped at newton_max updates.
 *   - rarefaction sampling at x/t = 0 blends star and outer states linearly in
 *     the head/tail speed fraction (two-shock star density).
 *   - HLL fallback uses first-order (cell-centred) states with Davis speeds;
 *     both faces of a bad cell are re-fluxed and every cell touching a re-fluxed
 *     face is re-updated from its old state (conservation is kept).
 *   - sweep order: x,y,z on even steps, z,y,x on odd steps.
 *   - ghosts filled once per step; the first sweep also updates the transverse
 *     ghost layers, the second the remaining axis' ghost layers, the third only
 *     active cells.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * No FMA contraction: every product and sum is rounded separately, in the
 * association written in the source.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double gamma;
    double rho_floor;
    double p_floor;
    double newton_tol;
    int32_t newton_max;
    int32_t fallback;     /* 1: HLL re-flux of cells that reach rho <= 0; 2: also of cells that
                             reach E - KE <= 0 (tested as 2 rho E - |m|^2 <= 0) */
    int32_t solver;       /* interface fluxes: 0 two-shock (Sec. 4.1.2), 1 HLL, 2 HLLC */
    int32_t options;      /* bit 0 contact steepening, bit 1 flattening, bit 2 diffusive flux,
                             bit 3 dual energy (a gas-energy field rides along, see pencil_step) */
} or_params;

typedef struct {
    int64_t interfaces;      /* Riemann problems solved */
    int64_t newton_iters;    /* Newton updates summed over interfaces */
    int64_t newton_nonconv;  /* interfaces that hit the iteration cap */
    int64_t hll_cells;       /* cells that triggered the HLL fallback */
    int64_t neg_after;       /* cells still failing the fallback's test after it */
    int64_t rho_floor_hits;  /* cell primitives raised to rho_floor */
    int64_t p_floor_hits;    /* cell primitives raised to p_floor */
    int64_t ge_pressure;     /* dual energy: zones whose pressure came from the gas energy */
} or_stats;

/* ----------------------------------------------------------------------- */
/* Two-shock Riemann solver (Sec. 4.1.2): both waves treated as shocks.     */
/* ----------------------------------------------------------------------- */

typedef struct {
    double pstar, ustar;           /* star-region pressure and velocity */
    double rho_sL, rho_sR;         /* star densities either side of the contact */
    double rho, u, p;              /* state at x/t = 0 */
    int iters;
    int converged;
} or_riemann_out;

/* Lagrangian shock speed W_s and star velocity for one side at pressure ps. */
static void shock_side(double ps, double rho, double p, double C, double gamma,
                       double *W, double *Z)
{
    double g = (gamma + 1.0) / (2.0 * gamma);
    double rad = 1.0 + g * (ps / p - 1.0);
    if (rad < 1e-6) rad = 1e-6;
    *W = C * sqrt(rad);
    /* slope magnitude of the shock curve, dp/du = 2 W^3 / (W^2 + C^2) */
    *Z = 2.0 * (*W) * (*W) * (*W) / ((*W) * (*W) + C * C);
    (void)rho;
}

/* The acoustic (linearised two-shock) starting guess for p*. */
static double plain_guess(double rl, double ul, double pl, double rr, double ur, double pr,
                          double gamma, double p_floor)
{
    double CL = sqrt(gamma * pl * rl);
    double CR = sqrt(gamma * pr * rr);
    double p0 = (CR * pl + CL * pr + CL * CR * (ul - ur)) / (CL + CR);
    return p0 > p_floor ? p0 : p_floor;
}

/* Newton iteration on f(p*) = u*_R(p*) - u*_L(p*) = 0 from guess p0.
 * Converged when |f| <= tol * (|u_L| + |u_R| + c_L + c_R), checked before each
 * update, or when the update no longer moves p* (pinned at the floor).
 * Returns the number of Newton updates taken. */
static int newton(double rl, double ul, double pl, double rr, double ur, double pr,
                  double p0, const or_params *P, double *pstar, int *conv)
{
    double CL = sqrt(P->gamma * pl * rl);
    double CR = sqrt(P->gamma * pr * rr);
    double uscale = (fabs(ul) + fabs(ur)) + (sqrt(P->gamma * pl / rl) + sqrt(P->gamma * pr / rr));
    double ps = p0 > P->p_floor ? p0 : P->p_floor;
    int it;
    *conv = 0;
    for (it = 0; it < P->newton_max; ++it) {
        double WL, ZL, WR, ZR;
        shock_side(ps, rl, pl, CL, P->gamma, &WL, &ZL);
        shock_side(ps, rr, pr, CR, P->gamma, &WR, &ZR);
        double usL = ul - (ps - pl) / WL;
        double usR = ur + (ps - pr) / WR;
        double f = usR - usL;
        if (fabs(f) <= P->newton_tol * uscale) { *conv = 1; break; }
        double pn = ps - ZL * ZR * f / (ZL + ZR);
        if (!(pn > P->p_floor)) pn = P->p_floor;
        if (pn == ps) { *conv = 1; break; }
        ps = pn;
    }
    *pstar = ps;
    return it;
}

/* Full two-shock solve and sampling at x/t = 0.  If p_guess > 0 it is used as
 * the starting guess; a guess that does not converge is retried from the
 * plain guess (the plain solver still decides the answer). */
static void riemann_twoshock(double rl, double ul, double pl, double rr, double ur, double pr,
                             double p_guess, const or_params *P, or_riemann_out *o)
{
    const double gamma = P->gamma;
    double ps;
    int conv;
    int it;
    if (p_guess > 0.0) {
        it = newton(rl, ul, pl, rr, ur, pr, p_guess, P, &ps, &conv);
        if (!conv) {
            int it2 = newton(rl, ul, pl, rr, ur, pr,
                             plain_guess(rl, ul, pl, rr, ur, pr, gamma, P->p_floor), P, &ps, &conv);
            it += it2;
        }
    } else {
        it = newton(rl, ul, pl, rr, ur, pr,
                    plain_guess(rl, ul, pl, rr, ur, pr, gamma, P->p_floor), P, &ps, &conv);
    }
    o->iters = it;
    o->converged = conv;

    double CL = sqrt(gamma * pl * rl);
    double CR = sqrt(gamma * pr * rr);
    double WL, ZL, WR, ZR;
    shock_side(ps, rl, pl, CL, gamma, &WL, &ZL);
    shock_side(ps, rr, pr, CR, gamma, &WR, &ZR);
    double usL = ul - (ps - pl) / WL;
    double usR = ur + (ps - pr) / WR;
    double us = (ZL * usL + ZR * usR) / (ZL + ZR);
    /* Lagrangian jump condition across each shock: [1/rho] = -[p] / W^2 */
    double rsL = 1.0 / (1.0 / rl - (ps - pl) / (WL * WL));
    double rsR = 1.0 / (1.0 / rr - (ps - pr) / (WR * WR));
    if (!(rsL > P->rho_floor)) rsL = P->rho_floor;
    if (!(rsR > P->rho_floor)) rsR = P->rho_floor;
    o->pstar = ps; o->ustar = us; o->rho_sL = rsL; o->rho_sR = rsR;

    /* sample the self-similar solution at x/t = 0 */
    double rho, u, p;
    if (us >= 0.0) {                                   /* contact moves right: left side */
        if (ps > pl) {                                 /* left shock */
            double S = ul - WL / rl;
            if (S >= 0.0) { rho = rl; u = ul; p = pl; }
            else          { rho = rsL; u = us; p = ps; }
        } else {                                       /* left rarefaction */
            double cl = sqrt(gamma * pl / rl);
            double cs = sqrt(gamma * ps / rsL);
            double Sh = ul - cl;
            double St = us - cs;
            if (Sh >= 0.0)      { rho = rl; u = ul; p = pl; }
            else if (St <= 0.0) { rho = rsL; u = us; p = ps; }
            else {
                double f = -Sh / (St - Sh);
                rho = rl + f * (rsL - rl);
                u = ul + f * (us - ul);
                p = pl + f * (ps - pl);
            }
        }
    } else {                                           /* contact moves left: right side */
        if (ps > pr) {
            double S = ur + WR / rr;
            if (S <= 0.0) { rho = rr; u = ur; p = pr; }
            else          { rho = rsR; u = us; p = ps; }
        } else {
            double cr = sqrt(gamma * pr / rr);
            double cs = sqrt(gamma * ps / rsR);
            double Sh = ur + cr;
            double St = us + cs;
            if (Sh <= 0.0)      { rho = rr; u = ur; p = pr; }
            else if (St >= 0.0) { rho = rsR; u = us; p = ps; }
            else {
                double f = Sh / (Sh - St);
                rho = rr + f * (rsR - rr);
                u = ur + f * (us - ur);
                p = pr + f * (ps - pr);
            }
        }
    }
    o->rho = rho; o->u = u; o->p = p;
}

/* Physical flux of the split 1-D equations for a primitive state (Sec. 4.1).
 * Components: mass, normal momentum, transverse momenta 1 and 2, total energy. */
static void phys_flux(double rho, double u, double p, double ut1, double ut2, double gamma,
                      double F[5])
{
    double gm1inv = 1.0 / (gamma - 1.0);
    double mflux = rho * u;
    F[0] = mflux;
    F[1] = mflux * u + p;
    F[2] = mflux * ut1;
    F[3] = mflux * ut2;
    double eint = p * gm1inv;
    double ke = 0.5 * rho * ((u * u + ut1 * ut1) + ut2 * ut2);
    F[4] = u * ((eint + ke) + p);
}

/* HLL flux with Davis signal-speed estimates (Sec. 4.1.2, fallback). */
static void hll_flux(double rl, double ul, double pl, double t1l, double t2l,
                     double rr, double ur, double pr, double t1r, double t2r,
                     double gamma, double F[5])
{
    double gm1inv = 1.0 / (gamma - 1.0);
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double SL = ul - cl < ur - cr ? ul - cl : ur - cr;
    double SR = ul + cl > ur + cr ? ul + cl : ur + cr;
    double FL[5], FR[5];
    phys_flux(rl, ul, pl, t1l, t2l, gamma, FL);
    phys_flux(rr, ur, pr, t1r, t2r, gamma, FR);
    if (SL >= 0.0) { memcpy(F, FL, sizeof FL); return; }
    if (SR <= 0.0) { memcpy(F, FR, sizeof FR); return; }
    double UL[5] = { rl, rl * ul, rl * t1l, rl * t2l,
                     pl * gm1inv + 0.5 * rl * ((ul * ul + t1l * t1l) + t2l * t2l) };
    double UR[5] = { rr, rr * ur, rr * t1r, rr * t2r,
                     pr * gm1inv + 0.5 * rr * ((ur * ur + t1r * t1r) + t2r * t2r) };
    for (int c = 0; c < 5; ++c)
        F[c] = (SR * FL[c] - SL * FR[c] + SL * SR * (UR[c] - UL[c])) / (SR - SL);
}

/* HLLC flux (Sec. 4.1.2 names HLLC among the Riemann solvers; Toro's
 * three-wave form): the Davis signal speeds of hll_flux, the contact speed
 *   S* = (pR - pL + rL uL (SL - uL) - rR uR (SR - uR)) / (rL (SL - uL) - rR (SR - uR)),
 * and on side K the star state
 *   U*K = rK (SK - uK)/(SK - S*) [1, S*, t1K, t2K, EK/rK + (S* - uK)(S* + pK/(rK (SK - uK)))]
 * with flux F*K = FK + SK (U*K - UK).  The interface takes FL (0 <= SL),
 * F*L (SL < 0 <= S*), F*R (S* < 0 < SR) or FR (SR <= 0). */
static void hllc_flux(double rl, double ul, double pl, double t1l, double t2l,
                      double rr, double ur, double pr, double t1r, double t2r,
                      double gamma, double F[5])
{
    double gm1inv = 1.0 / (gamma - 1.0);
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double SL = ul - cl < ur - cr ? ul - cl : ur - cr;
    double SR = ul + cl > ur + cr ? ul + cl : ur + cr;
    double FL[5], FR[5];
    phys_flux(rl, ul, pl, t1l, t2l, gamma, FL);
    phys_flux(rr, ur, pr, t1r, t2r, gamma, FR);
    if (SL >= 0.0) { memcpy(F, FL, sizeof FL); return; }
    if (SR <= 0.0) { memcpy(F, FR, sizeof FR); return; }
    double ml = rl * (SL - ul), mr = rr * (SR - ur);
    double Ss = ((pr - pl) + ul * ml - ur * mr) / (ml - mr);
    int left = Ss >= 0.0;
    double r = left ? rl : rr, u = left ? ul : ur, p = left ? pl : pr;
    double t1 = left ? t1l : t1r, t2 = left ? t2l : t2r, S = left ? SL : SR, m = left ? ml : mr;
    const double *FK = left ? FL : FR;
    double E = p * gm1inv + 0.5 * r * ((u * u + t1 * t1) + t2 * t2);
    double UK[5] = { r, r * u, r * t1, r * t2, E };
    double chi = m / (S - Ss);
    double Us[5] = { chi, chi * Ss, chi * t1, chi * t2, chi * (E / r + (Ss - u) * (Ss + p / m)) };
    for (int c = 0; c < 5; ++c) F[c] = FK[c] + S * (Us[c] - UK[c]);
}

/* ----------------------------------------------------------------------- */
/* One pencil: primitives -> PPM -> tracing -> Riemann -> flux -> update.   */
/* ----------------------------------------------------------------------- */

/* Pencil arrays, length L = n + 2 ng.  var index: 0 rho, 1 u_n, 2 p, 3 u_t1, 4 u_t2 */
typedef struct {
    int L;
    double *U[6];       /* conserved along the pencil: rho, m_n, m_t1, m_t2, E (and, with
                           dual energy, the gas energy ge = rho eps) */
    double *q[6];       /* primitives (index 5: specific internal energy eps) */
    double *c;          /* zone sound speed */
    double *dq[6];      /* limited slopes */
    double *qf[6];      /* unlimited interface values q_{s+1/2} */
    double *qL[6], *qR[6], *d[6], *q6[6];   /* monotone parabola per zone */
    double *sL[6];      /* left state at interface s+1/2 (from zone s) */
    double *sR[6];      /* right state at interface s-1/2 (from zone s) */
    double *F[6];       /* flux at interface s+1/2 */
    double *Uold[6];
    double *eta;        /* contact-steepening weight per zone */
    double *flat;       /* flattening weight per zone */
    double *uface;      /* dual energy: velocity at interface s+1/2 */
    double *buf;
} pencil;

static int pencil_alloc(pencil *pc, int L)
{
    int narr = 6 * 13 + 4;
    pc->L = L;
    pc->buf = (double *)calloc((size_t)narr * (size_t)L, sizeof(double));
    if (!pc->buf) return -1;
    double *b = pc->buf;
    for (int v = 0; v < 6; ++v) {
        pc->U[v] = b; b += L;  pc->q[v] = b; b += L;  pc->dq[v] = b; b += L;
        pc->qf[v] = b; b += L; pc->qL[v] = b; b += L; pc->qR[v] = b; b += L;
        pc->d[v] = b; b += L;  pc->q6[v] = b; b += L; pc->sL[v] = b; b += L;
        pc->sR[v] = b; b += L; pc->F[v] = b; b += L;  pc->Uold[v] = b; b += L;
        b += L;  /* spare */
    }
    pc->c = b; b += L;
    pc->eta = b; b += L;
    pc->flat = b; b += L;
    pc->uface = b;
    return 0;
}

/* Optional dissipation of the PPM reconstruction (Sec. 4.1 calls them
 * optional and defers to CW84; its formulas, on a uniform grid):
 *
 * Contact steepening (density only) of zone s, from the discontinuity
 * detector  eta~ = -(D_{s+1} - D_{s-1}) / (6 (rho_{s+1} - rho_{s-1})),
 * D_s = rho_{s+1} - 2 rho_s + rho_{s-1}, set to 0 where D_{s+1} D_{s-1} >= 0,
 * where |rho_{s+1} - rho_{s-1}| < 0.01 min(rho_{s+1}, rho_{s-1}), or where the
 * pressure jump is large against the density jump (a shock, not a contact:
 * |p_{s+1} - p_{s-1}| / min(p) > 0.1 gamma |rho_{s+1} - rho_{s-1}| / min(rho));
 * weight eta = max(0, min(20 (eta~ - 0.05), 1)).
 *
 * Flattening of zone s near strong shocks: w = 1 where the flow compresses
 * (u_{s-1} > u_{s+1}) and |p_{s+1} - p_{s-1}| > 0.33 min(p_{s+1}, p_{s-1});
 * weight f = w max(0, min(1, 10 ((p_{s+1} - p_{s-1}) / (p_{s+2} - p_{s-2}) - 0.75)))
 * (f = w where p_{s+2} = p_{s-2}).  Reading: CW84 also takes the max with the
 * upstream neighbour's weight, which needs pressures three zones away; that
 * max is dropped so every stencil fits the three ghost zones. */
static void dissipation_weights(pencil *pc, const or_params *P)
{
    const int L = pc->L;
    const double *r = pc->q[0], *u = pc->q[1], *p = pc->q[2];
    for (int s = 0; s < L; ++s) { pc->eta[s] = 0.0; pc->flat[s] = 0.0; }
    for (int s = 2; s < L - 2; ++s) {
        if (P->options & 1) {
            double Dm = r[s] - 2.0 * r[s - 1] + r[s - 2];
            double Dp = r[s + 2] - 2.0 * r[s + 1] + r[s];
            double dr = r[s + 1] - r[s - 1];
            double rmin = r[s + 1] < r[s - 1] ? r[s + 1] : r[s - 1];
            double pmin = p[s + 1] < p[s - 1] ? p[s + 1] : p[s - 1];
            double et = 0.0;
            int contact = fabs(p[s + 1] - p[s - 1]) / pmin <= 0.1 * P->gamma * (fabs(dr) / rmin);
            if (Dm * Dp < 0.0 && fabs(dr) >= 0.01 * rmin && contact) et = -(Dp - Dm) / (6.0 * dr);
            double e = 20.0 * (et - 0.05);
            pc->eta[s] = e < 0.0 ? 0.0 : (e > 1.0 ? 1.0 : e);
        }
        if (P->options & 2) {
            double dp1 = p[s + 1] - p[s - 1], dp2 = p[s + 2] - p[s - 2];
            double pmin = p[s + 1] < p[s - 1] ? p[s + 1] : p[s - 1];
            if (u[s - 1] - u[s + 1] > 0.0 && fabs(dp1) > 0.33 * pmin) {
                double f = 1.0;
                if (dp2 != 0.0) {
                    f = 10.0 * (dp1 / dp2 - 0.75);
                    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
                }
                pc->flat[s] = f;
            }
        }
    }
}

/* Domain-of-dependence average of zone parabola over its right (toward=+1) or
 * left (toward=-1) fraction sig of the zone (CW84 1.12). */
static double avg_right(double qR, double d, double q6, double sig)
{
    return qR - (0.5 * sig) * (d - (1.0 - sig * (2.0 / 3.0)) * q6);
}
static double avg_left(double qL, double d, double q6, double sig)
{
    return qL + (0.5 * sig) * (d + (1.0 - sig * (2.0 / 3.0)) * q6);
}

/* Characteristic state at an edge of zone s (CW84 3.6/3.7, Sec. 4.1).
 * side = +1: left state of the interface at the zone's right edge (waves with
 * lambda > 0 reach it); side = -1: right state of the interface at its left edge. */
static void trace_state(const pencil *pc, int s, int side, double dtdx, const or_params *P,
                        int nv, double out[6])
{
    const double gamma = P->gamma;
    double u = pc->q[1][s], c = pc->c[s];
    double lam[3] = { u - c, u, u + c };        /* -, 0, + waves */
    int reach[3];
    double I[3][6];
    for (int w = 0; w < 3; ++w) {
        reach[w] = side > 0 ? lam[w] > 0.0 : lam[w] < 0.0;
        double sig = side > 0 ? lam[w] * dtdx : -lam[w] * dtdx;
        for (int v = 0; v < nv; ++v) {
            if (side > 0) I[w][v] = avg_right(pc->qR[v][s], pc->d[v][s], pc->q6[v][s], sig);
            else          I[w][v] = avg_left(pc->qL[v][s], pc->d[v][s], pc->q6[v][s], sig);
        }
    }
    /* reference state: the fastest wave moving toward the interface */
    int wref = side > 0 ? 2 : 0;
    double rref, uref, pref;
    if (reach[wref]) { rref = I[wref][0]; uref = I[wref][1]; pref = I[wref][2]; }
    else if (side > 0) { rref = pc->qR[0][s]; uref = pc->qR[1][s]; pref = pc->qR[2][s]; }
    else { rref = pc->qL[0][s]; uref = pc->qL[1][s]; pref = pc->qL[2][s]; }
    if (!(rref > P->rho_floor)) rref = P->rho_floor;
    if (!(pref > P->p_floor)) pref = P->p_floor;
    double C = sqrt(gamma * pref * rref);
    double bp = 0.0, bm = 0.0, b0 = 0.0;
    if (reach[2]) bp = -(0.5 / C) * ((uref - I[2][1]) + (pref - I[2][2]) / C);
    if (reach[0]) bm = (0.5 / C) * ((uref - I[0][1]) - (pref - I[0][2]) / C);
    if (reach[1]) b0 = (pref - I[1][2]) / (C * C) + 1.0 / rref - 1.0 / I[1][0];
    double p = pref + (C * C) * (bp + bm);
    double un = uref + C * (bp - bm);
    double tau = 1.0 / rref - ((bp + bm) + b0);
    double rho = 1.0 / tau;
    if (!(rho > P->rho_floor)) rho = P->rho_floor;
    if (!(p > P->p_floor)) p = P->p_floor;
    out[0] = rho; out[1] = un; out[2] = p;
    for (int v = 3; v < nv; ++v) {      /* transverse velocities and eps: passive */
        if (reach[1]) out[v] = I[1][v];
        else out[v] = side > 0 ? pc->qR[v][s] : pc->qL[v][s];
    }
}

/* Does updated cell s fail the fallback test?  rho <= 0, and with mode 2 also
 * a non-positive internal energy, 2 rho E - |m|^2 <= 0 (Sec. 4.1.2 names negative
 * densities or energies; the paper's trigger is the density). */
static int fallback_fails(const pencil *pc, int s, const or_params *P)
{
    const double rho = pc->U[0][s];
    if (!(rho > 0.0)) return 1;
    if (P->fallback == 2) {
        const double m2 = (pc->U[1][s] * pc->U[1][s] + pc->U[2][s] * pc->U[2][s]) + pc->U[3][s] * pc->U[3][s];
        if (!((2.0 * rho) * pc->U[4][s] - m2 > 0.0)) return 1;
    }
    return 0;
}

/* Advance one pencil (already gathered into pc->U) by the split update along it.
 * Active cells are [ng, L-ng).  Returns nothing; pc->U is overwritten. */
/* Dual energy (Sec. 4.1.1: eta1 = 1e-3, eta2 = 0.1), the reading taken here:
 *   pressure: from E - KE, or from the gas energy ge where E - KE < eta1 E;
 *   ge = rho eps is carried with eps = ge / rho reconstructed, traced and
 *   upwinded (by the sign of u*) like a transverse velocity, its flux the mass
 *   flux times eps, and the source -p (u_{j+1/2} - u_{j-1/2}) dt/dx with the
 *   zone pressure at the start of the sweep and the Godunov interface
 *   velocities (the printed update's flux-difference sign is taken as garbled,
 *   as for the other fields); faces re-fluxed by the HLL fallback carry the HLL
 *   mass flux times the upwind zone eps and the mean of the two zone velocities;
 *   after the update ge is reset to E - KE where that exceeds eta2 times the
 *   largest E of the cell and its two pencil neighbours. */
static void pencil_step(pencil *pc, int ng, double dtdx, const or_params *P, or_stats *st)
{
    const int L = pc->L;
    const double gamma = P->gamma;
    const int dual = (P->options & 8) != 0;
    const int nv = dual ? 6 : 5;
    /* (a) primitives, Sec. 2.1 / 4.1 */
    for (int s = 0; s < L; ++s) {
        double rho = pc->U[0][s];
        if (!(rho >= P->rho_floor)) { rho = P->rho_floor; st->rho_floor_hits++; }
        double mn = pc->U[1][s], m1 = pc->U[2][s], m2 = pc->U[3][s], E = pc->U[4][s];
        double ke = 0.5 * ((mn * mn + m1 * m1) + m2 * m2) / rho;
        double p;
        if (dual && E - ke < 1e-3 * E) { p = (gamma - 1.0) * pc->U[5][s]; st->ge_pressure++; }
        else p = (gamma - 1.0) * (E - ke);
        if (!(p >= P->p_floor)) { p = P->p_floor; st->p_floor_hits++; }
        pc->q[0][s] = rho;
        pc->q[1][s] = mn / rho;
        pc->q[2][s] = p;
        pc->q[3][s] = m1 / rho;
        pc->q[4][s] = m2 / rho;
        if (dual) pc->q[5][s] = pc->U[5][s] / rho;
        pc->c[s] = sqrt(gamma * p / rho);
    }
    dissipation_weights(pc, P);
    /* (b) limited slopes, CW84 1.7-1.8 */
    for (int v = 0; v < nv; ++v) {
        const double *q = pc->q[v];
        for (int s = 1; s < L - 1; ++s) {
            double dl = q[s] - q[s - 1];
            double dr = q[s + 1] - q[s];
            double dc = 0.5 * (q[s + 1] - q[s - 1]);
            double r = 0.0;
            if (dl * dr > 0.0) {
                double a = fabs(dc), b = 2.0 * fabs(dl), e = 2.0 * fabs(dr);
                double m = a < b ? a : b;
                m = m < e ? m : e;
                r = dc >= 0.0 ? m : -m;
            }
            pc->dq[v][s] = r;
        }
        /* interface value between zones s and s+1, CW84 1.6 (uniform grid) */
        for (int s = 1; s < L - 2; ++s)
            pc->qf[v][s] = 0.5 * (q[s] + q[s + 1]) - (pc->dq[v][s + 1] - pc->dq[v][s]) / 6.0;
        /* (c) monotone parabola for zones 2..L-3, CW84 1.10, after the optional
         * contact steepening (density) and flattening */
        for (int s = 2; s < L - 2; ++s) {
            double qs = q[s], ql = pc->qf[v][s - 1], qr = pc->qf[v][s];
            if (v == 0 && pc->eta[s] > 0.0) {
                double e = pc->eta[s];
                ql = ql * (1.0 - e) + (q[s - 1] + 0.5 * pc->dq[v][s - 1]) * e;
                qr = qr * (1.0 - e) + (q[s + 1] - 0.5 * pc->dq[v][s + 1]) * e;
            }
            if (pc->flat[s] > 0.0) {
                double f = pc->flat[s];
                ql = f * qs + (1.0 - f) * ql;
                qr = f * qs + (1.0 - f) * qr;
            }
            if ((qr - qs) * (qs - ql) <= 0.0) {
                ql = qs; qr = qs;
            } else {
                double d = qr - ql;
                double q6 = 6.0 * (qs - 0.5 * (ql + qr));
                if (d * q6 > d * d) ql = 3.0 * qs - 2.0 * qr;
                else if (-(d * d) > d * q6) qr = 3.0 * qs - 2.0 * ql;
            }
            pc->qL[v][s] = ql;
            pc->qR[v][s] = qr;
            pc->d[v][s] = qr - ql;
            pc->q6[v][s] = 6.0 * (qs - 0.5 * (ql + qr));
        }
    }
    /* (d,e) characteristic states at the interfaces that bound active cells */
    for (int s = ng - 1; s <= L - ng - 1; ++s) {
        double st6[6];
        trace_state(pc, s, +1, dtdx, P, nv, st6);
        for (int v = 0; v < nv; ++v) pc->sL[v][s] = st6[v];
    }
    for (int s = ng; s <= L - ng; ++s) {
        double st6[6];
        trace_state(pc, s, -1, dtdx, P, nv, st6);
        for (int v = 0; v < nv; ++v) pc->sR[v][s] = st6[v];
    }
    /* (f,g) Riemann problem and flux at interface s+1/2, s = ng-1 .. L-ng-1 */
    for (int s = ng - 1; s <= L - ng - 1; ++s) {
        double rl = pc->sL[0][s], ul = pc->sL[1][s], pl = pc->sL[2][s];
        double rr = pc->sR[0][s + 1], ur = pc->sR[1][s + 1], pr = pc->sR[2][s + 1];
        double F[6];
        st->interfaces++;
        if (P->solver == 1) {
            hll_flux(rl, ul, pl, pc->sL[3][s], pc->sL[4][s], rr, ur, pr, pc->sR[3][s + 1], pc->sR[4][s + 1],
                     gamma, F);
        } else if (P->solver == 2) {
            hllc_flux(rl, ul, pl, pc->sL[3][s], pc->sL[4][s], rr, ur, pr, pc->sR[3][s + 1], pc->sR[4][s + 1],
                      gamma, F);
        } else {
            or_riemann_out o;
            riemann_twoshock(rl, ul, pl, rr, ur, pr, -1.0, P, &o);
            st->newton_iters += o.iters;
            if (!o.converged) st->newton_nonconv++;
            double t1 = o.ustar >= 0.0 ? pc->sL[3][s] : pc->sR[3][s + 1];
            double t2 = o.ustar >= 0.0 ? pc->sL[4][s] : pc->sR[4][s + 1];
            phys_flux(o.rho, o.u, o.p, t1, t2, gamma, F);
            if (dual) {
                F[5] = F[0] * (o.ustar >= 0.0 ? pc->sL[5][s] : pc->sR[5][s + 1]);
                pc->uface[s] = o.u;
            }
        }
        if (P->options & 4) {
            /* diffusive flux (CW84; optional in Sec. 4.1): 0.1 max(0, u_s - u_{s+1})
             * times the jump of the conserved state across the interface, the
             * conserved states rebuilt from the zone primitives */
            double du = pc->q[1][s] - pc->q[1][s + 1];
            if (du > 0.0) {
                double nu = 0.1 * du;
                double Ua[6], Ub[6];
                for (int z = 0; z < 2; ++z) {
                    double *Uz = z ? Ub : Ua;
                    int c = s + z;
                    double r = pc->q[0][c], u = pc->q[1][c], pz = pc->q[2][c];
                    double t1 = pc->q[3][c], t2 = pc->q[4][c];
                    Uz[0] = r; Uz[1] = r * u; Uz[2] = r * t1; Uz[3] = r * t2;
                    Uz[4] = pz / (gamma - 1.0) + 0.5 * r * ((u * u + t1 * t1) + t2 * t2);
                    if (dual) Uz[5] = r * pc->q[5][c];
                }
                for (int v = 0; v < nv; ++v) F[v] = F[v] + nu * (Ua[v] - Ub[v]);
            }
        }
        for (int v = 0; v < nv; ++v) pc->F[v][s] = F[v];
    }
    /* (h) conservative update of active cells, FP64 (and the gas energy) */
    for (int v = 0; v < nv; ++v)
        for (int s = 0; s < L; ++s) pc->Uold[v][s] = pc->U[v][s];
    for (int s = ng; s < L - ng; ++s) {
        for (int v = 0; v < 5; ++v)
            pc->U[v][s] = pc->Uold[v][s] + dtdx * (pc->F[v][s - 1] - pc->F[v][s]);
        if (dual)
            pc->U[5][s] = (pc->Uold[5][s] + dtdx * (pc->F[5][s - 1] - pc->F[5][s])) -
                          dtdx * pc->q[2][s] * (pc->uface[s] - pc->uface[s - 1]);
    }
    if (P->fallback) {
        /* HLL fallback (Sec. 4.1.2): re-flux both faces of each cell with rho <= 0
         * (mode 2: or E - KE <= 0) */
        int nbad = 0;
        for (int s = ng; s < L - ng; ++s) if (fallback_fails(pc, s, P)) nbad++;
        if (nbad) {
            char *mark = (char *)calloc((size_t)L, 1);       /* mark[s]: interface s+1/2 */
            for (int s = ng; s < L - ng; ++s)
                if (fallback_fails(pc, s, P)) { mark[s - 1] = 1; mark[s] = 1; st->hll_cells++; }
            for (int s = ng - 1; s <= L - ng - 1; ++s) {
                if (!mark[s]) continue;
                double F[5];
                hll_flux(pc->q[0][s], pc->q[1][s], pc->q[2][s], pc->q[3][s], pc->q[4][s],
                         pc->q[0][s + 1], pc->q[1][s + 1], pc->q[2][s + 1], pc->q[3][s + 1], pc->q[4][s + 1],
                         gamma, F);
                for (int v = 0; v < 5; ++v) pc->F[v][s] = F[v];
                if (dual) {
                    pc->F[5][s] = F[0] * (F[0] >= 0.0 ? pc->q[5][s] : pc->q[5][s + 1]);
                    pc->uface[s] = 0.5 * (pc->q[1][s] + pc->q[1][s + 1]);
                }
            }
            for (int s = ng; s < L - ng; ++s) {
                if (!mark[s - 1] && !mark[s]) continue;
                for (int v = 0; v < 5; ++v)
                    pc->U[v][s] = pc->Uold[v][s] + dtdx * (pc->F[v][s - 1] - pc->F[v][s]);
                if (dual)
                    pc->U[5][s] = (pc->Uold[5][s] + dtdx * (pc->F[5][s - 1] - pc->F[5][s])) -
                                  dtdx * pc->q[2][s] * (pc->uface[s] - pc->uface[s - 1]);
                if (fallback_fails(pc, s, P)) st->neg_after++;
            }
            free(mark);
        }
    }
    if (dual) {
        /* gas energy resynchronised where E - KE is reliable (Sec. 4.1.1, the selection of e):
         * E - KE above eta2 times the largest total energy of the cell and its two neighbours
         * along the pencil, all after the update (the ghost neighbours keep their values) */
        for (int s = ng; s < L - ng; ++s) {
            double rho = pc->U[0][s], E = pc->U[4][s];
            if (!(rho > 0.0)) continue;
            double ke = 0.5 * ((pc->U[1][s] * pc->U[1][s] + pc->U[2][s] * pc->U[2][s]) +
                               pc->U[3][s] * pc->U[3][s]) / rho;
            double emax = pc->U[4][s - 1];
            if (E > emax) emax = E;
            if (pc->U[4][s + 1] > emax) emax = pc->U[4][s + 1];
            if (E - ke > 0.1 * emax) pc->U[5][s] = E - ke;
        }
    }
}

/* ----------------------------------------------------------------------- */
/* Grid-level operations on one patch.                                      */
/* Field arrays: 5 x (nz+2g)(ny+2g)(nx+2g) doubles, x fastest.              */
/* ----------------------------------------------------------------------- */

static int64_t idx3(const int N[3], int i, int j, int k)
{
    return (int64_t)i + (int64_t)N[0] * ((int64_t)j + (int64_t)N[1] * (int64_t)k);
}

/* Periodic ghost fill of every ghost cell, edges and corners included (Sec. 3.1). */
void or_fill_periodic(double *U0, double *U1, double *U2, double *U3, double *U4,
                      const int32_t n[3], int32_t ng)
{
    double *U[5] = { U0, U1, U2, U3, U4 };
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    for (int k = 0; k < N[2]; ++k)
        for (int j = 0; j < N[1]; ++j)
            for (int i = 0; i < N[0]; ++i) {
                int a[3] = { i, j, k };
                int ghost = 0;
                int src[3];
                for (int d = 0; d < 3; ++d) {
                    int x = a[d] - ng;
                    if (x < 0 || x >= n[d]) ghost = 1;
                    x %= n[d];
                    if (x < 0) x += n[d];
                    src[d] = x + ng;
                }
                if (!ghost) continue;
                int64_t dst = idx3(N, i, j, k), sidx = idx3(N, src[0], src[1], src[2]);
                for (int v = 0; v < 5; ++v) U[v][dst] = U[v][sidx];
            }
}

/* External boundaries of a single grid (Sec. 3.1: reflecting, outflow or
 * periodic).  Axes are filled in turn, x then y then z, each over the full
 * extent of the other two axes, so edges and corners take both conditions.
 * Layer g = 1..ng outside the face:
 *   periodic:   the active cell n - g (left) / g - 1 (right) of the same axis
 *               (taken modulo n);
 *   reflecting: the mirror image about the face, active cell g - 1 (left) /
 *               n - g (right), with the momentum along the axis negated
 *               (needs n >= ng along that axis);
 *   outflow:    the boundary cell itself (zero gradient). */
void or_fill_boundary(double *U0, double *U1, double *U2, double *U3, double *U4,
                      const int32_t n[3], int32_t ng, const int32_t bc[3])
{
    double *U[5] = { U0, U1, U2, U3, U4 };
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    for (int d = 0; d < 3; ++d) {
        for (int k = 0; k < N[2]; ++k)
            for (int j = 0; j < N[1]; ++j)
                for (int i = 0; i < N[0]; ++i) {
                    int a[3] = { i, j, k };
                    int x = a[d] - ng;                    /* active index along d */
                    if (x >= 0 && x < n[d]) continue;
                    int src;
                    double sign = 1.0;
                    if (bc[d] == 0) {                     /* periodic */
                        src = ((x % n[d]) + n[d]) % n[d];
                    } else if (bc[d] == 1) {              /* reflecting */
                        src = x < 0 ? -x - 1 : 2 * n[d] - x - 1;
                        sign = -1.0;
                    } else {                              /* outflow */
                        src = x < 0 ? 0 : n[d] - 1;
                    }
                    int b[3] = { i, j, k };
                    b[d] = src + ng;
                    int64_t dst = idx3(N, i, j, k), sidx = idx3(N, b[0], b[1], b[2]);
                    for (int v = 0; v < 5; ++v) U[v][dst] = U[v][sidx];
                    U[1 + d][dst] = sign * U[1 + d][sidx];
                }
    }
}

/* Level timestep (Sec. 9): dt = cfl / max over active cells of
 * sum_d (c_s + |v_d|) / dx_d, with c_s = sqrt(gamma p / rho), a = 1.
 * Returns the max of the sum (the caller divides), so patches can be combined. */
double or_cfl_rate(const double *U0, const double *U1, const double *U2, const double *U3,
                   const double *U4, const int32_t n[3], int32_t ng, const double dx[3],
                   const or_params *P)
{
    const double *U[5] = { U0, U1, U2, U3, U4 };
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    double best = 0.0;
    for (int k = ng; k < ng + n[2]; ++k)
        for (int j = ng; j < ng + n[1]; ++j)
            for (int i = ng; i < ng + n[0]; ++i) {
                int64_t x = idx3(N, i, j, k);
                double rho = U[0][x];
                if (!(rho >= P->rho_floor)) rho = P->rho_floor;
                double mx = U[1][x], my = U[2][x], mz = U[3][x];
                double ke = 0.5 * ((mx * mx + my * my) + mz * mz) / rho;
                double p = (P->gamma - 1.0) * (U[4][x] - ke);
                if (!(p >= P->p_floor)) p = P->p_floor;
                double c = sqrt(P->gamma * p / rho);
                double r = ((c + fabs(mx / rho)) / dx[0] + (c + fabs(my / rho)) / dx[1])
                           + (c + fabs(mz / rho)) / dx[2];
                if (r > best) best = r;
            }
    return best;
}

/* One split sweep along axis dir over the pencils whose transverse storage
 * coordinates lie in [lo[a], hi[a]) for the two other axes a. */
/* One split sweep along axis dir over the pencils whose transverse storage
 * coordinates lie in [lo[a], hi[a]) for the two other axes a.  If fout is not
 * NULL, the final face fluxes of every pencil whose transverse coordinates are
 * active go to fout[((j2 * n[a1] + j1) * (n[dir] + 1) + f) * 5 + v], with j1, j2
 * the active transverse indices and f the face left of active cell f (f = n[dir]
 * is the right face of the last cell); v follows the pencil order rho, m_n,
 * m_t1, m_t2, E. */
int or_sweep_fluxes(double *U0, double *U1, double *U2, double *U3, double *U4,
                    const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                    const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats,
                    double *fout);

int or_sweep(double *U0, double *U1, double *U2, double *U3, double *U4,
             const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
             const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats)
{
    return or_sweep_fluxes(U0, U1, U2, U3, U4, n, ng, dx, dir, dt, lo, hi, P, stats, NULL);
}

static int sweep_ge(double *U0, double *U1, double *U2, double *U3, double *U4, double *ge,
                    const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                    const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats,
                    double *fout);

int or_sweep_fluxes(double *U0, double *U1, double *U2, double *U3, double *U4,
                    const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                    const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats,
                    double *fout)
{
    return sweep_ge(U0, U1, U2, U3, U4, NULL, n, ng, dx, dir, dt, lo, hi, P, stats, fout);
}

/* As or_sweep_fluxes, with the gas-energy field ge of the dual-energy option:
 * fout then holds six components per face, the sixth the gas-energy flux
 * (the mass flux times the upwind eps, Sec. 4.1.1), at
 * fout[((j2 * n[a1] + j1) * (n[dir] + 1) + f) * 6 + v]. */
int or_sweep_fluxes_dual(double *U0, double *U1, double *U2, double *U3, double *U4, double *ge,
                         const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                         const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats,
                         double *fout)
{
    if (!ge || !(P->options & 8)) return -2;
    return sweep_ge(U0, U1, U2, U3, U4, ge, n, ng, dx, dir, dt, lo, hi, P, stats, fout);
}

/* As or_sweep, with the gas-energy field ge of the dual-energy option (may be
 * NULL when the option is off). */
int or_sweep_dual(double *U0, double *U1, double *U2, double *U3, double *U4, double *ge,
                  const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                  const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats)
{
    return sweep_ge(U0, U1, U2, U3, U4, ge, n, ng, dx, dir, dt, lo, hi, P, stats, NULL);
}

static int sweep_ge(double *U0, double *U1, double *U2, double *U3, double *U4, double *ge,
                    const int32_t n[3], int32_t ng, const double dx[3], int32_t dir, double dt,
                    const int32_t lo[3], const int32_t hi[3], const or_params *P, or_stats *stats,
                    double *fout)
{
    double *U[5] = { U0, U1, U2, U3, U4 };
    if ((P->options & 8) && !ge) return -2;
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    int a1 = dir == 0 ? 1 : 0;           /* transverse axes in increasing order */
    int a2 = dir == 2 ? 1 : 2;
    int L = N[dir];
    double dtdx = dt / dx[dir];
    int64_t stride[3] = { 1, N[0], (int64_t)N[0] * N[1] };
    int cnt1 = hi[a1] - lo[a1], cnt2 = hi[a2] - lo[a2];
    int64_t npen = (int64_t)cnt1 * cnt2;
    int err = 0;
    or_stats tot = { 0 };
#pragma omp parallel
    {
        pencil pc;
        or_stats st = { 0 };
        int ok = pencil_alloc(&pc, L) == 0;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (int64_t t = 0; t < npen; ++t) {
            if (!ok) continue;
            int i1 = lo[a1] + (int)(t % cnt1), i2 = lo[a2] + (int)(t / cnt1);
            int64_t base = (int64_t)i1 * stride[a1] + (int64_t)i2 * stride[a2];
            /* conserved order along the pencil: rho, m_n, m_t1, m_t2, E */
            int mi[5] = { 0, 1 + dir, 1 + a1, 1 + a2, 4 };
            for (int s = 0; s < L; ++s)
                for (int v = 0; v < 5; ++v) pc.U[v][s] = U[mi[v]][base + s * stride[dir]];
            if (ge)
                for (int s = 0; s < L; ++s) pc.U[5][s] = ge[base + s * stride[dir]];
            pencil_step(&pc, ng, dtdx, P, &st);
            for (int s = ng; s < L - ng; ++s)
                for (int v = 0; v < 5; ++v) U[mi[v]][base + s * stride[dir]] = pc.U[v][s];
            if (ge)
                for (int s = ng; s < L - ng; ++s) ge[base + s * stride[dir]] = pc.U[5][s];
            if (fout) {
                int j1 = i1 - ng, j2 = i2 - ng;
                if (j1 >= 0 && j1 < n[a1] && j2 >= 0 && j2 < n[a2]) {
                    const int nf = ge ? 6 : 5;    /* with ge: the gas-energy flux too */
                    double *o = fout + ((int64_t)j2 * n[a1] + j1) * (int64_t)(n[dir] + 1) * nf;
                    for (int f = 0; f <= n[dir]; ++f)
                        for (int v = 0; v < nf; ++v) o[f * nf + v] = pc.F[v][ng - 1 + f];
                }
            }
        }
        if (ok) free(pc.buf);
#pragma omp critical
        {
            tot.interfaces += st.interfaces; tot.newton_iters += st.newton_iters;
            tot.newton_nonconv += st.newton_nonconv; tot.hll_cells += st.hll_cells;
            tot.neg_after += st.neg_after; tot.rho_floor_hits += st.rho_floor_hits;
            tot.p_floor_hits += st.p_floor_hits; tot.ge_pressure += st.ge_pressure;
        }
    }
    if (stats) {
        stats->interfaces += tot.interfaces; stats->newton_iters += tot.newton_iters;
        stats->newton_nonconv += tot.newton_nonconv; stats->hll_cells += tot.hll_cells;
        stats->neg_after += tot.neg_after; stats->rho_floor_hits += tot.rho_floor_hits;
        stats->p_floor_hits += tot.p_floor_hits; stats->ge_pressure += tot.ge_pressure;
    }
    return err ? -1 : 0;
}

/* Sweep order of step `step`: x,y,z when even, z,y,x when odd. */
void or_sweep_order(int32_t step, int32_t order[3])
{
    if (step % 2 == 0) { order[0] = 0; order[1] = 1; order[2] = 2; }
    else               { order[0] = 2; order[1] = 1; order[2] = 0; }
}

/* One full step of a periodic patch with the dual-energy gas-energy field ge:
 * ghost fill of U and ge, then the three split sweeps with transverse coverage. */
int or_step_periodic_dual(double *U0, double *U1, double *U2, double *U3, double *U4, double *ge,
                          const int32_t n[3], int32_t ng, const double dx[3], double dt,
                          int32_t step, const or_params *P, or_stats *stats)
{
    int32_t order[3];
    or_sweep_order(step, order);
    or_fill_periodic(U0, U1, U2, U3, U4, n, ng);
    or_fill_periodic(ge, ge, ge, ge, ge, n, ng);
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    int done[3] = { 0, 0, 0 };
    for (int q = 0; q < 3; ++q) {
        int d = order[q];
        int32_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (done[a]) { lo[a] = ng; hi[a] = ng + n[a]; }
            else         { lo[a] = 0;  hi[a] = N[a]; }
        }
        int r = or_sweep_dual(U0, U1, U2, U3, U4, ge, n, ng, dx, d, dt, lo, hi, P, stats);
        if (r) return r;
        done[d] = 1;
    }
    return 0;
}

/* One full step of a single grid with external boundaries bc[3] (as in
 * or_fill_boundary): ghost fill, then the three split sweeps with transverse
 * coverage. */
int or_step_boundary(double *U0, double *U1, double *U2, double *U3, double *U4,
                     const int32_t n[3], int32_t ng, const double dx[3], double dt,
                     int32_t step, const int32_t bc[3], const or_params *P, or_stats *stats)
{
    int32_t order[3];
    or_sweep_order(step, order);
    or_fill_boundary(U0, U1, U2, U3, U4, n, ng, bc);
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    int done[3] = { 0, 0, 0 };
    for (int q = 0; q < 3; ++q) {
        int d = order[q];
        int32_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (done[a]) { lo[a] = ng; hi[a] = ng + n[a]; }
            else         { lo[a] = 0;  hi[a] = N[a]; }
        }
        int r = or_sweep(U0, U1, U2, U3, U4, n, ng, dx, d, dt, lo, hi, P, stats);
        if (r) return r;
        done[d] = 1;
    }
    return 0;
}

/* One full step of a periodic patch: ghost fill, then three split sweeps with
 * the transverse coverage that lets ghosts be filled once per step. */
int or_step_periodic(double *U0, double *U1, double *U2, double *U3, double *U4,
                     const int32_t n[3], int32_t ng, const double dx[3], double dt,
                     int32_t step, const or_params *P, or_stats *stats)
{
    int32_t order[3];
    or_sweep_order(step, order);
    or_fill_periodic(U0, U1, U2, U3, U4, n, ng);
    int N[3] = { n[0] + 2 * ng, n[1] + 2 * ng, n[2] + 2 * ng };
    int done[3] = { 0, 0, 0 };
    for (int q = 0; q < 3; ++q) {
        int d = order[q];
        int32_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            /* axes already swept only need their active range; others need ghosts too */
            if (done[a]) { lo[a] = ng; hi[a] = ng + n[a]; }
            else         { lo[a] = 0;  hi[a] = N[a]; }
        }
        int r = or_sweep(U0, U1, U2, U3, U4, n, ng, dx, d, dt, lo, hi, P, stats);
        if (r) return r;
        done[d] = 1;
    }
    return 0;
}

/* Batched Riemann solves (test/parity entry): plain guess when pguess is NULL. */
void or_riemann_batch(int64_t count, const double *rl, const double *ul, const double *pl,
                      const double *rr, const double *ur, const double *pr,
                      const double *pguess, const or_params *P,
                      double *pstar, double *ustar, double *rho_face, double *u_face,
                      double *p_face, int32_t *iters)
{
    for (int64_t i = 0; i < count; ++i) {
        or_riemann_out o;
        riemann_twoshock(rl[i], ul[i], pl[i], rr[i], ur[i], pr[i],
                         pguess ? pguess[i] : -1.0, P, &o);
        if (pstar) pstar[i] = o.pstar;
        if (ustar) ustar[i] = o.ustar;
        if (rho_face) rho_face[i] = o.rho;
        if (u_face) u_face[i] = o.u;
        if (p_face) p_face[i] = o.p;
        if (iters) iters[i] = o.converged ? o.iters : -o.iters;
    }
}

/* Batched fluxes (solver 0 two-shock, 1 HLL, 2 HLLC) for given left/right
 * primitive states. */
void or_flux_batch(int64_t count, int32_t solver, const double *rl, const double *ul,
                   const double *pl, const double *t1l, const double *t2l,
                   const double *rr, const double *ur, const double *pr,
                   const double *t1r, const double *t2r, const or_params *P, double *F)
{
    for (int64_t i = 0; i < count; ++i) {
        double f[5];
        if (solver == 1) {
            hll_flux(rl[i], ul[i], pl[i], t1l[i], t2l[i], rr[i], ur[i], pr[i], t1r[i], t2r[i],
                     P->gamma, f);
        } else if (solver == 2) {
            hllc_flux(rl[i], ul[i], pl[i], t1l[i], t2l[i], rr[i], ur[i], pr[i], t1r[i], t2r[i],
                      P->gamma, f);
        } else {
            or_riemann_out o;
            riemann_twoshock(rl[i], ul[i], pl[i], rr[i], ur[i], pr[i], -1.0, P, &o);
            double t1 = o.ustar >= 0.0 ? t1l[i] : t1r[i];
            double t2 = o.ustar >= 0.0 ? t2l[i] : t2r[i];
            phys_flux(o.rho, o.u, o.p, t1, t2, P->gamma, f);
        }
        for (int v = 0; v < 5; ++v) F[5 * i + v] = f[v];
    }
}

/* Run one pencil of length L (conserved input U[v][s], v = rho, m_n, m_t1,
 * m_t2, E) and expose its intermediate arrays, each 5*L doubles laid out
 * [v][s]: monotone edge values qL, qR, curvature q6, traced left state at
 * s+1/2 (sL), traced right state at s-1/2 (sR), flux at s+1/2 (F), and the
 * updated conserved pencil (Unew).  For pinning the steps one by one. */
int or_pencil_debug(int32_t L, int32_t ng, const double *Uin, double dtdx, const or_params *P,
                    double *qL, double *qR, double *q6, double *sL, double *sR, double *F,
                    double *Unew, or_stats *stats)
{
    pencil pc;
    or_stats st = { 0 };
    if (pencil_alloc(&pc, L)) return -1;
    for (int v = 0; v < 5; ++v)
        for (int s = 0; s < L; ++s) pc.U[v][s] = Uin[v * L + s];
    pencil_step(&pc, ng, dtdx, P, &st);
    for (int v = 0; v < 5; ++v)
        for (int s = 0; s < L; ++s) {
            int64_t o = (int64_t)v * L + s;
            if (qL) qL[o] = pc.qL[v][s];
            if (qR) qR[o] = pc.qR[v][s];
            if (q6) q6[o] = pc.q6[v][s];
            if (sL) sL[o] = pc.sL[v][s];
            if (sR) sR[o] = pc.sR[v][s];
            if (F) F[o] = pc.F[v][s];
            if (Unew) Unew[o] = pc.U[v][s];
        }
    if (stats) *stats = st;
    free(pc.buf);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the pencil loops (timing only: results do not depend on it). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
