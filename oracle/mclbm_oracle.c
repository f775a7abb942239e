/*
 * Plain FP64 CPU oracle of the improved two-component pseudopotential
 * lattice Boltzmann method (Sedahmed, Coelho, Warda, arXiv:2111.08666).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference against
 * which the CUDA library is checked.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it; the
 * product path never does.  It shares no code, header or table with the
 * CUDA library.
 *
 * Every function below follows one step of Sec. 2 in the paper's order and
 * notation, written for clarity, not speed: plain loops over nodes, sums in
 * a fixed index order (i = 0..8, sigma = 1, 2), IEEE double precision, built
 * with -ffp-contract=off.  OpenMP only splits the independent per-node loops
 * over rows, so results do not depend on the thread count.
 *
 * Readings of passages the paper leaves open (each is also fixed by a test):
 *  - Eq. 7 is taken as nu = cs^2 (tau - 1/2); the relaxation-time/viscosity
 *    pairs printed in Sec. 4.1 (tau 3.5 -> nu 1, tau 0.62 -> nu 0.04) only
 *    hold with the minus sign.
 *  - The velocity entering Eqs. 2 and 11 is the barycentric velocity of
 *    Eq. 8 shifted by half the total force, u = (sum_s j_s + F/2)/rho, as
 *    the (1 - 1/(2 tau_s)) prefactor of Eq. 1 requires for the momentum
 *    balance; vel_shift = 0 selects the literal unshifted form.
 *  - Eq. 14 sums over ordered pairs sigma != sigma_bar:
 *    P = (rho1 + rho2)/3 + (G/3) rho1 rho2.
 *  - Eq. 26 (component 1 at the outlet): the missing f_{3,6,7} after
 *    streaming equal their pre-collision values of the previous step, which
 *    makes them constant from initialisation (array d5, rows 0-2).
 *  - Eq. 27 (component 2 at the inlet, Set-2) is read the same way: the
 *    missing f_{1,5,8} are constant from initialisation (d5, rows 3-5).
 *  - Eq. 28 (component 2 at the inlet, Set-3): the missing f_{1,5,8} keep
 *    their own post-collision values.
 *  - The three treatments of Sec. 2.3, selected by bc_set:
 *      Set-1: Zou-He for both components at both ends, the other component's
 *             density (rho_in2 at the inlet, rho_out1 at the outlet) fixed too;
 *      Set-2: Zou-He for component 1 at the inlet and component 2 at the
 *             outlet; Eq. 26 at the outlet and Eq. 27 at the inlet for the
 *             other component;
 *      Set-3 (the paper's, the default): as Set-2 but Eq. 28 at the inlet.
 *  - Multiple-relaxation-time collision (mrt = 1; not in the paper, which
 *    uses the SRT of Eq. 1): Eq. 1 with the scalar 1/tau_s replaced by a
 *    relaxation matrix diagonal in the moment basis of Lallemand and Luo,
 *      f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M S^F,
 *    S = diag(1, s_e, s_eps, w, s_q, w, s_q, w, w) with w = 1/tau_s (Eq. 6)
 *    on the momentum and stress moments; s_e, s_eps, s_q fixed rates, or 0
 *    for "w" (then the operator is the SRT one exactly), s_q = -1 for
 *    8 (2 - w) / (8 - w), which with s_e = s_eps = w puts half-way
 *    bounce-back walls exactly half-way for Poiseuille flow at any tau.
 *  - Zou-He (Eqs. 18-25) prescribes zero tangential velocity; u_x follows
 *    from the prescribed density.  Directions whose source lies beyond the
 *    open x ends are "missing"; directions whose source is solid are filled
 *    by half-way bounce-back first and count as known.
 *  - The improved virtual solid density (Eq. 17) is recomputed every step
 *    from the current densities; out-of-domain neighbours are excluded.
 *  - Solid nodes carry no populations (zeros) and enter no sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 lattice of Sec. 2.1: e_i and w_i, i = 0..8. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* index of the opposite direction, e_opp(i) = -e_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;  /* lattice sound speed squared, c_s = 1/sqrt(3) */
static const double INV_CS2 = 3.0;     /* 1 / c_s^2 */
static const double INV_CS4 = 9.0;     /* 1 / c_s^4 */

typedef struct {
    int nx, ny;
    double nu1, nu2;        /* kinematic viscosities (Eq. 7 reading above) */
    double g_coh, g_ads;    /* cohesion (Eq. 13) and adhesion (Eq. 15) */
    double gx, gy;          /* body acceleration: F^b = rho^sigma g */
    double rho_in1;         /* Set-3 inlet density of component 1 */
    double rho_out2;        /* Set-3 outlet density of component 2 */
    int open_x;             /* 1: Set-3 at x=0 and x=nx-1; 0: periodic x */
    int periodic_y;         /* 1: periodic y; 0: rows 0 and ny-1 are solid */
    int vel_shift;          /* 1: u^eq carries +F/2 (default reading) */
    int bc_set;             /* 1, 2 or 3 (0 counts as 3): treatment of Sec. 2.3 */
    double rho_in2;         /* Set-1 inlet density of component 2 */
    double rho_out1;        /* Set-1 outlet density of component 1 */
    int mrt;                /* 0: SRT collision of Eq. 1; 1: MRT (see header) */
    int pad2;
    double s_e, s_eps, s_q; /* MRT rates of the energy, energy-square and heat-flux moments */
} oracle_params;

#define IDX(p, y, x) ((size_t)(y) * (size_t)(p)->nx + (size_t)(x))
#define FIDX(p, c, i, y, x) \
    ((((size_t)(c) * 9 + (size_t)(i)) * (size_t)(p)->ny + (size_t)(y)) * (size_t)(p)->nx + (size_t)(x))

/* Wrap or reject a coordinate; returns 0 if the neighbour is outside. */
static int resolve(const oracle_params *p, int *x, int *y) {
    if (*y < 0 || *y >= p->ny) {
        if (!p->periodic_y) return 0;
        *y = (*y + p->ny) % p->ny;
    }
    if (*x < 0 || *x >= p->nx) {
        if (p->open_x) return 0;
        *x = (*x + p->nx) % p->nx;
    }
    return 1;
}

/* Eq. 2: second-order equilibrium with velocity u. */
void oracle_feq(double rho, double ux, double uy, double *feq) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = WGT[i] * rho *
                 (1.0 + eu * INV_CS2 + 0.5 * (eu * eu) * INV_CS4 - 0.5 * uu * INV_CS2);
    }
}

/* Eq. 11: S_i = w_i [ (e_i - u)/cs^2 + (e_i . u) e_i / cs^4 ] . F */
void oracle_source(double ux, double uy, double fx, double fy, double *s) {
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double ax = (EX[i] - ux) * INV_CS2 + eu * EX[i] * INV_CS4;
        double ay = (EY[i] - uy) * INV_CS2 + eu * EY[i] * INV_CS4;
        s[i] = WGT[i] * (ax * fx + ay * fy);
    }
}

/* Moment basis of the MRT collision (Lallemand and Luo): rows rho, e, eps,
 * j_x, q_x, j_y, q_y, p_xx, p_xy in the direction order of EX/EY; the rows
 * are orthogonal, so M^-1 = M^T diag(1 / |row|^2). */
static const double MRT_M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},        {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},     {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},     {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static const double MRT_NORM2[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};

/* f* of one component at one node by the MRT operator (header): the
 * deviation from equilibrium and the source are taken to moment space with
 * M, weighted by S and (I - S/2), and brought back with M^-1. */
static void mrt_collide(const oracle_params *p, double omega, const double *f, const double *feq,
                        const double *src, double *out) {
    double sq = p->s_q < 0.0 ? 8.0 * (2.0 - omega) / (8.0 - omega) : (p->s_q > 0.0 ? p->s_q : omega);
    double rate[9] = {1.0, p->s_e > 0.0 ? p->s_e : omega, p->s_eps > 0.0 ? p->s_eps : omega, omega, sq,
                      omega, sq, omega, omega};
    double g[9];
    for (int k = 0; k < 9; ++k) {
        double dev = 0.0, sm = 0.0;
        for (int i = 0; i < 9; ++i) {
            dev += MRT_M[k][i] * (f[i] - feq[i]);
            sm += MRT_M[k][i] * src[i];
        }
        g[k] = rate[k] * dev - (1.0 - 0.5 * rate[k]) * sm;
    }
    for (int i = 0; i < 9; ++i) {
        double back = 0.0;
        for (int k = 0; k < 9; ++k) back += MRT_M[k][i] * g[k] / MRT_NORM2[k];
        out[i] = f[i] - back;
    }
}

/* Eq. 14 with ordered pairs sigma != sigma_bar. */
double oracle_pressure(double g_coh, double rho1, double rho2) {
    return CS2 * (rho1 + rho2) + CS2 / 2.0 * g_coh * (rho1 * rho2 + rho2 * rho1);
}

/* Initial state: f = f^eq(rho^sigma, u = 0) on fluid nodes, taken as the
 * post-collision populations of step 0; d5 [6][ny] records component 1's
 * f_{3,6,7} on the outlet column (Eq. 26, rows 0-2) and component 2's
 * f_{1,5,8} on the inlet column (Eq. 27, rows 3-5). */
void oracle_init(const oracle_params *p, const uint8_t *solid,
                 const double *rho1, const double *rho2, double *f, double *d5) {
    size_t n = (size_t)p->nx * p->ny;
    memset(f, 0, 18 * n * sizeof(double));
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            if (solid[IDX(p, y, x)]) continue;
            double feq[9];
            oracle_feq(rho1[IDX(p, y, x)], 0.0, 0.0, feq);
            for (int i = 0; i < 9; ++i) f[FIDX(p, 0, i, y, x)] = feq[i];
            oracle_feq(rho2[IDX(p, y, x)], 0.0, 0.0, feq);
            for (int i = 0; i < 9; ++i) f[FIDX(p, 1, i, y, x)] = feq[i];
        }
    if (d5) {
        static const int OUT_MISSING[3] = {3, 6, 7};
        static const int IN_MISSING[3] = {1, 5, 8};
        for (int k = 0; k < 3; ++k)
            for (int y = 0; y < p->ny; ++y) {
                d5[(size_t)k * p->ny + y] = f[FIDX(p, 0, OUT_MISSING[k], y, p->nx - 1)];
                d5[(size_t)(3 + k) * p->ny + y] = f[FIDX(p, 1, IN_MISSING[k], y, 0)];
            }
    }
}

/* Zou-He pressure condition at the inlet column x = 0 for component c with
 * density rho (Eqs. 22-25; zero tangential velocity): fills the missing
 * f_{1,5,8} of node (0, y) from the known ones. */
static void zou_he_inlet(const oracle_params *p, double *fnew, int c, int y, double rho,
                         const int *missing) {
    double f0 = fnew[FIDX(p, c, 0, y, 0)], f2 = fnew[FIDX(p, c, 2, y, 0)];
    double f3 = fnew[FIDX(p, c, 3, y, 0)], f4 = fnew[FIDX(p, c, 4, y, 0)];
    double f6 = fnew[FIDX(p, c, 6, y, 0)], f7 = fnew[FIDX(p, c, 7, y, 0)];
    double ux = 1.0 - (f0 + f2 + f4 + 2.0 * (f3 + f6 + f7)) / rho;
    if (missing[1]) fnew[FIDX(p, c, 1, y, 0)] = f3 + 2.0 / 3.0 * rho * ux;
    if (missing[5]) fnew[FIDX(p, c, 5, y, 0)] = f7 - 0.5 * (f2 - f4) + 1.0 / 6.0 * (rho * ux);
    if (missing[8]) fnew[FIDX(p, c, 8, y, 0)] = f6 + 0.5 * (f2 - f4) + 1.0 / 6.0 * (rho * ux);
}

/* The same at the outlet column x = nx - 1 (Eqs. 18-21): fills f_{3,6,7}. */
static void zou_he_outlet(const oracle_params *p, double *fnew, int c, int y, double rho,
                          const int *missing) {
    int x = p->nx - 1;
    double f0 = fnew[FIDX(p, c, 0, y, x)], f1 = fnew[FIDX(p, c, 1, y, x)];
    double f2 = fnew[FIDX(p, c, 2, y, x)], f4 = fnew[FIDX(p, c, 4, y, x)];
    double f5 = fnew[FIDX(p, c, 5, y, x)], f8 = fnew[FIDX(p, c, 8, y, x)];
    double ux = -1.0 + (f0 + f2 + f4 + 2.0 * (f1 + f5 + f8)) / rho;
    if (missing[3]) fnew[FIDX(p, c, 3, y, x)] = f1 - 2.0 / 3.0 * rho * ux;
    if (missing[6]) fnew[FIDX(p, c, 6, y, x)] = f8 - 0.5 * (f2 - f4) - 1.0 / 6.0 * (rho * ux);
    if (missing[7]) fnew[FIDX(p, c, 7, y, x)] = f5 + 0.5 * (f2 - f4) - 1.0 / 6.0 * (rho * ux);
}

/*
 * Streaming (left side of Eq. 1) with half-way bounce-back, then the inlet
 * and outlet treatment of Sec. 2.3 (Set-1, -2 or -3, see bc_set).  fpost
 * holds post-collision populations of step t; fnew receives the populations
 * of step t+1 before collision.
 */
void oracle_stream_bc(const oracle_params *p, const uint8_t *solid,
                      const double *d5, const double *fpost, double *fnew) {
    size_t n = (size_t)p->nx * p->ny;
    const int set = p->bc_set == 1 || p->bc_set == 2 ? p->bc_set : 3;
    memset(fnew, 0, 18 * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            if (solid[IDX(p, y, x)]) continue;
            int missing[9] = {0};
            /* pull: f_i(x, t+1) = f*_i(x - e_i, t) */
            for (int i = 0; i < 9; ++i) {
                int sx = x - EX[i], sy = y - EY[i];
                int in_x = (sx >= 0 && sx < p->nx) || !p->open_x;
                if (!in_x) { missing[i] = 1; continue; }
                if (!resolve(p, &sx, &sy) || solid[IDX(p, sy, sx)]) {
                    /* half-way bounce-back: reflect own post-collision value */
                    for (int c = 0; c < 2; ++c)
                        fnew[FIDX(p, c, i, y, x)] = fpost[FIDX(p, c, OPP[i], y, x)];
                } else {
                    for (int c = 0; c < 2; ++c)
                        fnew[FIDX(p, c, i, y, x)] = fpost[FIDX(p, c, i, sy, sx)];
                }
            }
            if (!p->open_x) continue;
            if (x == 0) {
                /* inlet, component 1: Zou-He with rho_in1 (Eqs. 22-25) */
                zou_he_inlet(p, fnew, 0, y, p->rho_in1, missing);
                static const int IN_MISSING[3] = {1, 5, 8};
                if (set == 1) {
                    /* Set-1: component 2 by the same equations, rho_in2 */
                    zou_he_inlet(p, fnew, 1, y, p->rho_in2, missing);
                } else {
                    for (int k = 0; k < 3; ++k) {
                        int i = IN_MISSING[k];
                        if (!missing[i]) continue;
                        fnew[FIDX(p, 1, i, y, x)] =
                            set == 2 ? d5[(size_t)(3 + k) * p->ny + y] /* Set-2: Eq. 27 */
                                     : fpost[FIDX(p, 1, i, y, x)];    /* Set-3: own post-collision, Eq. 28 */
                    }
                }
            }
            if (x == p->nx - 1) {
                /* outlet, component 2: Zou-He with rho_out2 (Eqs. 18-21) */
                zou_he_outlet(p, fnew, 1, y, p->rho_out2, missing);
                if (set == 1) {
                    /* Set-1: component 1 by the same equations, rho_out1 */
                    zou_he_outlet(p, fnew, 0, y, p->rho_out1, missing);
                } else {
                    /* Set-2 and Set-3: open condition of Eq. 26 */
                    static const int OUT_MISSING[3] = {3, 6, 7};
                    for (int k = 0; k < 3; ++k) {
                        int i = OUT_MISSING[k];
                        if (missing[i]) fnew[FIDX(p, 0, i, y, x)] = d5[(size_t)k * p->ny + y];
                    }
                }
            }
        }
}

/* Eqs. 3-5: component densities and momenta on fluid nodes. */
void oracle_moments(const oracle_params *p, const uint8_t *solid, const double *f,
                    double *rho /*[2][ny][nx]*/, double *jx, double *jy) {
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x)
            for (int c = 0; c < 2; ++c) {
                double r = 0.0, mx = 0.0, my = 0.0;
                if (!solid[IDX(p, y, x)])
                    for (int i = 0; i < 9; ++i) {
                        double fi = f[FIDX(p, c, i, y, x)];
                        r += fi;
                        mx += EX[i] * fi;
                        my += EY[i] * fi;
                    }
                rho[c * n + IDX(p, y, x)] = r;
                if (jx) jx[c * n + IDX(p, y, x)] = mx;
                if (jy) jy[c * n + IDX(p, y, x)] = my;
            }
}

/*
 * Improved virtual solid density, Eqs. 16-17: at a solid node with at least
 * one fluid neighbour, s^sigma = chi^sigma * (sum_i w_i rho^sigma(x+e_i)(1-phi))
 * / (sum_i w_i (1-phi)), with chi^1 = 1 + xi and chi^2 = 1 - xi taken from the
 * node's own xi.  psi receives rho^sigma on fluid nodes and s^sigma on solid
 * nodes (0 where a solid node has no fluid neighbour).
 */
void oracle_ivsd(const oracle_params *p, const uint8_t *solid, const float *xi,
                 const double *rho, double *psi) {
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t id = IDX(p, y, x);
            if (!solid[id]) {
                psi[id] = rho[id];
                psi[n + id] = rho[n + id];
                continue;
            }
            double num1 = 0.0, num2 = 0.0, den = 0.0;
            for (int i = 0; i < 9; ++i) {
                int nx_ = x + EX[i], ny_ = y + EY[i];
                if (!resolve(p, &nx_, &ny_)) continue;
                size_t nid = IDX(p, ny_, nx_);
                double fluid = solid[nid] ? 0.0 : 1.0; /* 1 - phi */
                num1 += WGT[i] * rho[nid] * fluid;
                num2 += WGT[i] * rho[n + nid] * fluid;
                den += WGT[i] * fluid;
            }
            double chi1 = 1.0 + (double)xi[id], chi2 = 1.0 - (double)xi[id];
            psi[id] = den > 0.0 ? chi1 * num1 / den : 0.0;
            psi[n + id] = den > 0.0 ? chi2 * num2 / den : 0.0;
        }
}

/*
 * Total force, Eq. 12: cohesion (Eq. 13) over fluid neighbours with
 * psi = rho, adhesion (Eq. 15) over solid neighbours with the virtual solid
 * density, body force rho^sigma g.  At open x ends a neighbour beyond the
 * boundary is replaced by the one in the opposite direction (Sec. 2.1).
 */
void oracle_forces(const oracle_params *p, const uint8_t *solid, const double *rho,
                   const double *psi, double *fx /*[2][ny][nx]*/, double *fy) {
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t id = IDX(p, y, x);
            if (solid[id]) {
                fx[id] = fy[id] = fx[n + id] = fy[n + id] = 0.0;
                continue;
            }
            for (int c = 0; c < 2; ++c) {
                int cb = 1 - c; /* sigma_bar */
                double coh_x = 0.0, coh_y = 0.0, ads_x = 0.0, ads_y = 0.0;
                for (int i = 1; i < 9; ++i) {
                    int j = i;
                    int nx_ = x + EX[i], ny_ = y + EY[i];
                    if (p->open_x && (nx_ < 0 || nx_ >= p->nx)) {
                        j = OPP[i]; /* mirror: psi(x+e_i) = psi(x+e_opp(i)) */
                        nx_ = x + EX[j];
                        ny_ = y + EY[j];
                    }
                    if (!resolve(p, &nx_, &ny_)) continue; /* cannot happen: walls */
                    size_t nid = IDX(p, ny_, nx_);
                    double v = psi[(size_t)cb * n + nid];
                    if (solid[nid]) {
                        ads_x += WGT[i] * v * EX[i];
                        ads_y += WGT[i] * v * EY[i];
                    } else {
                        coh_x += WGT[i] * v * EX[i];
                        coh_y += WGT[i] * v * EY[i];
                    }
                }
                double r = rho[(size_t)c * n + id];
                fx[(size_t)c * n + id] = -p->g_coh * r * coh_x - p->g_ads * r * ads_x + r * p->gx;
                fy[(size_t)c * n + id] = -p->g_coh * r * coh_y - p->g_ads * r * ads_y + r * p->gy;
            }
        }
}

/*
 * Collision, Eq. 1 right-hand side: system relaxation time (Eq. 6),
 * equilibrium velocity (Eqs. 8-9), equilibrium (Eq. 2) and forcing (Eq. 11).
 */
void oracle_collide(const oracle_params *p, const uint8_t *solid, const double *f,
                    const double *rho, const double *jx, const double *jy,
                    const double *fx, const double *fy, double *fpost,
                    double *ueq_x, double *ueq_y) {
    size_t n = (size_t)p->nx * p->ny;
    memset(fpost, 0, 18 * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t id = IDX(p, y, x);
            if (solid[id]) {
                if (ueq_x) ueq_x[id] = 0.0;
                if (ueq_y) ueq_y[id] = 0.0;
                continue;
            }
            double r1 = rho[id], r2 = rho[n + id];
            double r = r1 + r2;                                      /* Eq. 5 */
            double tau_s = (r1 * p->nu1 + r2 * p->nu2) * INV_CS2 / r + 0.5; /* Eq. 6 */
            double omega = 1.0 / tau_s;
            /* Eq. 8: with a common tau_s the weights cancel, leaving the
             * barycentric velocity (plus F/2, see header) */
            double jsx = jx[id] + jx[n + id], jsy = jy[id] + jy[n + id];
            double ftx = fx[id] + fx[n + id], fty = fy[id] + fy[n + id];
            double ux, uy;
            if (p->vel_shift) {
                ux = (jsx + 0.5 * ftx) / r;
                uy = (jsy + 0.5 * fty) / r;
            } else {
                ux = jsx / r;
                uy = jsy / r;
            }
            if (ueq_x) ueq_x[id] = ux;
            if (ueq_y) ueq_y[id] = uy;
            for (int c = 0; c < 2; ++c) {
                double feq[9], s[9];
                oracle_feq(rho[(size_t)c * n + id], ux, uy, feq);
                oracle_source(ux, uy, fx[(size_t)c * n + id], fy[(size_t)c * n + id], s);
                if (p->mrt) {
                    double fin[9], fout[9];
                    for (int i = 0; i < 9; ++i) fin[i] = f[FIDX(p, c, i, y, x)];
                    mrt_collide(p, omega, fin, feq, s, fout);
                    for (int i = 0; i < 9; ++i) fpost[FIDX(p, c, i, y, x)] = fout[i];
                    continue;
                }
                for (int i = 0; i < 9; ++i) {
                    double fi = f[FIDX(p, c, i, y, x)];
                    fpost[FIDX(p, c, i, y, x)] =
                        fi - omega * (fi - feq[i]) + (1.0 - 0.5 * omega) * s[i];
                }
            }
        }
}

/*
 * Advance nsteps time steps.  f holds post-collision populations
 * [2][9][ny][nx] on entry and on exit.  If ux/uy are given they receive the
 * equilibrium velocity (Eq. 9) used by the last collision.  Returns 0, or -1
 * if memory could not be allocated.
 */
int oracle_step(const oracle_params *p, const uint8_t *solid, const float *xi,
                const double *d5, double *f, long nsteps, double *ux, double *uy) {
    size_t n = (size_t)p->nx * p->ny;
    double *fs = malloc(18 * n * sizeof(double));
    double *rho = malloc(2 * n * sizeof(double));
    double *jx = malloc(2 * n * sizeof(double));
    double *jy = malloc(2 * n * sizeof(double));
    double *psi = malloc(2 * n * sizeof(double));
    double *fx = malloc(2 * n * sizeof(double));
    double *fy = malloc(2 * n * sizeof(double));
    int rc = 0;
    if (!fs || !rho || !jx || !jy || !psi || !fx || !fy) {
        rc = -1;
        goto done;
    }
    for (long t = 0; t < nsteps; ++t) {
        int last = (t == nsteps - 1);
        oracle_stream_bc(p, solid, d5, f, fs);
        oracle_moments(p, solid, fs, rho, jx, jy);
        oracle_ivsd(p, solid, xi, rho, psi);
        oracle_forces(p, solid, rho, psi, fx, fy);
        oracle_collide(p, solid, fs, rho, jx, jy, fx, fy, f, last ? ux : NULL,
                       last ? uy : NULL);
    }
done:
    free(fs); free(rho); free(jx); free(jy); free(psi); free(fx); free(fy);
    return rc;
}

/*
 * Diagnostics of a post-collision state (Sec. 4.2.1):
 *   out[0], out[1]  per-component mass, sum over fluid nodes of sum_i f_i
 *   out[2]          water saturation by count: fluid nodes with rho2 > rho1
 *                   over all fluid nodes
 *   out[3]          water saturation by mass: sum rho2 / sum (rho1 + rho2)
 *   out[4], out[5]  boundary pressures P_in, P_out: mean of Eq. 14 over the
 *                   fluid nodes of column 0 (nx-1) farther than 2 nodes in y
 *                   from any solid node of that column (NaN if none)
 *   out[6]          capillary pressure P_in - P_out
 *   out[7]          number of fluid nodes
 * Sums run serially in row-major order.
 */
void oracle_diagnostics(const oracle_params *p, const uint8_t *solid, const double *f,
                        double *out) {
    double m1 = 0.0, m2 = 0.0, nfluid = 0.0, nwater = 0.0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            if (solid[IDX(p, y, x)]) continue;
            double r1 = 0.0, r2 = 0.0;
            for (int i = 0; i < 9; ++i) {
                r1 += f[FIDX(p, 0, i, y, x)];
                r2 += f[FIDX(p, 1, i, y, x)];
            }
            m1 += r1;
            m2 += r2;
            nfluid += 1.0;
            if (r2 > r1) nwater += 1.0;
        }
    out[0] = m1;
    out[1] = m2;
    out[2] = nfluid > 0 ? nwater / nfluid : NAN;
    out[3] = (m1 + m2) > 0 ? m2 / (m1 + m2) : NAN;
    for (int side = 0; side < 2; ++side) {
        int x = side == 0 ? 0 : p->nx - 1;
        double sum = 0.0, cnt = 0.0;
        for (int y = 0; y < p->ny; ++y) {
            if (solid[IDX(p, y, x)]) continue;
            int near = 0;
            for (int d = -2; d <= 2 && !near; ++d) {
                int yy = y + d, xx = x;
                if (!resolve(p, &xx, &yy)) { near = 1; break; }
                if (solid[IDX(p, yy, xx)]) near = 1;
            }
            if (near) continue;
            double r1 = 0.0, r2 = 0.0;
            for (int i = 0; i < 9; ++i) {
                r1 += f[FIDX(p, 0, i, y, x)];
                r2 += f[FIDX(p, 1, i, y, x)];
            }
            sum += oracle_pressure(p->g_coh, r1, r2);
            cnt += 1.0;
        }
        out[4 + side] = cnt > 0 ? sum / cnt : NAN;
    }
    out[6] = out[4] - out[5];
    out[7] = nfluid;
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
