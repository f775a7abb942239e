// Device building blocks of one update: population encoding, the pull with
// bounce-back and Set-3 boundaries from global memory, the interaction
// force, the velocity and the forced BGK collision.  Shared by the step
// kernels and the read-out kernels.
#pragma once

#include "lbm.cuh"

namespace mclbm {

// wrap by one period (v in [-n, 2n))
__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
// wrap by any number of periods
__device__ __forceinline__ int pmod(int v, int n) { return ((v % n) + n) % n; }

// element offset of node (x, y) in a population plane
__device__ __forceinline__ long long site_of(const Geometry &g, int x, int y) {
    return (long long)(y + HY) * g.pitch + g.hx + x;
}

// ---------------------------------------------------------------------------
// Population codec (global memory).
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ typename P::real_t pop_load(const typename P::store_t *f,
                                                       long long plane, int c, int i,
                                                       long long site) {
    using R = typename P::real_t;
    R v = to_real(__ldg(f + (long long)(c * 9 + i) * plane + site));
    if constexpr (P::ref) v += wgt<R>(i) * to_real(__ldg(f + (long long)(18 + c) * plane + site));
    return v;
}

// Encode and store the 2 x 9 post-collision populations of one node at
// element offset site (and, for periodic x, at its ghost images).
template <class P>
__device__ __forceinline__ void pop_store_site(typename P::store_t *f, long long plane,
                                               long long site, const typename P::real_t fs[2][9],
                                               typename P::real_t rho1,
                                               typename P::real_t rho2) {
    using R = typename P::real_t;
    using S = typename P::store_t;
    if constexpr (P::ref) {
        const S h1 = from_real<S>(rho1), h2 = from_real<S>(rho2);
        f[18 * plane + site] = h1;
        f[19 * plane + site] = h2;
        const R q1 = to_real(h1), q2 = to_real(h2);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[(long long)i * plane + site] = from_real<S>(fs[0][i] - wgt<R>(i) * q1);
            f[(long long)(9 + i) * plane + site] = from_real<S>(fs[1][i] - wgt<R>(i) * q2);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[(long long)i * plane + site] = from_real<S>(fs[0][i]);
            f[(long long)(9 + i) * plane + site] = from_real<S>(fs[1][i]);
        }
    }
}

// Store the ghost images of node (x, y) (periodic x and/or y); the node's
// own site is not written.
template <class P>
__device__ __forceinline__ void pop_store_ghosts(const Geometry &g, const Params &p,
                                                 typename P::store_t *f, int x, int y,
                                                 const typename P::real_t fs[2][9],
                                                 typename P::real_t rho1,
                                                 typename P::real_t rho2) {
    const bool px = !p.open_x, py = p.periodic_y != 0;
    if (!px && !py) return;
    const bool near_x = px && (x < g.hx || x >= g.nx - g.hx);
    const bool near_y = py && (y < HY || y >= g.ny - HY);
    if (!near_x && !near_y) return;
    // every image (x + a nx, y + b ny) inside the ghost frame, except a = b = 0
    const int ax0 = px ? -((x + g.hx) / g.nx) : 0, ax1 = px ? (g.nx + g.hx - 1 - x) / g.nx : 0;
    const int by0 = py ? -((y + HY) / g.ny) : 0, by1 = py ? (g.ny + HY - 1 - y) / g.ny : 0;
    for (int a = ax0; a <= ax1; ++a)
        for (int b = by0; b <= by1; ++b) {
            if (a == 0 && b == 0) continue;
            pop_store_site<P>(f, g.plane, site_of(g, x + a * g.nx, y + b * g.ny), fs, rho1, rho2);
        }
}

template <class P>
__device__ __forceinline__ void pop_store_node(const Geometry &g, const Params &p,
                                               typename P::store_t *f, int x, int y,
                                               const typename P::real_t fs[2][9],
                                               typename P::real_t rho1, typename P::real_t rho2) {
    pop_store_site<P>(f, g.plane, site_of(g, x, y), fs, rho1, rho2);
    pop_store_ghosts<P>(g, p, f, x, y, fs, rho1, rho2);
}

// Geometry code of (x, y) with periodic wrap where the lattice is periodic,
// GEO_OUTSIDE beyond a non-periodic edge.
__device__ __forceinline__ uint8_t geo_at(const Geometry &g, const Params &p, int x, int y) {
    if (y < 0 || y >= g.ny) {
        if (!p.periodic_y) return GEO_OUTSIDE;
        y = pmod(y, g.ny);
    }
    if (x < 0 || x >= g.nx) {
        if (p.open_x) return GEO_OUTSIDE;
        x = pmod(x, g.nx);
    }
    return g.geo[(long long)y * g.gpitch + GEO_HX + x];
}

// Inlet/outlet pressure treatment of Sec. 2.3 at a fluid node of the open
// columns x = 0 and x = nx - 1, after streaming; f holds the streamed
// populations, own(c, i) the node's own post-collision value.
//   inlet:  component 1 by Zou-He with rho_in1 (Eqs. 22-25); component 2 by
//           Zou-He with rho_in2 (Set-1), frozen at initialisation (Eq. 27,
//           Set-2) or its own post-collision values (Eq. 28, Set-3);
//   outlet: component 2 by Zou-He with rho_out2 (Eqs. 18-21); component 1 by
//           Zou-He with rho_out1 (Set-1) or frozen at initialisation (Eq. 26,
//           Sets 2 and 3).
// Zou-He takes zero tangential velocity; u_x follows from the density.
template <class R>
__device__ __forceinline__ void zou_he_in(R g[9], R rin) {
    const R ux = R(1) - (g[0] + g[2] + g[4] + R(2) * (g[3] + g[6] + g[7])) / rin;
    const R d24 = R(0.5) * (g[2] - g[4]);
    const R ru6 = rin * ux * (R(1) / R(6));
    g[1] = g[3] + (R(2) / R(3)) * rin * ux;
    g[5] = g[7] - d24 + ru6;
    g[8] = g[6] + d24 + ru6;
}
template <class R>
__device__ __forceinline__ void zou_he_out(R g[9], R rout) {
    const R ux = R(-1) + (g[0] + g[2] + g[4] + R(2) * (g[1] + g[5] + g[8])) / rout;
    const R d24 = R(0.5) * (g[2] - g[4]);
    const R ru6 = rout * ux * (R(1) / R(6));
    g[3] = g[1] - (R(2) / R(3)) * rout * ux;
    g[6] = g[8] - d24 - ru6;
    g[7] = g[5] + d24 - ru6;
}

template <class R, class Own>
__device__ __forceinline__ void apply_open_bc(const StepArgs &a, int x, int y, Own own, R f[2][9]) {
    if (!a.p.open_x) return;
    const R *d5 = static_cast<const R *>(a.d5);
    if (x == 0) {
        zou_he_in<R>(f[0], par<R>(a.p.rho_in1, a.p.rho_in1_f));
        if (a.p.bc_set == 1) {
            zou_he_in<R>(f[1], par<R>(a.p.rho_in2, a.p.rho_in2_f));
        } else if (a.p.bc_set == 2) {
            f[1][1] = d5[3 * a.g.ny + y];
            f[1][5] = d5[4 * a.g.ny + y];
            f[1][8] = d5[5 * a.g.ny + y];
        } else {
            f[1][1] = own(1, 1);
            f[1][5] = own(1, 5);
            f[1][8] = own(1, 8);
        }
    }
    if (x == a.g.nx - 1) {
        zou_he_out<R>(f[1], par<R>(a.p.rho_out2, a.p.rho_out2_f));
        if (a.p.bc_set == 1) {
            zou_he_out<R>(f[0], par<R>(a.p.rho_out1, a.p.rho_out1_f));
        } else {
            f[0][3] = d5[y];
            f[0][6] = d5[a.g.ny + y];
            f[0][7] = d5[2 * a.g.ny + y];
        }
    }
}

// Populations f_i(x, t+1) of fluid node (x, y) before collision, pulled
// from global memory: f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) when the source
// is solid (half-way bounce-back), then the open-end treatment (Sec. 2.3).  srcgeo(i)
// returns the geometry code of the source x - e_i.
template <class P, class SrcGeo>
__device__ __forceinline__ void pull_node(const StepArgs &a, int x, int y, SrcGeo srcgeo,
                                          typename P::real_t f[2][9]) {
    using R = typename P::real_t;
    using S = typename P::store_t;
    const S *fin = static_cast<const S *>(a.fin);
    const long long plane = a.g.plane;
    const long long site = site_of(a.g, x, y);
    const bool at_in = a.p.open_x && x == 0;
    const bool at_out = a.p.open_x && x == a.g.nx - 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool missing = (at_in && ex(i) == 1) || (at_out && ex(i) == -1);
        if (missing) {
            f[0][i] = R(0);
            f[1][i] = R(0);
            continue;
        }
        if (i == 0) {
            f[0][0] = pop_load<P>(fin, plane, 0, 0, site);
            f[1][0] = pop_load<P>(fin, plane, 1, 0, site);
            continue;
        }
        if (srcgeo(i) != GEO_FLUID) {
            f[0][i] = pop_load<P>(fin, plane, 0, opp(i), site);
            f[1][i] = pop_load<P>(fin, plane, 1, opp(i), site);
        } else {
            const long long ss = site_of(a.g, wrap(x - ex(i), a.g.nx), wrap(y - ey(i), a.g.ny));
            f[0][i] = pop_load<P>(fin, plane, 0, i, ss);
            f[1][i] = pop_load<P>(fin, plane, 1, i, ss);
        }
    }
    apply_open_bc<R>(a, x, y, [&](int c, int i) { return pop_load<P>(fin, plane, c, i, site); }, f);
}

// e_i . (vx, vy) without multiplications by 0 or 1 (i is a constant in the
// unrolled loops, so this folds to at most one add)
template <class R>
__device__ __forceinline__ R edot(int i, R vx, R vy) {
    R v = R(0);
    if (ex(i) > 0) v = vx;
    if (ex(i) < 0) v = -vx;
    if (ey(i) > 0) v = ex(i) ? v + vy : vy;
    if (ey(i) < 0) v = ex(i) ? v - vy : -vy;
    return v;
}

// Interaction force on both components at a fluid node (Eqs. 12, 13, 15):
// F^s = -rho^s [G_coh sum_fluid w_i psi^sb(x+e_i) e_i
//              + G_ads sum_solid w_i s^sb(x+e_i) e_i] + rho^s g.
// Both sums are taken as one, each neighbour weighted by G_coh w_i or
// G_ads w_i.  nb(i, &code, &psi1, &psi2) returns the neighbour used for
// direction i (already mirrored at an open end); with OUTSIDE = false the
// caller guarantees that no neighbour is outside the lattice.
template <class R, bool OUTSIDE = true, class Nb>
__device__ __forceinline__ void node_force(const Params &p, R rho1, R rho2, Nb nb,
                                           R &fx1, R &fy1, R &fx2, R &fy2) {
    const R gc = par<R>(p.g_coh, p.g_coh_f), ga = par<R>(p.g_ads, p.g_ads_f);
    const R gc_a = gc * wgt<R>(1), gc_d = gc * wgt<R>(5);  // axis and diagonal weights
    const R ga_a = ga * wgt<R>(1), ga_d = ga * wgt<R>(5);
    R sx1 = 0, sy1 = 0, sx2 = 0, sy2 = 0;  // sums over psi (or s) of the other component
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        uint8_t code;
        R s1, s2;
        nb(i, code, s1, s2);
        const bool diag = i >= 5;
        const R k = code == GEO_FLUID ? (diag ? gc_d : gc_a) : (diag ? ga_d : ga_a);
        R a1 = k * s2, a2 = k * s1;
        if (OUTSIDE && code == GEO_OUTSIDE) a1 = a2 = R(0);
        if (ex(i)) {
            sx1 = ex(i) > 0 ? sx1 + a1 : sx1 - a1;
            sx2 = ex(i) > 0 ? sx2 + a2 : sx2 - a2;
        }
        if (ey(i)) {
            sy1 = ey(i) > 0 ? sy1 + a1 : sy1 - a1;
            sy2 = ey(i) > 0 ? sy2 + a2 : sy2 - a2;
        }
    }
    fx1 = rho1 * (par<R>(p.gx, p.gx_f) - sx1);
    fy1 = rho1 * (par<R>(p.gy, p.gy_f) - sy1);
    fx2 = rho2 * (par<R>(p.gx, p.gx_f) - sx2);
    fy2 = rho2 * (par<R>(p.gy, p.gy_f) - sy2);
}

// System relaxation time (Eq. 6) and common velocity (Eqs. 8-9) of a node.
template <class R>
__device__ __forceinline__ void node_velocity(const Params &p, const R f[2][9], R rho1, R rho2,
                                              R fx, R fy, R &omega, R &ux, R &uy) {
    const R rho = rho1 + rho2;
    const R inv_rho = R(1) / rho;
    const R tau = (rho1 * par<R>(p.nu1, p.nu1_f) + rho2 * par<R>(p.nu2, p.nu2_f)) * R(3) * inv_rho + R(0.5);
    omega = R(1) / tau;
    R jx = 0, jy = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R fi = f[0][i] + f[1][i];
        if (ex(i)) jx += R(ex(i)) * fi;
        if (ey(i)) jy += R(ey(i)) * fi;
    }
    if (p.vel_shift) {
        jx += R(0.5) * fx;
        jy += R(0.5) * fy;
    }
    ux = jx * inv_rho;
    uy = jy * inv_rho;
}

// Forced BGK collision of both components (Eqs. 1, 2, 11), in place on f:
//   f*_i = (1 - omega) f_i + omega rho^s E_i + (1 - omega/2) S^s_i
// with f^eq_i = rho^s E_i, E_i = w_i [1 - 1.5 u.u + e_i.u (3 + 4.5 e_i.u)]
// shared by the components, and the source of Eq. 11 written as
//   S^s_i = w_i (3 + 9 e_i.u) e_i.F^s - 3 w_i u.F^s.
// Since sum_i f^eq_i = rho^s and sum_i S^s_i = 0, the post-collision
// populations sum to rho^s = sum_i f_i; f*_0 is taken from that identity so
// that rounding of the weights cannot bias the mass.
template <class R>
__device__ __forceinline__ void collide_pair(R f[2][9], R rho1, R rho2, R ux, R uy, R fx1, R fy1,
                                             R fx2, R fy2, R omega) {
    const R keep = R(1) - omega;
    const R pref = R(1) - R(0.5) * omega;
    const R q1 = omega * rho1, q2 = omega * rho2;
    const R gx1 = pref * fx1, gy1 = pref * fy1, gx2 = pref * fx2, gy2 = pref * fy2;
    const R ub = R(1) - R(1.5) * (ux * ux + uy * uy);
    const R v1 = R(3) * (ux * gx1 + uy * gy1), v2 = R(3) * (ux * gx2 + uy * gy2);
    R r1 = 0, r2 = 0;
    // the directions in opposite pairs (i, opp(i)): e_opp . u = -e_i . u, so
    // E_i and E_opp share the even part w (ub + 4.5 (e.u)^2) and differ in
    // the sign of 3 w e.u, and the sources in the sign of their e.F term
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = k < 2 ? k + 1 : k + 3, j = opp(i);
        const R w = wgt<R>(i);
        const R eu = edot<R>(i, ux, uy);
        const R even = w * (ub + R(4.5) * eu * eu), odd = (R(3) * w) * eu;
        const R ai = w * R(3) + (R(9) * w) * eu, aj = w * R(3) - (R(9) * w) * eu;
        const R g1 = edot<R>(i, gx1, gy1), g2 = edot<R>(i, gx2, gy2);
        const R wv1 = w * v1, wv2 = w * v2;
        const R s1i = ai * g1 - wv1, s1j = -(aj * g1) - wv1;
        const R s2i = ai * g2 - wv2, s2j = -(aj * g2) - wv2;
        f[0][i] = keep * f[0][i] + (q1 * (even + odd) + s1i);
        f[0][j] = keep * f[0][j] + (q1 * (even - odd) + s1j);
        f[1][i] = keep * f[1][i] + (q2 * (even + odd) + s2i);
        f[1][j] = keep * f[1][j] + (q2 * (even - odd) + s2j);
        r1 += f[0][i] + f[0][j];
        r2 += f[1][i] + f[1][j];
    }
    f[0][0] = rho1 - r1;
    f[1][0] = rho2 - r2;
}

// Multiple-relaxation-time variant of the collision (not in the paper,
// which uses the SRT of Eq. 1): Eq. 1 with 1/tau_s replaced by a relaxation
// matrix diagonal in the moment basis of Lallemand and Luo,
//   m = (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy) = M f,
//   m* = m - S (m - m^eq) + (I - S/2) M S^F,   f* = M^-1 m*,
// S = diag(-, s_e, s_eps, w, s_q, w, s_q, w, w), w = 1/tau_s.  The moments
// of f^eq (Eq. 2) and of the source (Eq. 11) are taken in closed form:
//   e^eq = rho (3 u.u - 2), eps^eq = rho (1 - 3 u.u), j^eq = rho u,
//   q^eq = -rho u, p_xx^eq = rho (u_x^2 - u_y^2), p_xy^eq = rho u_x u_y;
//   source: e 6 u.F, eps -6 u.F, j F, q -F, p_xx 2 (u_x F_x - u_y F_y),
//   p_xy u_x F_y + u_y F_x.
// The rows of M are orthogonal with squared norms (9, 36, 36, 6, 12, 6, 12,
// 4, 4), which gives M^-1 = M^T diag(1 / norm).  f*_0 follows from mass.
template <class R>
__device__ __forceinline__ void mrt_one(R g[9], R rho, R ux, R uy, R fx, R fy, R w, R se, R seps, R sq) {
    const R ax = g[1] + g[2] + g[3] + g[4], dg = g[5] + g[6] + g[7] + g[8];
    const R uu = ux * ux + uy * uy, uf = ux * fx + uy * fy;
    const R e = R(-4) * g[0] - ax + R(2) * dg;
    const R eps = R(4) * g[0] - R(2) * ax + dg;
    const R jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    const R jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    const R qx = R(-2) * (g[1] - g[3]) + g[5] - g[6] - g[7] + g[8];
    const R qy = R(-2) * (g[2] - g[4]) + g[5] + g[6] - g[7] - g[8];
    const R pxx = g[1] - g[2] + g[3] - g[4];
    const R pxy = g[5] - g[6] + g[7] - g[8];
    auto relax = [](R m, R meq, R s, R src) { return m - s * (m - meq) + (R(1) - R(0.5) * s) * src; };
    const R e2 = relax(e, rho * (R(3) * uu - R(2)), se, R(6) * uf);
    const R eps2 = relax(eps, rho * (R(1) - R(3) * uu), seps, R(-6) * uf);
    const R jx2 = relax(jx, rho * ux, w, fx), jy2 = relax(jy, rho * uy, w, fy);
    const R qx2 = relax(qx, -rho * ux, sq, -fx), qy2 = relax(qy, -rho * uy, sq, -fy);
    const R pxx2 = relax(pxx, rho * (ux * ux - uy * uy), w, R(2) * (ux * fx - uy * fy));
    const R pxy2 = relax(pxy, rho * ux * uy, w, ux * fy + uy * fx);
    const R r9 = rho * (R(1) / R(9));
    const R ea = r9 - e2 * (R(1) / R(36)) - eps2 * (R(1) / R(18));  // common part of the axis directions
    const R ed = r9 + e2 * (R(1) / R(18)) + eps2 * (R(1) / R(36));  // of the diagonals
    const R jx6 = jx2 * (R(1) / R(6)), jy6 = jy2 * (R(1) / R(6));
    const R qx6 = qx2 * (R(1) / R(6)), qy6 = qy2 * (R(1) / R(6));
    const R qx12 = qx2 * (R(1) / R(12)), qy12 = qy2 * (R(1) / R(12));
    const R pxx4 = pxx2 * R(0.25), pxy4 = pxy2 * R(0.25);
    g[1] = ea + jx6 - qx6 + pxx4;
    g[2] = ea + jy6 - qy6 - pxx4;
    g[3] = ea - jx6 + qx6 + pxx4;
    g[4] = ea - jy6 + qy6 - pxx4;
    g[5] = ed + jx6 + qx12 + jy6 + qy12 + pxy4;
    g[6] = ed - jx6 - qx12 + jy6 + qy12 - pxy4;
    g[7] = ed - jx6 - qx12 - jy6 - qy12 + pxy4;
    g[8] = ed + jx6 + qx12 - jy6 - qy12 - pxy4;
    g[0] = rho - (g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8]);
}

// The MRT collision of both components with the lattice's rates.
template <class R>
__device__ __forceinline__ void collide_mrt(const Params &p, R f[2][9], R rho1, R rho2, R ux, R uy, R fx1,
                                            R fy1, R fx2, R fy2, R omega) {
    const R se = p.s_e > 0 ? par<R>(p.s_e, p.s_e_f) : omega;
    const R seps = p.s_eps > 0 ? par<R>(p.s_eps, p.s_eps_f) : omega;
    const R sq = p.s_q > 0 ? par<R>(p.s_q, p.s_q_f)
                           : (p.s_q < 0 ? R(8) * (R(2) - omega) / (R(8) - omega) : omega);
    mrt_one<R>(f[0], rho1, ux, uy, fx1, fy1, omega, se, seps, sq);
    mrt_one<R>(f[1], rho2, ux, uy, fx2, fy2, omega, se, seps, sq);
}

// The collision of both components: the SRT of Eq. 1 (collide_pair), or the
// MRT variant when the lattice asks for it.  CM selects at compile time:
// 0 SRT only, 1 MRT only, 2 by the lattice's flag.
template <class R, int CM = 2>
__device__ __forceinline__ void collide(const Params &p, R f[2][9], R rho1, R rho2, R ux, R uy, R fx1, R fy1,
                                        R fx2, R fy2, R omega) {
    if constexpr (CM == 0) {
        collide_pair<R>(f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
    } else if constexpr (CM == 1) {
        collide_mrt<R>(p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
    } else {
        if (p.mrt)
            collide_mrt<R>(p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
        else
            collide_pair<R>(f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
    }
}

}  // namespace mclbm
