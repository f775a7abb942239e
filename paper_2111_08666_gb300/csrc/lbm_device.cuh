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

// ---------------------------------------------------------------------------
// Set-3 boundary treatment (Sec. 2.3) on pulled populations f of a node at
// an open end; own(c, i) returns the node's own post-collision f*.
//   x = 0:     component 1 Zou-He with rho_in (Eqs. 22-25) for f_1, f_5, f_8;
//              component 2 keeps its own post-collision f_1, f_5, f_8 (Eq. 28)
//   x = nx-1:  component 2 Zou-He with rho_out (Eqs. 18-21) for f_3, f_6, f_7;
//              component 1 takes the recorded values of Eq. 26.
// ---------------------------------------------------------------------------
template <class R, class Own>
__device__ __forceinline__ void apply_set3(const StepArgs &a, int x, int y, Own own, R f[2][9]) {
    if (!a.p.open_x) return;
    if (x == 0) {
        const R rin = R(a.p.rho_in1);
        const R ux = R(1) - (f[0][0] + f[0][2] + f[0][4] + R(2) * (f[0][3] + f[0][6] + f[0][7])) / rin;
        const R d24 = R(0.5) * (f[0][2] - f[0][4]);
        const R ru6 = rin * ux * (R(1) / R(6));
        f[0][1] = f[0][3] + (R(2) / R(3)) * rin * ux;
        f[0][5] = f[0][7] - d24 + ru6;
        f[0][8] = f[0][6] + d24 + ru6;
        f[1][1] = own(1, 1);
        f[1][5] = own(1, 5);
        f[1][8] = own(1, 8);
    }
    if (x == a.g.nx - 1) {
        const R rout = R(a.p.rho_out2);
        const R ux = R(-1) + (f[1][0] + f[1][2] + f[1][4] + R(2) * (f[1][1] + f[1][5] + f[1][8])) / rout;
        const R d24 = R(0.5) * (f[1][2] - f[1][4]);
        const R ru6 = rout * ux * (R(1) / R(6));
        f[1][3] = f[1][1] - (R(2) / R(3)) * rout * ux;
        f[1][6] = f[1][8] - d24 - ru6;
        f[1][7] = f[1][5] + d24 - ru6;
        const R *d5 = static_cast<const R *>(a.d5);
        f[0][3] = d5[y];
        f[0][6] = d5[a.g.ny + y];
        f[0][7] = d5[2 * a.g.ny + y];
    }
}

// Populations f_i(x, t+1) of fluid node (x, y) before collision, pulled
// from global memory: f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) when the source
// is solid (half-way bounce-back), then Set-3 at the open ends.  srcgeo(i)
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
    apply_set3<R>(a, x, y, [&](int c, int i) { return pop_load<P>(fin, plane, c, i, site); }, f);
}

// Interaction force on both components at a fluid node (Eqs. 12, 13, 15):
// F^s = -rho^s [G_coh sum_fluid w_i psi^sb(x+e_i) e_i
//              + G_ads sum_solid w_i s^sb(x+e_i) e_i] + rho^s g.
// nb(i, &code, &psi1, &psi2) returns the neighbour used for direction i
// (already mirrored at an open end).
template <class R, class Nb>
__device__ __forceinline__ void node_force(const Params &p, R rho1, R rho2, Nb nb,
                                           R &fx1, R &fy1, R &fx2, R &fy2) {
    R cx1 = 0, cy1 = 0, cx2 = 0, cy2 = 0;  // cohesion sums over psi of the other component
    R ax1 = 0, ay1 = 0, ax2 = 0, ay2 = 0;  // adhesion sums
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        uint8_t code;
        R s1, s2;
        nb(i, code, s1, s2);
        const R w = wgt<R>(i);
        if (code == GEO_FLUID) {
            if (ex(i)) { cx1 += R(ex(i)) * w * s2; cx2 += R(ex(i)) * w * s1; }
            if (ey(i)) { cy1 += R(ey(i)) * w * s2; cy2 += R(ey(i)) * w * s1; }
        } else if (code != GEO_OUTSIDE) {
            if (ex(i)) { ax1 += R(ex(i)) * w * s2; ax2 += R(ex(i)) * w * s1; }
            if (ey(i)) { ay1 += R(ey(i)) * w * s2; ay2 += R(ey(i)) * w * s1; }
        }
    }
    const R gc = R(p.g_coh), ga = R(p.g_ads);
    fx1 = -rho1 * (gc * cx1 + ga * ax1) + rho1 * R(p.gx);
    fy1 = -rho1 * (gc * cy1 + ga * ay1) + rho1 * R(p.gy);
    fx2 = -rho2 * (gc * cx2 + ga * ax2) + rho2 * R(p.gx);
    fy2 = -rho2 * (gc * cy2 + ga * ay2) + rho2 * R(p.gy);
}

// System relaxation time (Eq. 6) and common velocity (Eqs. 8-9) of a node.
template <class R>
__device__ __forceinline__ void node_velocity(const Params &p, const R f[2][9], R rho1, R rho2,
                                              R fx, R fy, R &omega, R &ux, R &uy) {
    const R rho = rho1 + rho2;
    const R inv_rho = R(1) / rho;
    const R tau = (rho1 * R(p.nu1) + rho2 * R(p.nu2)) * R(3) * inv_rho + R(0.5);
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

// Forced BGK collision of one component (Eqs. 1, 2, 11), in place on f.
// rho = sum_i f_i.  Since sum_i f^eq_i = rho and sum_i S_i = 0, the
// post-collision populations also sum to rho; f*_0 is taken from that
// identity so that rounding of the weights cannot bias the mass.
template <class R>
__device__ __forceinline__ void collide_component(R f[9], R rho, R ux, R uy, R fx, R fy,
                                                  R omega) {
    const R uu = R(1.5) * (ux * ux + uy * uy);
    const R uf = ux * fx + uy * fy;
    const R pref = R(1) - R(0.5) * omega;
    const R base = rho * (R(1) - uu);
    R rest = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R eu = R(ex(i)) * ux + R(ey(i)) * uy;
        const R ef = R(ex(i)) * fx + R(ey(i)) * fy;
        const R w = wgt<R>(i);
        const R feq = w * (base + rho * eu * (R(3) + R(4.5) * eu));
        // S_i = w_i [ 3 (e_i - u) . F + 9 (e_i . u)(e_i . F) ]
        const R src = w * (R(3) * (ef - uf) + R(9) * eu * ef);
        f[i] = f[i] - omega * (f[i] - feq) + pref * src;
        rest += f[i];
    }
    f[0] = rho - rest;
}

}  // namespace mclbm
