// Kernels off the per-step path: initialisation at rest, population
// import/export, the FP64 diagnostics reduction and the field read-outs.
#include "lbm_device.cuh"

namespace mclbm {

namespace {

constexpr int BLK = 256;

inline int blocks_for(long long n, int per = BLK) { return (int)((n + per - 1) / per); }

// f_i = f_i^eq(rho^sigma, u = 0) = w_i rho^sigma (Eq. 2 at rest); records
// component 1's outlet f_{3,6,7} (Eq. 26) and component 2's inlet f_{1,5,8}
// (Eq. 27, Set-2).
template <class P>
__global__ void init_equilibrium_kernel(Geometry g, Params p, const double *rho1,
                                        const double *rho2, typename P::store_t *f,
                                        typename P::real_t *d5) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const bool fluid = g.geo[(long long)y * g.gpitch + GEO_HX + x] == GEO_FLUID;
    const R r1 = fluid ? R(rho1[k]) : R(0), r2 = fluid ? R(rho2[k]) : R(0);
    R fs[2][9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fs[0][i] = wgt<R>(i) * r1;
        fs[1][i] = wgt<R>(i) * r2;
    }
    pop_store_node<P>(g, p, f, x, y, fs, r1, r2);
    if (x == g.nx - 1) {
        d5[y] = fs[0][3];
        d5[g.ny + y] = fs[0][6];
        d5[2 * g.ny + y] = fs[0][7];
    }
    if (x == 0) {
        d5[3 * g.ny + y] = fs[1][1];
        d5[4 * g.ny + y] = fs[1][5];
        d5[5 * g.ny + y] = fs[1][8];
    }
}

template <class P>
__global__ void import_kernel(Geometry g, Params p, const double *src, typename P::store_t *f,
                              typename P::real_t *d5) {
    using R = typename P::real_t;
    const long long n = (long long)g.nx * g.ny;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const bool fluid = g.geo[(long long)y * g.gpitch + GEO_HX + x] == GEO_FLUID;
    R fs[2][9];
    R r[2] = {R(0), R(0)};
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fs[c][i] = fluid ? R(src[(c * 9 + i) * n + k]) : R(0);
            r[c] += fs[c][i];
        }
    pop_store_node<P>(g, p, f, x, y, fs, r[0], r[1]);
    if (x == g.nx - 1) {
        d5[y] = fs[0][3];
        d5[g.ny + y] = fs[0][6];
        d5[2 * g.ny + y] = fs[0][7];
    }
    if (x == 0) {
        d5[3 * g.ny + y] = fs[1][1];
        d5[4 * g.ny + y] = fs[1][5];
        d5[5 * g.ny + y] = fs[1][8];
    }
}

template <class P>
__global__ void export_kernel(Geometry g, const typename P::store_t *f, double *dst) {
    const long long n = (long long)g.nx * g.ny;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long site = site_of(g, x, y);
    const bool fluid = g.geo[(long long)y * g.gpitch + GEO_HX + x] == GEO_FLUID;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            dst[(c * 9 + i) * n + k] = fluid ? (double)pop_load<P>(f, g.plane, c, i, site) : 0.0;
}

// Geometry ghost columns for the current x boundary mode: with periodic x
// the hx columns on each side repeat the opposite edge (matching the
// population ghosts); everything else outside 0..nx-1 is outside.
__global__ void geo_ghost_kernel(Geometry g, int open_x) {
    const int y = blockIdx.x;
    uint8_t *row = const_cast<uint8_t *>(g.geo) + (long long)y * g.gpitch;
    for (int c = threadIdx.x; c < g.gpitch; c += blockDim.x) {
        const int x = c - GEO_HX;
        if (x >= 0 && x < g.nx) continue;
        uint8_t code = GEO_OUTSIDE;
        if (!open_x && x >= -g.hx && x < g.nx + g.hx) code = row[GEO_HX + pmod(x, g.nx)];
        row[c] = code;
    }
}

// Population ghost columns for periodic x: copy the hx edge columns of
// every plane of the current state to the opposite side (rows 0..ny-1).
template <class P>
__global__ void pop_ghost_cols_kernel(Geometry g, typename P::store_t *f) {
    const int y = blockIdx.x;
    const int ng = 2 * g.hx;
    for (int k = threadIdx.x; k < P::planes * ng; k += blockDim.x) {
        const int pl = k / ng, j = k % ng;
        const int gx = j < g.hx ? j - g.hx : g.nx + (j - g.hx);
        const long long base = (long long)pl * g.plane;
        f[base + site_of(g, gx, y)] = f[base + site_of(g, pmod(gx, g.nx), y)];
    }
}

// Population ghost rows for periodic y: copy whole rows (ghost columns
// included) of every plane to the rows beyond the opposite edge.
template <class P>
__global__ void pop_ghost_rows_kernel(Geometry g, typename P::store_t *f) {
    const int j = blockIdx.x;  // 0..2 HY - 1
    const int gy = j < HY ? j - HY : g.ny + (j - HY);
    const int sy = pmod(gy, g.ny);
    for (long long k = threadIdx.x; k < (long long)P::planes * g.pitch; k += blockDim.x) {
        const long long base = (k / g.pitch) * g.plane;
        const int col = (int)(k % g.pitch);
        f[base + (long long)(gy + HY) * g.pitch + col] = f[base + (long long)(sy + HY) * g.pitch + col];
    }
}

// Padded copy of the geometry for the tensor copies of the tile kernel:
// row r holds lattice row r - HY (ghost columns included); rows beyond the
// lattice repeat the opposite edge when y is periodic and are outside
// otherwise, as are the spare rows at the end.
__global__ void geo_pad_kernel(Geometry g, uint8_t *pad, int rows, int periodic_y) {
    const int r = blockIdx.x;
    const int y = r - HY;
    int src = -1;
    if (y >= 0 && y < g.ny) src = y;
    else if (periodic_y && y >= -HY && y < g.ny + HY) src = pmod(y, g.ny);
    for (int c = threadIdx.x; c < g.gpitch; c += blockDim.x)
        pad[(long long)r * g.gpitch + c] = src >= 0 ? g.geo[(long long)src * g.gpitch + c] : GEO_OUTSIDE;
}

template <class P>
__device__ __forceinline__ void node_rho(const Geometry &g, const typename P::store_t *f,
                                         long long site, typename P::real_t &r1,
                                         typename P::real_t &r2) {
    r1 = 0;
    r2 = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        r1 += pop_load<P>(f, g.plane, 0, i, site);
        r2 += pop_load<P>(f, g.plane, 1, i, site);
    }
}

__device__ __forceinline__ bool is_fluid(const Geometry &g, int x, int y) {
    return g.geo[(long long)y * g.gpitch + GEO_HX + x] == GEO_FLUID;
}

// ---------------------------------------------------------------------------
// Diagnostics: per-block partial sums (FP64) in a scratch array, then a
// single-block pass that adds the partials in block order, so the result
// does not depend on scheduling.
//   acc[0] mass1  acc[1] mass2  acc[2] fluid nodes  acc[3] water nodes
//   acc[4] P_in sum  acc[5] P_in count  acc[6] P_out sum  acc[7] P_out count
//   acc[8] nodes with a non-finite or negative density
// ---------------------------------------------------------------------------
constexpr int NACC = 9;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool pressure_site(const Geometry &g, const Params &p, int x, int y) {
    // more than 2 nodes in y from any solid node of the column (Sec. 2.3:
    // the average leaves out the values near the walls)
    for (int d = -2; d <= 2; ++d) {
        int yy = y + d;
        if (yy < 0 || yy >= g.ny) {
            if (!p.periodic_y) return false;
            yy = (yy + g.ny) % g.ny;
        }
        if (!is_fluid(g, x, yy)) return false;
    }
    return true;
}

template <class P>
__global__ void __launch_bounds__(BLK) diag_partial_kernel(Geometry g, Params p,
                                                           const typename P::store_t *f,
                                                           double *partial) {
    using R = typename P::real_t;
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    const long long n = (long long)g.nx * g.ny;
    for (long long k = (long long)blockIdx.x * BLK + threadIdx.x; k < n;
         k += (long long)gridDim.x * BLK) {
        const int x = (int)(k % g.nx), y = (int)(k / g.nx);
        const long long site = site_of(g, x, y);
        if (!is_fluid(g, x, y)) continue;
        R r1, r2;
        node_rho<P>(g, f, site, r1, r2);
        const double d1 = (double)r1, d2 = (double)r2;
        acc[0] += d1;
        acc[1] += d2;
        acc[2] += 1.0;
        acc[3] += (d2 > d1) ? 1.0 : 0.0;
        if (!(d1 >= 0.0) || !(d2 >= 0.0) || !isfinite(d1) || !isfinite(d2)) acc[8] += 1.0;
        if ((x == 0 || x == g.nx - 1) && pressure_site(g, p, x, y)) {
            const double P_ = (d1 + d2) / 3.0 + p.g_coh / 3.0 * d1 * d2;  // Eq. 14
            const int o = x == 0 ? 4 : 6;
            acc[o] += P_;
            acc[o + 1] += 1.0;
        }
    }
    __shared__ double red[BLK / 32][NACC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NACC) {
        double s = 0.0;
        for (int w = 0; w < BLK / 32; ++w) s += red[w][threadIdx.x];
        partial[(long long)blockIdx.x * NACC + threadIdx.x] = s;
    }
}

__global__ void diag_final_kernel(const double *partial, int nblocks, double *out,
                                  unsigned long long *bad) {
    __shared__ double tot[NACC];
    if (threadIdx.x < NACC) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * NACC + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ULL);
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = tot[2] > 0 ? tot[3] / tot[2] : nan;
        out[3] = (tot[0] + tot[1]) > 0 ? tot[1] / (tot[0] + tot[1]) : nan;
        out[4] = tot[5] > 0 ? tot[4] / tot[5] : nan;
        out[5] = tot[7] > 0 ? tot[6] / tot[7] : nan;
        out[6] = out[4] - out[5];
        out[7] = tot[2];
        if (bad && tot[8] > 0) atomicAdd(bad, (unsigned long long)tot[8]);
    }
}

// ---------------------------------------------------------------------------
// Field read-outs into dense [ny][nx] arrays.
// ---------------------------------------------------------------------------
template <class P>
__global__ void density_kernel(Geometry g, const typename P::store_t *f, int comp, double *out) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long site = site_of(g, x, y);
    R r = 0;
    if (is_fluid(g, x, y))
#pragma unroll
        for (int i = 0; i < 9; ++i) r += pop_load<P>(f, g.plane, comp, i, site);
    out[k] = (double)r;
}

template <class P>
__global__ void pressure_kernel(Geometry g, Params p, const typename P::store_t *f, double *out) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long site = site_of(g, x, y);
    double v = 0.0;
    if (is_fluid(g, x, y)) {
        R r1, r2;
        node_rho<P>(g, f, site, r1, r2);
        v = ((double)r1 + (double)r2) / 3.0 + p.g_coh / 3.0 * (double)r1 * (double)r2;
    }
    out[k] = v;
}

template <class P>
__global__ void phase_kernel(Geometry g, const typename P::store_t *f, float *out) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long site = site_of(g, x, y);
    float v = 0.0f;
    if (is_fluid(g, x, y)) {
        R r1, r2;
        node_rho<P>(g, f, site, r1, r2);
        v = (float)((r1 - r2) / (r1 + r2));
    }
    out[k] = v;
}

// Velocity read-out.  The stored state is post-collision; summing Eq. 1's
// first moment over both components gives J* = J + F (with the half-force
// velocity shift) or J* = J + (1 - 1/(2 tau_s)) F (without), so the velocity
// of the last collision is recovered from J*, the densities and the force
// of the same state: u = (J* - F/2)/rho, resp. (J* - (1 - 1/(2 tau_s)) F)/rho.
// Pass 1: densities; pass 2: pseudopotentials with virtual solid densities;
// pass 3: force and velocity.
template <class P>
__global__ void vel_rho_kernel(Geometry g, const typename P::store_t *f,
                               typename P::real_t *rho) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    R r1 = 0, r2 = 0;
    if (is_fluid(g, x, y)) node_rho<P>(g, f, site_of(g, x, y), r1, r2);
    const long long n = (long long)g.nx * g.ny;
    rho[k] = r1;
    rho[n + k] = r2;
}

template <class R>
__global__ void vel_psi_kernel(Geometry g, Params p, const R *rho, R *psi) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long n = (long long)g.nx * g.ny;
    const uint8_t code = g.geo[(long long)y * g.gpitch + GEO_HX + x];
    if (code == GEO_FLUID) {
        psi[k] = rho[k];
        psi[n + k] = rho[n + k];
        return;
    }
    R n1 = 0, n2 = 0, den = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int nx_ = x + ex(i), ny_ = y + ey(i);
        if (geo_at(g, p, nx_, ny_) != GEO_FLUID) continue;
        nx_ = pmod(nx_, g.nx);
        ny_ = pmod(ny_, g.ny);
        const long long ns = (long long)ny_ * g.nx + nx_;
        const R w = wgt<R>(i);
        n1 += w * rho[ns];
        n2 += w * rho[n + ns];
        den += w;
    }
    R s1 = 0, s2 = 0;
    if (den > R(0)) {
        s1 = chi_at<R>(g, 2 * code) * n1 / den;
        s2 = chi_at<R>(g, 2 * code + 1) * n2 / den;
    }
    psi[k] = s1;
    psi[n + k] = s2;
}

template <class P>
__global__ void vel_final_kernel(Geometry g, Params p, const typename P::store_t *f,
                                 const typename P::real_t *rho, const typename P::real_t *psi,
                                 double *ux_out, double *uy_out) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    const int x = (int)(k % g.nx), y = (int)(k / g.nx);
    const long long site = site_of(g, x, y);
    const long long n = (long long)g.nx * g.ny;
    if (!is_fluid(g, x, y)) {
        ux_out[k] = 0.0;
        uy_out[k] = 0.0;
        return;
    }
    const R r1 = rho[k], r2 = rho[n + k];
    const bool mirror_in = p.open_x && x == 0;
    const bool mirror_out = p.open_x && x == g.nx - 1;
    R fx1, fy1, fx2, fy2;
    node_force<R>(p, r1, r2,
                  [&](int i, uint8_t &code, R &s1, R &s2) {
                      int dx = ex(i), dy = ey(i);
                      if ((mirror_in && dx < 0) || (mirror_out && dx > 0)) {
                          dx = -dx;
                          dy = -dy;
                      }
                      code = geo_at(g, p, x + dx, y + dy);
                      s1 = s2 = R(0);
                      if (code != GEO_OUTSIDE) {
                          const long long ns =
                              (long long)pmod(y + dy, g.ny) * g.nx + pmod(x + dx, g.nx);
                          s1 = psi[ns];
                          s2 = psi[n + ns];
                      }
                  },
                  fx1, fy1, fx2, fy2);
    R jx = 0, jy = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R fi = pop_load<P>(f, g.plane, 0, i, site) + pop_load<P>(f, g.plane, 1, i, site);
        jx += R(ex(i)) * fi;
        jy += R(ey(i)) * fi;
    }
    const R rho_t = r1 + r2;
    const R Fx = fx1 + fx2, Fy = fy1 + fy2;
    R c = R(0.5);
    if (!p.vel_shift) {
        const R tau = (r1 * par<R>(p.nu1, p.nu1_f) + r2 * par<R>(p.nu2, p.nu2_f)) * R(3) / rho_t + R(0.5);
        c = R(1) - R(0.5) / tau;
    }
    ux_out[k] = (double)((jx - c * Fx) / rho_t);
    uy_out[k] = (double)((jy - c * Fy) / rho_t);
}

Geometry geometry_of(const Lattice &L) { return L.geometry(); }

template <class F>
cudaError_t dispatch(const Lattice &L, F &&fn) {
    switch (L.prec) {
        case MCLBM_FP64: return fn(P64{});
        case MCLBM_FP32: return fn(P32{});
        case MCLBM_FP32_DEV: return fn(P32D{});
        case MCLBM_FP16_DEV: return fn(P16D{});
        default: return fn(PB16D{});
    }
}

// Warm-start blend in place: at a fluid node whose predicted phase field
// phi_hat lies on the other side of zero from the node's own phase
// (rho1 > rho2 is component 1's side) and by more than `flip`, the node is
// re-initialised at rest, f_i = w_i rho^sigma (Eq. 2 at u = 0), with the
// separated-phase densities of phi_hat: rho1 = lo + (hi - lo)(1 + phi)/2,
// rho2 = lo + (hi - lo)(1 - phi)/2, phi clamped to [-1, 1].  Every other
// node keeps its populations, so the previous equilibrium survives
// wherever no change of phase is predicted.  The number of replaced nodes
// is added to *changed (one atomic per warp).
template <class P>
__global__ void blend_phase_kernel(Geometry g, Params p, typename P::store_t *f, const float *phi,
                                   double hi, double lo, double flip, unsigned long long *changed) {
    using R = typename P::real_t;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool change = false;
    if (k < (long long)g.nx * g.ny) {
        const int x = (int)(k % g.nx), y = (int)(k / g.nx);
        if (is_fluid(g, x, y)) {
            R r1, r2;
            node_rho<P>(g, f, site_of(g, x, y), r1, r2);
            const double ph = fmin(1.0, fmax(-1.0, (double)phi[k]));
            change = ((ph > 0.0) != (r1 > r2)) && fabs(ph) > flip;
            if (change) {
                const R n1 = R(lo + (hi - lo) * (1.0 + ph) * 0.5), n2 = R(lo + (hi - lo) * (1.0 - ph) * 0.5);
                R fs[2][9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    fs[0][i] = wgt<R>(i) * n1;
                    fs[1][i] = wgt<R>(i) * n2;
                }
                pop_store_node<P>(g, p, f, x, y, fs, n1, n2);
            }
        }
    }
    const unsigned int votes = __ballot_sync(0xffffffffu, change);
    if ((threadIdx.x & 31) == 0 && votes) atomicAdd(changed, (unsigned long long)__popc(votes));
}

}  // namespace

int diag_blocks_for(const Lattice &L) {
    long long n = (long long)L.nx * L.ny;
    int b = blocks_for(n, BLK * 8);
    return b < 1 ? 1 : (b > 1216 ? 1216 : b);
}

// Component densities from a phase field: rho1 = lo + (hi - lo)(1 + phi)/2,
// rho2 = lo + (hi - lo)(1 - phi)/2, phi clamped to [-1, 1].
__global__ void phase_densities_kernel(const float *phi, long long n, double hi, double lo, double *r1,
                                       double *r2) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double p = fmin(1.0, fmax(-1.0, (double)phi[k]));
    r1[k] = lo + (hi - lo) * (1.0 + p) * 0.5;
    r2[k] = lo + (hi - lo) * (1.0 - p) * 0.5;
}

cudaError_t launch_phase_densities(Lattice &L, const float *phi, double hi, double lo, double *r1,
                                   double *r2) {
    const long long n = (long long)L.nx * L.ny;
    phase_densities_kernel<<<blocks_for(n), BLK, 0, L.stream>>>(phi, n, hi, lo, r1, r2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_blend_phase(Lattice &L, const float *phi, double hi, double lo, double flip,
                               unsigned long long *changed) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        blend_phase_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, L.p, static_cast<typename P::store_t *>(L.f[L.cur]), phi, hi, lo, flip, changed);
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_init_equilibrium(Lattice &L, const double *rho1, const double *rho2) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        init_equilibrium_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, L.p, rho1, rho2, static_cast<typename P::store_t *>(L.f[L.cur]),
            static_cast<typename P::real_t *>(L.d5));
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_set_populations(Lattice &L, const double *src) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        import_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, L.p, src, static_cast<typename P::store_t *>(L.f[L.cur]),
            static_cast<typename P::real_t *>(L.d5));
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_get_populations(Lattice &L, double *dst) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        export_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, static_cast<const typename P::store_t *>(L.f[L.cur]), dst);
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_diagnostics(Lattice &L) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        diag_partial_kernel<P><<<L.diag_blocks, BLK, 0, L.stream>>>(
            g, L.p, static_cast<const typename P::store_t *>(L.f[L.cur]), L.diag_partial);
        diag_final_kernel<<<1, 32, 0, L.stream>>>(L.diag_partial, L.diag_blocks, L.diag_out,
                                                  L.bad_flag);
        count_launch(2);
        return cudaGetLastError();
    });
}

cudaError_t launch_geo_ghosts(Lattice &L) {
    geo_ghost_kernel<<<L.ny, 128, 0, L.stream>>>(geometry_of(L), L.p.open_x);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (L.geo_pad) {
        geo_pad_kernel<<<L.geo_pad_rows, 128, 0, L.stream>>>(geometry_of(L), L.geo_pad,
                                                             L.geo_pad_rows, L.p.periodic_y);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        auto *f = static_cast<typename P::store_t *>(L.f[L.cur]);
        if (!L.p.open_x) {
            pop_ghost_cols_kernel<P><<<L.ny, 128, 0, L.stream>>>(g, f);
            count_launch();
        }
        if (L.p.periodic_y) {
            pop_ghost_rows_kernel<P><<<2 * HY, 256, 0, L.stream>>>(g, f);
            count_launch();
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_density(Lattice &L, int comp, double *out) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        density_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, static_cast<const typename P::store_t *>(L.f[L.cur]), comp, out);
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_pressure(Lattice &L, double *out) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        pressure_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, L.p, static_cast<const typename P::store_t *>(L.f[L.cur]), out);
        count_launch();
        return cudaGetLastError();
    });
}

cudaError_t launch_phase(Lattice &L, float *out) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        phase_kernel<P><<<blocks_for((long long)L.nx * L.ny), BLK, 0, L.stream>>>(
            g, static_cast<const typename P::store_t *>(L.f[L.cur]), out);
        count_launch();
        return cudaGetLastError();
    });
}

size_t velocity_scratch_bytes(const Lattice &L) {
    return 4 * (size_t)L.nx * L.ny * L.real_bytes;
}

cudaError_t launch_velocity(Lattice &L, double *ux, double *uy, void *scratch) {
    const Geometry g = geometry_of(L);
    return dispatch(L, [&](auto tag) {
        using P = decltype(tag);
        using R = typename P::real_t;
        R *rho = static_cast<R *>(scratch);
        R *psi = rho + 2 * (long long)g.nx * g.ny;
        const int nb = blocks_for((long long)L.nx * L.ny);
        const auto *f = static_cast<const typename P::store_t *>(L.f[L.cur]);
        vel_rho_kernel<P><<<nb, BLK, 0, L.stream>>>(g, f, rho);
        vel_psi_kernel<R><<<nb, BLK, 0, L.stream>>>(g, L.p, rho, psi);
        vel_final_kernel<P><<<nb, BLK, 0, L.stream>>>(g, L.p, f, rho, psi, ux, uy);
        count_launch(3);
        return cudaGetLastError();
    });
}

}  // namespace mclbm
