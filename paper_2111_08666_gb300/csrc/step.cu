// Fused stream-collide-force kernel, 2-D tile variant: one launch per time
// step.  The row-sweeping strip kernel (sweep.cu) is the default; this one
// pulls straight from global memory and serves as the second, independent
// formulation that the strip kernel is checked against.
//
// One CTA owns a TX x TY tile.  The force at a node needs the pseudopotential
// of its 8 neighbours (Eq. 13), and a solid neighbour's virtual density
// needs the densities of that neighbour's fluid neighbours (Eq. 17), so the
// densities of the tile plus a 2-node ring are formed in shared memory from
// pulled populations (the ring's pulls mostly hit L2: they are the
// neighbouring tiles' own data).  Per node the kernel reads and writes each
// of the 18 populations once from HBM.
//
// Phases (one __syncthreads between each):
//   0  geometry codes of the tile + 3 ring into shared memory
//   1  pull + bounce-back + Set-3 for the tile (kept in registers) and the
//      2-ring; component densities (Eq. 3) into shared memory
//   2  virtual solid densities (Eqs. 16-17) of solid nodes in the 1-ring
//   3  forces (Eqs. 12-15, boundary mirror), tau_s and u (Eqs. 6-9),
//      collision (Eqs. 1, 2, 11), store
#include "lbm_device.cuh"

namespace mclbm {

template <class P, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) fused_step_kernel(const StepArgs a) {
    using R = typename P::real_t;
    using S = typename P::store_t;
    constexpr int NT = TX * TY;
    constexpr int RX = TX + 4, RY = TY + 4;  // density frame: tile + 2
    constexpr int GX = TX + 6, GY = TY + 6;  // geometry frame: tile + 3
    __shared__ uint8_t geo_s[GY][GX];
    __shared__ R rho_s[2][RY][RX];

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;

    for (int k = tid; k < GX * GY; k += NT) {
        const int gx = k % GX, gy = k / GX;
        const int x = x0 - 3 + gx, y = y0 - 3 + gy;
        uint8_t code = geo_at(a.g, a.p, x, y);
        // a node beyond the last row/column of a non-periodic edge, or past
        // the lattice in a ragged tile, is outside
        geo_s[gy][gx] = code;
    }
    __syncthreads();

    // ---- phase 1: own node -------------------------------------------------
    const int tx = tid % TX, ty = tid / TX;
    const int x = x0 + tx, y = y0 + ty;
    // In a ragged edge tile a position past the lattice is the periodic image
    // of a real node (or outside); its density is still needed by the ring.
    const bool fluid = geo_s[ty + 3][tx + 3] == GEO_FLUID;
    const bool own = (x < a.g.nx) && (y < a.g.ny) && fluid;
    R f[2][9];
    R rho1 = 0, rho2 = 0;
    if (fluid) {
        pull_node<P>(a, pmod(x, a.g.nx), pmod(y, a.g.ny),
                     [&](int i) { return geo_s[ty + 3 - ey(i)][tx + 3 - ex(i)]; }, f);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            rho1 += f[0][i];
            rho2 += f[1][i];
        }
    }
    rho_s[0][ty + 2][tx + 2] = rho1;
    rho_s[1][ty + 2][tx + 2] = rho2;

    // ---- phase 1: the 2-ring -----------------------------------------------
    constexpr int RING = 4 * RX + 4 * TY;
    for (int k = tid; k < RING; k += NT) {
        int rx, ry;
        if (k < 2 * RX) {
            ry = k / RX;
            rx = k % RX;
        } else if (k < 4 * RX) {
            const int kk = k - 2 * RX;
            ry = TY + 2 + kk / RX;
            rx = kk % RX;
        } else {
            const int kk = k - 4 * RX;
            ry = 2 + kk / 4;
            const int col = kk % 4;
            rx = col < 2 ? col : TX + col;
        }
        R r1 = 0, r2 = 0;
        if (geo_s[ry + 1][rx + 1] == GEO_FLUID) {
            const int gx = pmod(x0 - 2 + rx, a.g.nx);
            const int gy = pmod(y0 - 2 + ry, a.g.ny);
            R h[2][9];
            pull_node<P>(a, gx, gy, [&](int i) { return geo_s[ry + 1 - ey(i)][rx + 1 - ex(i)]; }, h);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                r1 += h[0][i];
                r2 += h[1][i];
            }
        }
        rho_s[0][ry][rx] = r1;
        rho_s[1][ry][rx] = r2;
    }
    __syncthreads();

    // ---- phase 2: virtual solid densities in the 1-ring and tile -------------
    constexpr int V = (TX + 2) * (TY + 2);
    for (int k = tid; k < V; k += NT) {
        const int rx = 1 + k % (TX + 2), ry = 1 + k / (TX + 2);
        const uint8_t code = geo_s[ry + 1][rx + 1];
        if (code == GEO_FLUID || code == GEO_OUTSIDE) continue;
        R n1 = 0, n2 = 0, den = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (geo_s[ry + 1 + ey(i)][rx + 1 + ex(i)] == GEO_FLUID) {
                const R w = wgt<R>(i);
                n1 += w * rho_s[0][ry + ey(i)][rx + ex(i)];
                n2 += w * rho_s[1][ry + ey(i)][rx + ex(i)];
                den += w;
            }
        }
        R s1 = 0, s2 = 0;
        if (den > R(0)) {
            const R inv = R(1) / den;
            s1 = chi_at<R>(a.g, 2 * code) * n1 * inv;
            s2 = chi_at<R>(a.g, 2 * code + 1) * n2 * inv;
        }
        rho_s[0][ry][rx] = s1;
        rho_s[1][ry][rx] = s2;
    }
    __syncthreads();

    // ---- phase 3: forces, collision, store -----------------------------------
    if (!own) return;
    const bool mirror_in = a.p.open_x && x == 0;
    const bool mirror_out = a.p.open_x && x == a.g.nx - 1;
    R fx1, fy1, fx2, fy2;
    node_force<R>(a.p, rho1, rho2,
                  [&](int i, uint8_t &code, R &s1, R &s2) {
                      int dx = ex(i), dy = ey(i);
                      // Sec. 2.1: a neighbour beyond an open end is replaced by
                      // the one in the opposite direction
                      if ((mirror_in && dx < 0) || (mirror_out && dx > 0)) {
                          dx = -dx;
                          dy = -dy;
                      }
                      code = geo_s[ty + 3 + dy][tx + 3 + dx];
                      s1 = rho_s[0][ty + 2 + dy][tx + 2 + dx];
                      s2 = rho_s[1][ty + 2 + dy][tx + 2 + dx];
                  },
                  fx1, fy1, fx2, fy2);
    R omega, ux, uy;
    node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
    collide<R>(a.p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
    pop_store_node<P>(a.g, a.p, static_cast<S *>(a.fout), x, y, f, rho1, rho2);
}

template <class P, int TX, int TY>
static cudaError_t launch_tile(Lattice &L, const StepArgs &a) {
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY);
    fused_step_kernel<P, TX, TY><<<grid, TX * TY, 0, L.stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_prec(Lattice &L, const StepArgs &a, int tile_cfg) {
    switch (tile_cfg) {
        case 1: return launch_tile<P, 32, 4>(L, a);
        case 2: return launch_tile<P, 64, 4>(L, a);
        case 3: return launch_tile<P, 32, 16>(L, a);
        default: return launch_tile<P, 32, 8>(L, a);
    }
}

cudaError_t launch_step_tile(Lattice &L, int tile_cfg) {
    StepArgs a;
    a.g = L.geometry();
    a.p = L.p;
    a.p.round_fp32();
    a.fin = L.f[L.cur];
    a.fout = L.f[1 - L.cur];
    a.d5 = L.d5;
    a.err = L.err;
    a.wait_ns = L.wait_ns;
    a.rows_per_cta = 0;
    cudaError_t e;
    switch (L.prec) {
        case MCLBM_FP64: e = launch_prec<P64>(L, a, tile_cfg); break;
        case MCLBM_FP32: e = launch_prec<P32>(L, a, tile_cfg); break;
        case MCLBM_FP32_DEV: e = launch_prec<P32D>(L, a, tile_cfg); break;
        case MCLBM_FP16_DEV: e = launch_prec<P16D>(L, a, tile_cfg); break;
        default: e = launch_prec<PB16D>(L, a, tile_cfg); break;
    }
    if (e == cudaSuccess) L.cur = 1 - L.cur;
    return e;
}

}  // namespace mclbm
