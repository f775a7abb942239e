// Fused stream-collide-force kernel, row-sweeping strip variant (default).
//
// One CTA of W threads owns a strip of W columns and a band of rows, and
// walks down it one row per iteration.  Raw post-collision rows (all
// direction planes, plus HX ghost/halo columns on each side, plus the
// geometry row) are staged in a ring of NR shared-memory slots by TMA bulk
// copies (cp.async.bulk, completion on an mbarrier per slot), issued several
// rows ahead by one thread.  Every population is read from HBM once and
// from shared memory twice:
//   stage A(q): pull + bounce-back + Set-3 for row q over the strip and a
//               2-column halo; component densities (Eq. 3) into a 5-row ring
//   stage B(q): improved virtual solid densities (Eqs. 16-17) of the solid
//               nodes of row q over the strip and a 1-column halo
//   stage C(q): pull again for the strip's own nodes, forces (Eqs. 12-15
//               with the boundary mirror), tau_s and u (Eqs. 6-9), forced
//               collision (Eqs. 1, 2, 11), coalesced stores
// Iteration k runs A(q+2), B(q+1), C(q) with q = y_lo + k - 4, so C(q) sees
// the densities of rows q-2..q+2 and the virtual densities of rows q-1..q+1.
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer);
// on expiry the CTA records MCLBM_ERR_TIMEOUT in the error word, waits a
// bounded time for the copies it issued, and returns.
#include "async_copy.cuh"
#include "lbm_device.cuh"

namespace mclbm {

namespace {

template <class P, int W, int NR>
struct SweepLayout {
    using S = typename P::store_t;
    using R = typename P::real_t;
    static constexpr int HX = P::hx;
    static constexpr int NPL = P::planes;
    static constexpr int RW = W + 2 * HX;          // staged population row width
    static constexpr int GW = W + 2 * GEO_HX;      // staged geometry row width (bytes)
    static constexpr int RHO_W = W + 4;            // density ring row width
    static constexpr size_t raw_bytes = (size_t)NR * NPL * RW * sizeof(S);
    static constexpr size_t geo_off = raw_bytes;
    static constexpr size_t geo_bytes = (size_t)NR * GW;
    static constexpr size_t rho_off = (geo_off + geo_bytes + 15) / 16 * 16;
    static constexpr size_t rho_bytes = (size_t)5 * 2 * RHO_W * sizeof(R);
    static constexpr size_t bar_off = (rho_off + rho_bytes + 15) / 16 * 16;
    static constexpr size_t total = bar_off + NR * sizeof(uint64_t);
    static constexpr uint32_t row_tx = (uint32_t)(NPL * RW * sizeof(S) + GW);
    static_assert((RW * sizeof(S)) % 16 == 0, "bulk copy size must be a multiple of 16 bytes");
    static_assert(GW % 16 == 0, "geometry copy size must be a multiple of 16 bytes");
    static_assert(HX >= 3, "halo must cover the stencil reach");
};

template <class P, int W, int NR>
__global__ void __launch_bounds__(W) sweep_step_kernel(const StepArgs a) {
    using L = SweepLayout<P, W, NR>;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int HX = L::HX, RW = L::RW, GW = L::GW, NPL = L::NPL, RHO_W = L::RHO_W;

    extern __shared__ __align__(128) unsigned char smem[];
    S *raw = reinterpret_cast<S *>(smem);
    uint8_t *geo = smem + L::geo_off;
    R *rho = reinterpret_cast<R *>(smem + L::rho_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);

    const Geometry &g = a.g;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int y_lo = blockIdx.y * a.rows_per_cta;
    if (y_lo >= g.ny) return;
    const int y_hi = min(y_lo + a.rows_per_cta, g.ny);
    const int nraw = (y_hi - y_lo) + 6;  // rows y_lo-3 .. y_hi+2
    const S *fin = static_cast<const S *>(a.fin);

    auto raw_at = [&](int slot, int plane, int idx) -> S { return raw[(slot * NPL + plane) * RW + idx]; };
    auto geo_at_s = [&](int slot, int lx) -> uint8_t { return geo[slot * GW + GEO_HX + lx]; };
    auto rho_ring = [&](int q, int c, int lx) -> R & {
        return rho[(((q - y_lo + 2) % 5) * 2 + c) * RHO_W + lx + 2];
    };

    // producer: stage raw row j (lattice row y_lo - 3 + j) into slot j % NR
    auto issue = [&](int j) {
        const int slot = j % NR;
        const int q = y_lo - 3 + j;
        if ((q >= 0 && q < g.ny) || a.p.periodic_y) {
            const int qq = pmod(q, g.ny);
            fence_proxy_async();
            mbar_expect_tx(&bar[slot], L::row_tx);
            // element x0 - HX of the row is column x0 + hx - HX = x0 in memory
            const S *src = fin + (long long)(qq + HY) * g.pitch + x0;
            for (int p = 0; p < NPL; ++p)
                bulk_g2s(raw + (slot * NPL + p) * RW, src + (long long)p * g.plane,
                         RW * sizeof(S), &bar[slot]);
            bulk_g2s(geo + slot * GW, g.geo + (long long)qq * g.gpitch + x0, GW, &bar[slot]);
        } else {
            // a row beyond a wall edge: nothing to copy, mark it outside
            uint32_t *gw = reinterpret_cast<uint32_t *>(geo + slot * GW);
            for (int k = 0; k < GW / 4; ++k) gw[k] = 0xffffffffu;
            mbar_arrive(&bar[slot]);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < NR; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0) {
        for (; issued < NR && issued < nraw; ++issued) issue(issued);
    }

    // populations of node lx of row q (raw index j of row q), pulled from the
    // staged rows: stream, bounce-back, Set-3
    auto pull = [&](int q, int jq, int lx, R f[2][9]) {
        const int x = x0 + lx;
        const int s0 = jq % NR;
        const bool at_in = a.p.open_x && x == 0;
        const bool at_out = a.p.open_x && x == g.nx - 1;
        auto dec = [&](int slot, int c, int i, int idx) -> R {
            R v = to_real(raw_at(slot, c * 9 + i, idx));
            if constexpr (P::ref) v += wgt<R>(i) * to_real(raw_at(slot, 18 + c, idx));
            return v;
        };
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const bool missing = (at_in && ex(i) == 1) || (at_out && ex(i) == -1);
            if (missing) {
                f[0][i] = R(0);
                f[1][i] = R(0);
                continue;
            }
            const int ss = (jq - ey(i)) % NR;
            if (i != 0 && geo_at_s(ss, lx - ex(i)) != GEO_FLUID) {
                f[0][i] = dec(s0, 0, opp(i), lx + HX);
                f[1][i] = dec(s0, 1, opp(i), lx + HX);
            } else {
                f[0][i] = dec(ss, 0, i, lx - ex(i) + HX);
                f[1][i] = dec(ss, 1, i, lx - ex(i) + HX);
            }
        }
        // halo rows of a periodic-y lattice lie outside 0..ny-1: the outlet
        // values of Eq. 26 are indexed by the wrapped row
        apply_open_bc<R>(a, x, pmod(q, g.ny), [&](int c, int i) { return dec(s0, c, i, lx + HX); }, f);
    };

    bool bad = false;    // this thread saw a wait run out
    bool abort = false;  // some thread of the CTA did (uniform)
    int waited = 0;
    const int K = (y_hi - y_lo) + 4;
    for (int k = 0; k < K; ++k) {
        while (waited <= k + 2 && waited < nraw) {
            bad |= !mbar_wait(&bar[waited % NR], (waited / NR) & 1, a.wait_ns);
            ++waited;
        }
        // ---- A: densities of row qA over columns -2 .. W+1 -------------------
        const int qA = y_lo - 2 + k;
        const int jA = k + 1;
        for (int lx = tid - 2; lx < W + 2; lx += W) {
            R r1 = 0, r2 = 0;
            if (geo_at_s(jA % NR, lx) == GEO_FLUID) {
                R f[2][9];
                pull(qA, jA, lx, f);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    r1 += f[0][i];
                    r2 += f[1][i];
                }
            }
            rho_ring(qA, 0, lx) = r1;
            rho_ring(qA, 1, lx) = r2;
        }
        if (__syncthreads_or(bad)) {
            abort = true;
            break;
        }
        // ---- producer: refill the slot of raw row k-3 -------------------------
        if (tid == 0 && k >= 3 && issued < nraw && issued == k - 3 + NR) {
            issue(issued);
            ++issued;
        }
        // ---- B: virtual solid densities of row qB over columns -1 .. W --------
        const int qB = qA - 1;
        if (k >= 2) {
            const int jB = k;
            for (int lx = tid - 1; lx < W + 1; lx += W) {
                const uint8_t code = geo_at_s(jB % NR, lx);
                if (code == GEO_FLUID || code == GEO_OUTSIDE) continue;
                R n1 = 0, n2 = 0, den = 0;
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    if (geo_at_s((jB + ey(i)) % NR, lx + ex(i)) == GEO_FLUID) {
                        const R w = wgt<R>(i);
                        n1 += w * rho_ring(qB + ey(i), 0, lx + ex(i));
                        n2 += w * rho_ring(qB + ey(i), 1, lx + ex(i));
                        den += w;
                    }
                }
                R s1 = 0, s2 = 0;
                if (den > R(0)) {
                    const R inv = R(1) / den;
                    s1 = chi_at<R>(g, 2 * code) * n1 * inv;
                    s2 = chi_at<R>(g, 2 * code + 1) * n2 * inv;
                }
                rho_ring(qB, 0, lx) = s1;
                rho_ring(qB, 1, lx) = s2;
            }
        }
        __syncthreads();
        // ---- C: collision of row qC -------------------------------------------
        const int qC = qA - 2;
        if (k >= 4) {
            const int jC = k - 1;
            const int lx = tid;
            const int x = x0 + lx;
            if (x < g.nx && geo_at_s(jC % NR, lx) == GEO_FLUID) {
                R f[2][9];
                pull(qC, jC, lx, f);
                R rho1 = 0, rho2 = 0;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    rho1 += f[0][i];
                    rho2 += f[1][i];
                }
                const bool mirror_in = a.p.open_x && x == 0;
                const bool mirror_out = a.p.open_x && x == g.nx - 1;
                R fx1, fy1, fx2, fy2;
                node_force<R>(a.p, rho1, rho2,
                              [&](int i, uint8_t &code, R &s1, R &s2) {
                                  int dx = ex(i), dy = ey(i);
                                  // Sec. 2.1: a neighbour beyond an open end is
                                  // replaced by the one in the opposite direction
                                  if ((mirror_in && dx < 0) || (mirror_out && dx > 0)) {
                                      dx = -dx;
                                      dy = -dy;
                                  }
                                  code = geo_at_s((jC + dy) % NR, lx + dx);
                                  s1 = rho_ring(qC + dy, 0, lx + dx);
                                  s2 = rho_ring(qC + dy, 1, lx + dx);
                              },
                              fx1, fy1, fx2, fy2);
                R omega, ux, uy;
                node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
                collide<R>(a.p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
                pop_store_node<P>(g, a.p, static_cast<S *>(a.fout), x, qC, f, rho1, rho2);
            }
        }
    }
    if (abort && tid == 0) {
        atomicExch(a.err, MCLBM_ERR_TIMEOUT);
        // let the copies this CTA issued land before its shared memory goes
        for (int j = waited; j < issued; ++j) mbar_wait(&bar[j % NR], (j / NR) & 1, DRAIN_LIMIT_NS);
    }
}

template <class P, int W, int NR>
cudaError_t launch_sweep_cfg(Lattice &L, StepArgs a) {
    using Lay = SweepLayout<P, W, NR>;
    // resident CTA slots of this kernel on the device (queried once)
    static int slots = 0;
    if (slots == 0) {
        cudaError_t e = cudaFuncSetAttribute(sweep_step_kernel<P, W, NR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, L.device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_step_kernel<P, W, NR>, W,
                                                      Lay::total);
        slots = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
    }
    const int strips = (L.nx + W - 1) / W;
    // bands of rows so that the grid fills the resident CTA slots about
    // twice; a band is at least 16 rows (the pipeline start costs 6 rows)
    int bands = (2 * slots + strips - 1) / strips;
    int rows = (L.ny + bands - 1) / bands;
    if (rows < 16) rows = 16;
    bands = (L.ny + rows - 1) / rows;
    a.rows_per_cta = rows;
    dim3 grid(strips, bands);
    sweep_step_kernel<P, W, NR><<<grid, W, Lay::total, L.stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool sweep_supported(const Lattice &L) {
    // the strip copies need the pitch and plane strides the layout provides
    return L.pitch >= ((L.nx + SWEEP_W - 1) / SWEEP_W) * SWEEP_W + 2 * L.hx;
}

cudaError_t launch_step_sweep(Lattice &L) {
    StepArgs a;
    a.g = L.geometry();
    a.p = L.p;
    a.p.round_fp32();
    a.fin = L.f[L.cur];
    a.fout = L.f[1 - L.cur];
    a.d5 = L.d5;
    a.err = L.err;
    a.wait_ns = L.wait_ns;
    a.rows_per_cta = 16;
    cudaError_t e;
    switch (L.prec) {
        case MCLBM_FP64: e = launch_sweep_cfg<P64, 64, 8>(L, a); break;
        case MCLBM_FP32: e = launch_sweep_cfg<P32, 128, 8>(L, a); break;
        case MCLBM_FP32_DEV: e = launch_sweep_cfg<P32D, 128, 7>(L, a); break;
        case MCLBM_FP16_DEV: e = launch_sweep_cfg<P16D, 128, 8>(L, a); break;
        default: e = launch_sweep_cfg<PB16D, 128, 8>(L, a); break;
    }
    if (e == cudaSuccess) L.cur = 1 - L.cur;
    return e;
}

}  // namespace mclbm
