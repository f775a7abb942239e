// Fused stream-collide-force kernel, 2-D tile variant staged by TMA
// (default for the FP32 and deviation storages).
//
// One CTA owns a TX x TY tile.  One elected thread copies the tile and its
// 3-node ring, all direction planes at once, into shared memory with a
// single 3-D tensor copy (cp.async.bulk.tensor, completion on an mbarrier);
// the ghost columns and rows of the layout make that ring one rectangular
// box even at periodic edges.  Everything else reads shared memory:
//   lists   fluid positions of the density frame (tile + 2), solid positions
//           of the 1-ring, fluid nodes of the tile, compacted with warp
//           ballots so that lanes are not spent on solid nodes
//   A       pull + bounce-back + Set-3 and component densities (Eq. 3) on
//           the density frame
//   B       improved virtual solid densities (Eqs. 16-17) on the 1-ring
//   C       forces (Eqs. 12-15, boundary mirror), tau_s and u (Eqs. 6-9) and
//           the forced collision (Eqs. 1, 2, 11) of the tile's fluid nodes,
//           written into an output tile in shared memory
// and one tensor copy stores the output tile (whole 32-byte sectors, so no
// partially written sector has to be fetched first).  Ghost images of edge
// nodes are stored directly.  The wait for the input copy is bounded.
#include <cuda.h>

#include <cstring>

#include "async_copy.cuh"
#include "lbm_device.cuh"

namespace mclbm {

namespace {

template <class P, int TX, int TY>
struct TileLayout {
    using S = typename P::store_t;
    using R = typename P::real_t;
    static constexpr int NT = TX * TY;
    static constexpr int HX = P::hx;
    static constexpr int NPL = P::planes;
    static constexpr int RXW = TX + 2 * HX;  // staged input: columns x0-HX .. x0+TX+HX-1
    static constexpr int RYH = TY + 6;       // rows y0-3 .. y0+TY+2
    static constexpr int PSTR = RYH * RXW;   // plane stride of the staged input
    static constexpr int DXW = TX + 4;       // density frame: tile + 2
    static constexpr int DYH = TY + 4;
    static constexpr int GXW = TX + 8;       // geometry frame: columns x0-4 .. x0+TX+3
    static constexpr int GYH = TY + 6;
    static constexpr int N1 = DXW * DYH;
    static constexpr int N2 = (DXW - 2) * (DYH - 2);
    static constexpr int N3 = TX * TY;
    static constexpr size_t in_bytes = (size_t)NPL * PSTR * sizeof(S);
    static constexpr size_t out_off = (in_bytes + 127) / 128 * 128;
    static constexpr size_t out_bytes = (size_t)NPL * TY * TX * sizeof(S);
    static constexpr size_t rho_off = (out_off + out_bytes + 15) / 16 * 16;
    static constexpr size_t rho_bytes = (size_t)2 * N1 * sizeof(R);
    static constexpr size_t geo_off = (rho_off + rho_bytes + 15) / 16 * 16;
    static constexpr size_t geo_bytes = (size_t)GYH * GXW;
    static constexpr size_t l1_off = (geo_off + geo_bytes + 15) / 16 * 16;
    static constexpr size_t l2_off = l1_off + (size_t)N1 * 2;
    static constexpr size_t l3_off = l2_off + (size_t)N2 * 2;
    static constexpr size_t cnt_off = (l3_off + (size_t)N3 * 2 + 15) / 16 * 16;
    static constexpr size_t bar_off = cnt_off + 16;
    static constexpr size_t total = bar_off + 8;
    static_assert((RXW * sizeof(S)) % 16 == 0, "tensor box rows must be whole 16-byte chunks");
    static_assert((TX * sizeof(S)) % 16 == 0, "store box rows must be whole 16-byte chunks");
    static_assert(GXW % 4 == 0, "geometry rows are loaded as 32-bit words");
    static_assert(HX >= 3, "halo must cover the stencil reach");
};

// Append val to a shared list when flag is set; all 32 lanes of the warp
// must call it together.
__device__ __forceinline__ void list_append(bool flag, uint16_t val, uint16_t *list, int *count) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// One tile (bx, by) of one lattice.  The caller has initialised the
// mbarrier at bar_off; parity is the phase this tile's input copy completes.
// Returns false (uniformly over the CTA) if the wait for the copy ran out.
template <class P, int TX, int TY>
__device__ __forceinline__ bool tma_tile_body(const CUtensorMap *tin, const CUtensorMap *tout,
                                              const StepArgs &a, int bx, int by, uint32_t parity,
                                              unsigned char *smem) {
    using L = TileLayout<P, TX, TY>;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int NT = L::NT, HX = L::HX, RXW = L::RXW, PSTR = L::PSTR, DXW = L::DXW,
                  GXW = L::GXW;

    const S *in = reinterpret_cast<const S *>(smem);
    S *out = reinterpret_cast<S *>(smem + L::out_off);
    R *rho = reinterpret_cast<R *>(smem + L::rho_off);
    uint8_t *geo = smem + L::geo_off;
    uint16_t *l1 = reinterpret_cast<uint16_t *>(smem + L::l1_off);
    uint16_t *l2 = reinterpret_cast<uint16_t *>(smem + L::l2_off);
    uint16_t *l3 = reinterpret_cast<uint16_t *>(smem + L::l3_off);
    int *cnt = reinterpret_cast<int *>(smem + L::cnt_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);

    const Geometry &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * TX, y0 = by * TY;

    __syncthreads();  // a previous tile of this CTA is done with shared memory
    if (tid == 0) {
        cnt[0] = cnt[1] = cnt[2] = 0;
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)L::in_bytes);
        // element (x0 - HX, y0 - 3) is column x0, row y0 + HY - 3 in memory
        tma_load_3d(smem, tin, x0, y0 + HY - 3, 0, bar);
    }
    // geometry frame; rows beyond a wall edge are outside
    for (int k = tid; k < L::GYH * (GXW / 4); k += NT) {
        const int r = k / (GXW / 4), cw = k % (GXW / 4);
        const int y = y0 - 3 + r;
        uint32_t word = 0xffffffffu;
        if ((y >= 0 && y < g.ny) || a.p.periodic_y) {
            const int yy = pmod(y, g.ny);
            word = *reinterpret_cast<const uint32_t *>(g.geo + (long long)yy * g.gpitch + GEO_HX +
                                                       x0 - 4 + 4 * cw);
        }
        reinterpret_cast<uint32_t *>(geo)[k] = word;
    }
    __syncthreads();
    auto geo_s = [&](int r, int c) -> uint8_t { return geo[r * GXW + c]; };

    // ---- work lists ---------------------------------------------------------
    // L1: fluid positions of the density frame that no collision thread
    // pulls: the 2-ring, and in a ragged edge tile the positions past the
    // lattice edge (periodic images whose densities the edge nodes need).
    // The tile's own nodes are pulled by the threads that collide them (L3).
    for (int base = warp * 32; base < L::N1; base += NT) {
        const int k = base + lane;
        bool f = false;
        if (k < L::N1) {
            const int dr = k / DXW, dc = k % DXW;
            const bool own = dr >= 2 && dr < TY + 2 && dc >= 2 && dc < TX + 2 &&
                             x0 - 2 + dc < g.nx && y0 - 2 + dr < g.ny;
            const bool fl = geo_s(dr + 1, dc + 2) == GEO_FLUID;
            if (!fl || own) {
                rho[k] = R(0);
                rho[L::N1 + k] = R(0);
            }
            f = fl && !own;
        }
        list_append(f, (uint16_t)k, l1, &cnt[0]);
    }
    for (int base = warp * 32; base < L::N2; base += NT) {
        const int k = base + lane;
        bool f = false;
        int pos = 0;
        if (k < L::N2) {
            const int dr = 1 + k / (DXW - 2), dc = 1 + k % (DXW - 2);
            const uint8_t code = geo_s(dr + 1, dc + 2);
            f = code != GEO_FLUID && code != GEO_OUTSIDE;
            pos = dr * DXW + dc;
        }
        list_append(f, (uint16_t)pos, l2, &cnt[1]);
    }
    for (int base = warp * 32; base < L::N3; base += NT) {
        const int k = base + lane;
        bool f = false;
        if (k < L::N3) {
            const int ty = k / TX, tx = k % TX;
            f = x0 + tx < g.nx && y0 + ty < g.ny && geo_s(ty + 3, tx + 4) == GEO_FLUID;
        }
        list_append(f, (uint16_t)k, l3, &cnt[2]);
    }

    const bool bad = !mbar_wait(bar, parity, WAIT_LIMIT_NS);
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicExch(a.err, MCLBM_ERR_TIMEOUT);
        return false;
    }

    // populations of the node at staged row r, column c (geometry row r,
    // column c - HX + 4) with lattice column x and wrapped row y
    auto pull = [&](int r, int c, int x, int y, R f[2][9]) {
        const int gc = c - HX + 4;
        const bool at_in = a.p.open_x && x == 0;
        const bool at_out = a.p.open_x && x == g.nx - 1;
        auto dec = [&](int plane, int comp, int pos) -> R {
            R v = to_real(in[(comp * 9 + plane) * PSTR + pos]);
            if constexpr (P::ref) v += wgt<R>(plane) * to_real(in[(18 + comp) * PSTR + pos]);
            return v;
        };
        const int own = r * RXW + c;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if ((at_in && ex(i) == 1) || (at_out && ex(i) == -1)) {
                f[0][i] = R(0);
                f[1][i] = R(0);
                continue;
            }
            // half-way bounce-back reads the node's own opposite population
            const bool solid_src = i != 0 && geo_s(r - ey(i), gc - ex(i)) != GEO_FLUID;
            const int pos = solid_src ? own : own - ey(i) * RXW - ex(i);
            const int pl = solid_src ? opp(i) : i;
            f[0][i] = dec(pl, 0, pos);
            f[1][i] = dec(pl, 1, pos);
        }
        apply_set3<R>(a, x, y, [&](int comp, int i) { return dec(i, comp, own); }, f);
    };

    // ---- A: densities on the density frame -----------------------------------
    // ring positions (the frame reaches at most 2 rows past an edge, and
    // ny >= 3, so one period of wrap suffices)
    const int n1 = cnt[0];
    for (int k = tid; k < n1; k += NT) {
        const int pos = l1[k];
        const int dr = pos / DXW, dc = pos % DXW;
        R f[2][9];
        pull(dr + 1, dc - 2 + HX, x0 - 2 + dc, wrap(y0 - 2 + dr, g.ny), f);
        R r1 = 0, r2 = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r1 += f[0][i];
            r2 += f[1][i];
        }
        rho[pos] = r1;
        rho[L::N1 + pos] = r2;
    }
    // the tile's own fluid nodes: each thread pulls at most one and keeps its
    // populations in registers for the collision
    const int n3 = cnt[2];
    const bool have = tid < n3;
    int ty = 0, tx = 0;
    R f[2][9];
    R rho1 = 0, rho2 = 0;
    if (have) {
        const int idx = l3[tid];
        ty = idx / TX;
        tx = idx % TX;
        pull(ty + 3, tx + HX, x0 + tx, y0 + ty, f);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            rho1 += f[0][i];
            rho2 += f[1][i];
        }
        rho[(ty + 2) * DXW + tx + 2] = rho1;
        rho[L::N1 + (ty + 2) * DXW + tx + 2] = rho2;
    }
    __syncthreads();

    // ---- B: virtual solid densities on the 1-ring ------------------------------
    const int n2 = cnt[1];
    for (int k = tid; k < n2; k += NT) {
        const int pos = l2[k];
        const int dr = pos / DXW, dc = pos % DXW;
        const uint8_t code = geo_s(dr + 1, dc + 2);
        R n1s = 0, n2s = 0, den = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (geo_s(dr + 1 + ey(i), dc + 2 + ex(i)) == GEO_FLUID) {
                const R w = wgt<R>(i);
                const int q = pos + ey(i) * DXW + ex(i);
                n1s += w * rho[q];
                n2s += w * rho[L::N1 + q];
                den += w;
            }
        }
        R s1 = 0, s2 = 0;
        if (den > R(0)) {
            const R inv = R(1) / den;
            s1 = R(g.chi[2 * code]) * n1s * inv;
            s2 = R(g.chi[2 * code + 1]) * n2s * inv;
        }
        rho[pos] = s1;
        rho[L::N1 + pos] = s2;
    }
    __syncthreads();

    // ---- C: collision of the tile's fluid nodes ---------------------------------
    S *fout = static_cast<S *>(a.fout);
    if (have) {
        const int x = x0 + tx, y = y0 + ty;
        const bool mirror_in = a.p.open_x && x == 0;
        const bool mirror_out = a.p.open_x && x == g.nx - 1;
        const int dpos = (ty + 2) * DXW + tx + 2;
        R fx1, fy1, fx2, fy2;
        node_force<R>(a.p, rho1, rho2,
                      [&](int i, uint8_t &code, R &s1, R &s2) {
                          int dx = ex(i), dy = ey(i);
                          // Sec. 2.1: a neighbour beyond an open end is replaced
                          // by the one in the opposite direction
                          if ((mirror_in && dx < 0) || (mirror_out && dx > 0)) {
                              dx = -dx;
                              dy = -dy;
                          }
                          code = geo_s(ty + 3 + dy, tx + 4 + dx);
                          s1 = rho[dpos + dy * DXW + dx];
                          s2 = rho[L::N1 + dpos + dy * DXW + dx];
                      },
                      fx1, fy1, fx2, fy2);
        R omega, ux, uy;
        node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
        collide_component<R>(f[0], rho1, ux, uy, fx1, fy1, omega);
        collide_component<R>(f[1], rho2, ux, uy, fx2, fy2, omega);
        // output tile, planes of TY x TX in the layout of the store box
        const int o = ty * TX + tx;
        constexpr int OSTR = TX * TY;
        if constexpr (P::ref) {
            const S h1 = from_real<S>(rho1), h2 = from_real<S>(rho2);
            out[18 * OSTR + o] = h1;
            out[19 * OSTR + o] = h2;
            const R q1 = to_real(h1), q2 = to_real(h2);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                out[i * OSTR + o] = from_real<S>(f[0][i] - wgt<R>(i) * q1);
                out[(9 + i) * OSTR + o] = from_real<S>(f[1][i] - wgt<R>(i) * q2);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                out[i * OSTR + o] = from_real<S>(f[0][i]);
                out[(9 + i) * OSTR + o] = from_real<S>(f[1][i]);
            }
        }
        pop_store_ghosts<P>(g, a.p, fout, x, y, f, rho1, rho2);
    }
    // make the generic-proxy writes of the output tile visible to the copy engine
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
        // element (x0, y0) is column hx + x0, row HY + y0; the store map's
        // extent ends at the lattice edge, so ghost columns and rows are kept
        tma_store_3d(tout, g.hx + x0, HY + y0, 0, out);
        bulk_commit();
        bulk_wait_read();
    }
    return true;
}

template <class P, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2)
    tma_tile_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                    const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TileLayout<P, TX, TY>::bar_off);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    tma_tile_body<P, TX, TY>(&tin, &tout, a, blockIdx.x, blockIdx.y, 0, smem);
}

// Many lattices in one persistent launch: CTAs walk a work list of
// (lattice, tile) items; every lattice's arguments and tensor descriptors
// travel in the kernel parameters.
struct BatchArgs {
    int ncases, total;
    int tiles_x[MAX_BATCH];
    int first[MAX_BATCH + 1];  // first work item of each lattice
    StepArgs a[MAX_BATCH];
    CUtensorMap tin[MAX_BATCH];
    CUtensorMap tout[MAX_BATCH];
};

template <class P, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2) tma_batch_kernel(const __grid_constant__ BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TileLayout<P, TX, TY>::bar_off);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    uint32_t parity = 0;
    for (int w = blockIdx.x; w < b.total; w += gridDim.x) {
        int c = 0;
        while (c + 1 < b.ncases && w >= b.first[c + 1]) ++c;
        const int t = w - b.first[c];
        if (!tma_tile_body<P, TX, TY>(&b.tin[c], &b.tout[c], b.a[c], t % b.tiles_x[c],
                                      t / b.tiles_x[c], parity, smem))
            return;
        parity ^= 1u;
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor descriptors and launch.
// ---------------------------------------------------------------------------
static_assert(sizeof(BatchArgs) < 32000, "batch arguments must fit the kernel parameter space");

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

struct TileShape {
    int tx, ty, hx;
};

// shape 0: the default tile of each precision; shape 1: 32 x 8
TileShape shape_of(mclbm_precision p, int shape = 0) {
    const int hx = (p == MCLBM_FP16_DEV || p == MCLBM_BF16_DEV) ? 8 : 4;
    if (p == MCLBM_FP64) return {0, 0, 0};
    if (shape == 1) return {32, 8, hx};
    return {32, p == MCLBM_FP32_DEV ? 12 : 16, hx};
}

CUtensorMapDataType dtype_of(mclbm_precision p) {
    switch (p) {
        case MCLBM_FP16_DEV: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        case MCLBM_BF16_DEV: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    }
}

template <class P, int TX, int TY>
cudaError_t launch_tma_cfg(Lattice &L, const StepArgs &a) {
    using Lay = TileLayout<P, TX, TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(tma_tile_kernel<P, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const CUtensorMap *maps = static_cast<const CUtensorMap *>(L.tmaps);
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY);
    // read through the input map of the current buffer, store through the
    // output map of the other one
    tma_tile_kernel<P, TX, TY><<<grid, TX * TY, Lay::total, L.stream>>>(
        maps[2 * L.cur], maps[2 * (1 - L.cur) + 1], a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool tma_supported(const Lattice &L) { return L.tmaps != nullptr; }

// Input and output descriptors of both population buffers for a tile shape:
// maps[2 b] input of buffer b, maps[2 b + 1] output into buffer b.
int encode_tile_maps(const Lattice &L, int shape, CUtensorMap *maps) {
    const TileShape sh = shape_of(L.prec, shape);
    EncodeTiledFn enc = encode_fn();
    if (sh.tx == 0 || !enc) return fail(MCLBM_ERR_STATE, "TMA descriptors not available");
    const cuuint64_t sb = L.store_bytes;
    for (int b = 0; b < 2; ++b) {
        // input: the whole padded array, box = tile + 3-node ring, all planes
        const cuuint64_t dim_in[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.ny + 2 * HY,
                                      (cuuint64_t)L.planes};
        const cuuint64_t stride[2] = {(cuuint64_t)L.pitch * sb, (cuuint64_t)L.plane * sb};
        const cuuint32_t box_in[3] = {(cuuint32_t)(sh.tx + 2 * sh.hx), (cuuint32_t)(sh.ty + 6),
                                      (cuuint32_t)L.planes};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&maps[2 * b], dtype_of(L.prec), 3, L.f[b], dim_in, stride, box_in, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        // output: extent ends at the lattice edge so the store never writes
        // ghost columns or rows; box = the tile, all planes
        const cuuint64_t dim_out[3] = {(cuuint64_t)(L.hx + L.nx), (cuuint64_t)(HY + L.ny),
                                       (cuuint64_t)L.planes};
        const cuuint32_t box_out[3] = {(cuuint32_t)sh.tx, (cuuint32_t)sh.ty, (cuuint32_t)L.planes};
        CUresult r2 = enc(&maps[2 * b + 1], dtype_of(L.prec), 3, L.f[b], dim_out, stride, box_out,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
            return fail(MCLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" +
                                            std::to_string((int)r) + ", " +
                                            std::to_string((int)r2) + ")");
    }
    return MCLBM_OK;
}

int tma_prepare(Lattice &L) {
    if (shape_of(L.prec).tx == 0 || !encode_fn()) return MCLBM_OK;  // other kernels serve
    CUtensorMap *maps = new (std::nothrow) CUtensorMap[4];
    if (!maps) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    if (int rc = encode_tile_maps(L, 0, maps)) {
        delete[] maps;
        return rc;
    }
    L.tmaps = maps;
    return MCLBM_OK;
}

size_t tile_maps_bytes() { return 4 * sizeof(CUtensorMap); }

int tile_maps_for(const Lattice &L, int shape, void *out) {
    return encode_tile_maps(L, shape, static_cast<CUtensorMap *>(out));
}

template <class P, int TX, int TY>
cudaError_t launch_batch_cfg(Lattice *const *cases, int n, const CUtensorMap *maps, int grid,
                             cudaStream_t stream, int *slots_out) {
    using Lay = TileLayout<P, TX, TY>;
    static int slots = 0;
    if (slots == 0) {
        cudaError_t e = cudaFuncSetAttribute(tma_batch_kernel<P, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_batch_kernel<P, TX, TY>, TX * TY,
                                                      Lay::total);
        slots = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
    }
    if (slots_out) *slots_out = slots;
    if (!cases) return cudaSuccess;  // query only
    static BatchArgs b;  // host staging of the parameter block
    std::memset(&b, 0, sizeof(b));
    b.ncases = n;
    int total = 0;
    for (int c = 0; c < n; ++c) {
        const Lattice &L = *cases[c];
        b.tiles_x[c] = (L.nx + TX - 1) / TX;
        b.first[c] = total;
        total += b.tiles_x[c] * ((L.ny + TY - 1) / TY);
        StepArgs &a = b.a[c];
        a.g = L.geometry();
        a.p = L.p;
        a.fin = L.f[L.cur];
        a.fout = L.f[1 - L.cur];
        a.d5 = L.d5;
        a.err = L.err;
        a.rows_per_cta = 0;
        b.tin[c] = maps[4 * c + 2 * L.cur];
        b.tout[c] = maps[4 * c + 2 * (1 - L.cur) + 1];
    }
    b.first[n] = total;
    b.total = total;
    const int g = grid > 0 ? (grid < total ? grid : total) : (slots < total ? slots : total);
    tma_batch_kernel<P, TX, TY><<<g, TX * TY, Lay::total, stream>>>(b);
    count_launch();
    return cudaGetLastError();
}

void tma_release(Lattice &L) {
    delete[] static_cast<CUtensorMap *>(L.tmaps);
    L.tmaps = nullptr;
}

cudaError_t launch_step_tma(Lattice &L) {
    StepArgs a;
    a.g = L.geometry();
    a.p = L.p;
    a.fin = L.f[L.cur];
    a.fout = L.f[1 - L.cur];
    a.d5 = L.d5;
    a.err = L.err;
    a.rows_per_cta = 0;
    cudaError_t e;
    switch (L.prec) {
        case MCLBM_FP32: e = launch_tma_cfg<P32, 32, 16>(L, a); break;
        case MCLBM_FP32_DEV: e = launch_tma_cfg<P32D, 32, 12>(L, a); break;
        case MCLBM_FP16_DEV: e = launch_tma_cfg<P16D, 32, 16>(L, a); break;
        case MCLBM_BF16_DEV: e = launch_tma_cfg<PB16D, 32, 16>(L, a); break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) L.cur = 1 - L.cur;
    return e;
}

}  // namespace mclbm

namespace mclbm {

int batch_slots(mclbm_precision p, int shape) {
    int slots = 0;
    switch (p) {
        case MCLBM_FP32:
            shape ? launch_batch_cfg<P32, 32, 8>(nullptr, 0, nullptr, 0, 0, &slots)
                  : launch_batch_cfg<P32, 32, 16>(nullptr, 0, nullptr, 0, 0, &slots);
            break;
        case MCLBM_FP32_DEV:
            shape ? launch_batch_cfg<P32D, 32, 8>(nullptr, 0, nullptr, 0, 0, &slots)
                  : launch_batch_cfg<P32D, 32, 12>(nullptr, 0, nullptr, 0, 0, &slots);
            break;
        case MCLBM_FP16_DEV:
            shape ? launch_batch_cfg<P16D, 32, 8>(nullptr, 0, nullptr, 0, 0, &slots)
                  : launch_batch_cfg<P16D, 32, 16>(nullptr, 0, nullptr, 0, 0, &slots);
            break;
        case MCLBM_BF16_DEV:
            shape ? launch_batch_cfg<PB16D, 32, 8>(nullptr, 0, nullptr, 0, 0, &slots)
                  : launch_batch_cfg<PB16D, 32, 16>(nullptr, 0, nullptr, 0, 0, &slots);
            break;
        default: break;
    }
    return slots;
}

// One persistent launch advancing every lattice of a batch by one step
// (all share the precision and are at the same buffer parity).  grid <= 0
// means one CTA per resident slot.
cudaError_t launch_step_batch(Lattice *const *cases, int n, const void *maps, int shape, int grid,
                              cudaStream_t stream) {
    if (n < 1 || n > MAX_BATCH) return cudaErrorInvalidValue;
    const CUtensorMap *m = static_cast<const CUtensorMap *>(maps);
    cudaError_t e;
    const mclbm_precision p = cases[0]->prec;
    switch (p) {
        case MCLBM_FP32:
            e = shape ? launch_batch_cfg<P32, 32, 8>(cases, n, m, grid, stream, nullptr)
                      : launch_batch_cfg<P32, 32, 16>(cases, n, m, grid, stream, nullptr);
            break;
        case MCLBM_FP32_DEV:
            e = shape ? launch_batch_cfg<P32D, 32, 8>(cases, n, m, grid, stream, nullptr)
                      : launch_batch_cfg<P32D, 32, 12>(cases, n, m, grid, stream, nullptr);
            break;
        case MCLBM_FP16_DEV:
            e = shape ? launch_batch_cfg<P16D, 32, 8>(cases, n, m, grid, stream, nullptr)
                      : launch_batch_cfg<P16D, 32, 16>(cases, n, m, grid, stream, nullptr);
            break;
        case MCLBM_BF16_DEV:
            e = shape ? launch_batch_cfg<PB16D, 32, 8>(cases, n, m, grid, stream, nullptr)
                      : launch_batch_cfg<PB16D, 32, 16>(cases, n, m, grid, stream, nullptr);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess)
        for (int c = 0; c < n; ++c) cases[c]->cur = 1 - cases[c]->cur;
    return e;
}

}  // namespace mclbm
