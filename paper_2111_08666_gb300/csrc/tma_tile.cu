// Fused stream-collide-force kernel, 2-D tiles staged by TMA (default for
// the FP32 and deviation storages), in a persistent form that serves one
// lattice or a batch of lattices.
//
// A CTA walks a work list of (lattice, TX x TY tile) items.  For each tile,
// one elected thread copies the tile and its 3-node ring, all direction
// planes at once, into shared memory with a 3-D tensor copy, and the
// geometry codes of the same frame with a 2-D tensor copy; both complete on
// one mbarrier (waits bounded).  The ghost columns and rows of the layouts
// make the ring one rectangular box even at periodic edges.  Then, from
// shared memory:
//   lists   fluid positions of the density frame that need a pull of their
//           own (the 2-ring, periodic images in ragged edge tiles), solid
//           positions of the 1-ring, and the tile's fluid nodes, compacted
//           with warp ballots so that lanes are not spent on solid nodes
//   A       pull + bounce-back + Set-3 and component densities (Eq. 3); each
//           thread keeps the pulled populations of its own tile node
//   (the staged input is no longer read: the next tile's copies are issued)
//   B       improved virtual solid densities (Eqs. 16-17) on the 1-ring
//   C       forces (Eqs. 12-15, boundary mirror), tau_s and u (Eqs. 6-9) and
//           the forced collision (Eqs. 1, 2, 11) into an output tile
// and one tensor copy stores the output tile (whole 32-byte sectors, so no
// partially written sector is fetched first).  Ghost images of edge nodes
// are stored directly.  The store's extent ends at the last whole 16-byte
// chunk of a lattice row: a tensor store clipped inside a chunk was seen to
// write the rest of that chunk, which at a periodic edge is a ghost column
// another CTA fills, so the few columns past that chunk go by plain stores.
#include <cuda.h>

#include <cstring>
#include <new>
#include <type_traits>

#include "async_copy.cuh"
#include "lbm_device.cuh"

namespace mclbm {

namespace {

// geometry frame: columns x0-16 .. x0+TX+15 (a 16-byte aligned box)
constexpr int GO = 16;

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
    static constexpr int GXW = TX + 2 * GO;  // geometry frame width (bytes)
    static constexpr int GYH = TY + 6;
    static constexpr int N1 = DXW * DYH;
    static constexpr int N2 = (DXW - 2) * (DYH - 2);
    static constexpr int N3 = TX * TY;
    static constexpr size_t in_bytes = (size_t)NPL * PSTR * sizeof(S);
    static constexpr size_t out_off = (in_bytes + 127) / 128 * 128;
    static constexpr size_t out_bytes = (size_t)NPL * TY * TX * sizeof(S);
    static constexpr size_t geo_bytes = (size_t)GYH * GXW;
    static constexpr size_t geo_off = (out_off + out_bytes + 127) / 128 * 128;  // two buffers
    static constexpr size_t rho_off = (geo_off + 2 * geo_bytes + 127) / 128 * 128;
    static constexpr size_t rho_bytes = (size_t)2 * N1 * sizeof(R);
    static constexpr size_t l1_off = (rho_off + rho_bytes + 15) / 16 * 16;
    static constexpr size_t l2_off = l1_off + (size_t)N1 * 2;
    static constexpr size_t l3_off = l2_off + (size_t)N2 * 2;
    static constexpr size_t cnt_off = (l3_off + (size_t)N3 * 2 + 15) / 16 * 16;
    static constexpr size_t bar_off = cnt_off + 16;
    static constexpr size_t total = bar_off + 8;
    static constexpr uint32_t tx_bytes = (uint32_t)(in_bytes + geo_bytes);
    static_assert((RXW * sizeof(S)) % 16 == 0, "tensor box rows must be whole 16-byte chunks");
    static_assert((TX * sizeof(S)) % 16 == 0, "store box rows must be whole 16-byte chunks");
    static_assert(GXW % 16 == 0 && geo_bytes % 16 == 0, "geometry box rows must be 16-byte chunks");
    static_assert(HX >= 3, "halo must cover the stencil reach");
};

// Columns [0, store_cols) of a population row go by the tensor store: the
// row up to the last whole 16-byte chunk that ends inside the lattice.
__host__ __device__ constexpr int store_cols(int hx, int nx, int elem_bytes) {
    return (hx + nx) / (16 / elem_bytes) * (16 / elem_bytes);
}

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

// The lattices of a launch; every lattice's arguments and tensor descriptors
// travel in the kernel parameters.
struct BatchArgs {
    int ncases, total;
    int tiles_x[MAX_BATCH];
    int first[MAX_BATCH + 1];  // first work item of each lattice
    StepArgs a[MAX_BATCH];
    CUtensorMap tin[MAX_BATCH];   // input populations (whole padded array)
    CUtensorMap tout[MAX_BATCH];  // output populations (extent ends at the lattice edge)
    CUtensorMap tgeo[MAX_BATCH];  // padded geometry codes
};

__device__ __forceinline__ int case_of(const BatchArgs &b, int w) {
    int c = 0;
    while (c + 1 < b.ncases && w >= b.first[c + 1]) ++c;
    return c;
}

template <class P, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2) tma_tile_kernel(const __grid_constant__ BatchArgs b) {
    using L = TileLayout<P, TX, TY>;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int NT = L::NT, HX = L::HX, RXW = L::RXW, PSTR = L::PSTR, DXW = L::DXW,
                  GXW = L::GXW;

    extern __shared__ __align__(128) unsigned char smem[];
    const S *in = reinterpret_cast<const S *>(smem);
    S *out = reinterpret_cast<S *>(smem + L::out_off);
    R *rho = reinterpret_cast<R *>(smem + L::rho_off);
    uint16_t *l1 = reinterpret_cast<uint16_t *>(smem + L::l1_off);
    uint16_t *l2 = reinterpret_cast<uint16_t *>(smem + L::l2_off);
    uint16_t *l3 = reinterpret_cast<uint16_t *>(smem + L::l3_off);
    int *cnt = reinterpret_cast<int *>(smem + L::cnt_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage tile w: populations into the input buffer, geometry into frame gb
    auto issue = [&](int w, int gb) {
        const int c = case_of(b, w);
        const int t = w - b.first[c];
        const int x0 = (t % b.tiles_x[c]) * TX, y0 = (t / b.tiles_x[c]) * TY;
        fence_proxy_async();
        mbar_expect_tx(bar, L::tx_bytes);
        // element (x0 - HX, y0 - 3) is column x0, row y0 + HY - 3 in memory
        tma_load_3d(smem, &b.tin[c], x0, y0 + HY - 3, 0, bar);
        // geometry (x0 - 16, y0 - 3) is column x0, row y0 + HY - 3 of the padded copy
        tma_load_2d(smem + L::geo_off + gb * L::geo_bytes, &b.tgeo[c], x0, y0 + HY - 3, bar);
    };

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if ((int)blockIdx.x >= b.total) return;
    if (tid == 0) issue(blockIdx.x, 0);

    uint32_t parity = 0;
    int gb = 0;
    for (int w = blockIdx.x; w < b.total; w += gridDim.x) {
        const int c = case_of(b, w);
        const StepArgs &a = b.a[c];
        const Geometry &g = a.g;
        const int t = w - b.first[c];
        const int x0 = (t % b.tiles_x[c]) * TX, y0 = (t / b.tiles_x[c]) * TY;
        const uint8_t *geo = smem + L::geo_off + gb * L::geo_bytes;
        auto geo_s = [&](int r, int col) -> uint8_t { return geo[r * GXW + col]; };

        if (tid == 0) cnt[0] = cnt[1] = cnt[2] = 0;
        const bool bad = !mbar_wait(bar, parity, WAIT_LIMIT_NS);
        if (__syncthreads_or(bad)) {
            if (tid == 0) {
                atomicExch(a.err, MCLBM_ERR_TIMEOUT);
                // give the outstanding copy a last, short chance to land
                mbar_wait(bar, parity, DRAIN_LIMIT_NS);
                bulk_wait_read();
            }
            return;
        }

        // ---- work lists (geometry only) --------------------------------------
        for (int base = warp * 32; base < L::N1; base += NT) {
            const int k = base + lane;
            bool f = false;
            if (k < L::N1) {
                const int dr = k / DXW, dc = k % DXW;
                const bool own = dr >= 2 && dr < TY + 2 && dc >= 2 && dc < TX + 2 &&
                                 x0 - 2 + dc < g.nx && y0 - 2 + dr < g.ny;
                const bool fl = geo_s(dr + 1, dc - 2 + GO) == GEO_FLUID;
                if (!fl || own) {
                    rho[k] = R(0);
                    rho[L::N1 + k] = R(0);
                }
                // the 2-ring, and in a ragged edge tile the positions past the
                // lattice edge (periodic images the edge nodes need)
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
                const uint8_t code = geo_s(dr + 1, dc - 2 + GO);
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
                f = x0 + tx < g.nx && y0 + ty < g.ny && geo_s(ty + 3, tx + GO) == GEO_FLUID;
            }
            list_append(f, (uint16_t)k, l3, &cnt[2]);
        }
        __syncthreads();

        // populations of the node at staged row r, column c with lattice
        // column x and wrapped row y (geometry frame row r, column c - HX + GO)
        auto pull = [&](int r, int c, int x, int y, R f[2][9]) {
            const int gc = c - HX + GO;
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

        // ---- A: densities on the density frame -------------------------------
        // (the frame reaches at most 2 rows past an edge and ny >= 3, so one
        // period of wrap suffices)
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
        // the tile's own fluid nodes: each thread pulls at most one and keeps
        // its populations in registers for the collision
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
        // the staged input has been read: bring in the next tile meanwhile
        if (tid == 0 && w + (int)gridDim.x < b.total) issue(w + gridDim.x, gb ^ 1);

        // ---- B: virtual solid densities on the 1-ring ----------------------------
        const int n2 = cnt[1];
        for (int k = tid; k < n2; k += NT) {
            const int pos = l2[k];
            const int dr = pos / DXW, dc = pos % DXW;
            const uint8_t code = geo_s(dr + 1, dc - 2 + GO);
            R n1s = 0, n2s = 0, den = 0;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if (geo_s(dr + 1 + ey(i), dc - 2 + GO + ex(i)) == GEO_FLUID) {
                    const R w8 = wgt<R>(i);
                    const int q = pos + ey(i) * DXW + ex(i);
                    n1s += w8 * rho[q];
                    n2s += w8 * rho[L::N1 + q];
                    den += w8;
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
        // the previous tile's output copy must have read the output buffer
        if (tid == 0) bulk_wait_read();
        __syncthreads();

        // ---- C: collision of the tile's fluid nodes --------------------------------
        if (have) {
            const int x = x0 + tx, y = y0 + ty;
            const bool mirror_in = a.p.open_x && x == 0;
            const bool mirror_out = a.p.open_x && x == g.nx - 1;
            const int dpos = (ty + 2) * DXW + tx + 2;
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
                              code = geo_s(ty + 3 + dy, tx + GO + dx);
                              s1 = rho[dpos + dy * DXW + dx];
                              s2 = rho[L::N1 + dpos + dy * DXW + dx];
                          },
                          fx1, fy1, fx2, fy2);
            R omega, ux, uy;
            node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
            collide_component<R>(f[0], rho1, ux, uy, fx1, fy1, omega);
            collide_component<R>(f[1], rho2, ux, uy, fx2, fy2, omega);
            // output tile: planes of TY x TX in the layout of the store box
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
            if (g.hx + x >= store_cols(g.hx, g.nx, sizeof(S)))
                pop_store_site<P>(static_cast<S *>(a.fout), g.plane, site_of(g, x, y), f, rho1, rho2);
            pop_store_ghosts<P>(g, a.p, static_cast<S *>(a.fout), x, y, f, rho1, rho2);
        }
        // make the generic-proxy writes of the output tile visible to the copy engine
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && g.hx + x0 < store_cols(g.hx, g.nx, sizeof(S))) {
            // element (x0, y0) is column hx + x0, row HY + y0; the store map's
            // extent ends inside the lattice, so ghost columns and rows are kept
            tma_store_3d(&b.tout[c], g.hx + x0, HY + y0, 0, out);
            bulk_commit();
        }
        parity ^= 1u;
        gb ^= 1;
    }
    if (tid == 0) bulk_wait_read();
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

// descriptors of one lattice for one tile shape:
// [0] input of buffer 0, [1] output into buffer 0, [2] input of buffer 1,
// [3] output into buffer 1, [4] padded geometry
constexpr int MAPS_PER_CASE = 5;

template <class P, int TX, int TY>
cudaError_t launch_cfg(Lattice *const *cases, int n, const CUtensorMap *maps, int grid,
                       cudaStream_t stream, int *slots_out) {
    using Lay = TileLayout<P, TX, TY>;
    static int slots = 0;
    if (slots == 0) {
        cudaError_t e = cudaFuncSetAttribute(tma_tile_kernel<P, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_tile_kernel<P, TX, TY>, TX * TY,
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
        const CUtensorMap *m = maps + MAPS_PER_CASE * c;
        b.tin[c] = m[2 * L.cur];               // read the current buffer
        b.tout[c] = m[2 * (1 - L.cur) + 1];    // store into the other one
        b.tgeo[c] = m[4];
    }
    b.first[n] = total;
    b.total = total;
    const int g = grid > 0 ? (grid < total ? grid : total) : (slots < total ? slots : total);
    tma_tile_kernel<P, TX, TY><<<g, TX * TY, Lay::total, stream>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_prec(Lattice *const *cases, int n, const CUtensorMap *maps, int shape,
                        int grid, cudaStream_t stream, int *slots) {
    constexpr bool dev32 = std::is_same<P, P32D>::value;
    if (shape == 1) return launch_cfg<P, 32, 8>(cases, n, maps, grid, stream, slots);
    return launch_cfg<P, 32, dev32 ? 12 : 16>(cases, n, maps, grid, stream, slots);
}

cudaError_t launch_any(mclbm_precision p, Lattice *const *cases, int n, const CUtensorMap *maps,
                       int shape, int grid, cudaStream_t stream, int *slots) {
    switch (p) {
        case MCLBM_FP32: return launch_prec<P32>(cases, n, maps, shape, grid, stream, slots);
        case MCLBM_FP32_DEV: return launch_prec<P32D>(cases, n, maps, shape, grid, stream, slots);
        case MCLBM_FP16_DEV: return launch_prec<P16D>(cases, n, maps, shape, grid, stream, slots);
        case MCLBM_BF16_DEV: return launch_prec<PB16D>(cases, n, maps, shape, grid, stream, slots);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Descriptors of one lattice for a tile shape (MAPS_PER_CASE of them).
int encode_tile_maps(const Lattice &L, int shape, void *out) {
    CUtensorMap *maps = static_cast<CUtensorMap *>(out);
    const TileShape sh = shape_of(L.prec, shape);
    EncodeTiledFn enc = encode_fn();
    if (sh.tx == 0 || !enc || !L.geo_pad)
        return fail(MCLBM_ERR_STATE, "TMA descriptors not available");
    const cuuint64_t sb = L.store_bytes;
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int b = 0; b < 2; ++b) {
        // input: the whole padded array, box = tile + 3-node ring, all planes
        const cuuint64_t dim_in[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.ny + 2 * HY,
                                      (cuuint64_t)L.planes};
        const cuuint64_t stride[2] = {(cuuint64_t)L.pitch * sb, (cuuint64_t)L.plane * sb};
        const cuuint32_t box_in[3] = {(cuuint32_t)(sh.tx + 2 * sh.hx), (cuuint32_t)(sh.ty + 6),
                                      (cuuint32_t)L.planes};
        CUresult r = enc(&maps[2 * b], dtype_of(L.prec), 3, L.f[b], dim_in, stride, box_in, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        // output: extent ends inside the lattice (at a 16-byte chunk) so the
        // store never writes ghost columns or rows; box = the tile, all planes
        const cuuint64_t dim_out[3] = {(cuuint64_t)store_cols(L.hx, L.nx, (int)sb),
                                       (cuuint64_t)(HY + L.ny), (cuuint64_t)L.planes};
        const cuuint32_t box_out[3] = {(cuuint32_t)sh.tx, (cuuint32_t)sh.ty, (cuuint32_t)L.planes};
        CUresult r2 = enc(&maps[2 * b + 1], dtype_of(L.prec), 3, L.f[b], dim_out, stride, box_out,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
            return fail(MCLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" +
                                            std::to_string((int)r) + ", " +
                                            std::to_string((int)r2) + ")");
    }
    // geometry: the padded byte array, box = the tile's geometry frame
    const cuuint64_t gdim[2] = {(cuuint64_t)L.gpitch, (cuuint64_t)L.geo_pad_rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)L.gpitch};
    const cuuint32_t gbox[2] = {(cuuint32_t)(sh.tx + 2 * GO), (cuuint32_t)(sh.ty + 6)};
    CUresult r = enc(&maps[4], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, L.geo_pad, gdim, gstride, gbox,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(MCLBM_ERR_CUDA, "cuTensorMapEncodeTiled (geometry) failed (" +
                                        std::to_string((int)r) + ")");
    return MCLBM_OK;
}

bool tma_supported(const Lattice &L) { return L.tmaps != nullptr; }

int tma_prepare(Lattice &L) {
    if (shape_of(L.prec).tx == 0 || !encode_fn() || !L.geo_pad) return MCLBM_OK;  // other kernels serve
    CUtensorMap *maps = new (std::nothrow) CUtensorMap[MAPS_PER_CASE];
    if (!maps) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    if (int rc = encode_tile_maps(L, 0, maps)) {
        delete[] maps;
        return rc;
    }
    L.tmaps = maps;
    return MCLBM_OK;
}

void tma_release(Lattice &L) {
    delete[] static_cast<CUtensorMap *>(L.tmaps);
    L.tmaps = nullptr;
}

size_t tile_maps_bytes() { return MAPS_PER_CASE * sizeof(CUtensorMap); }

int tile_maps_for(const Lattice &L, int shape, void *out) { return encode_tile_maps(L, shape, out); }

int batch_slots(mclbm_precision p, int shape) {
    int slots = 0;
    launch_any(p, nullptr, 0, nullptr, shape, 0, 0, &slots);
    return slots;
}

// One persistent launch advancing every lattice given by one step (all
// share the precision and are at the same buffer parity).  grid <= 0 means
// one CTA per resident slot.
cudaError_t launch_step_batch(Lattice *const *cases, int n, const void *maps, int shape, int grid,
                              cudaStream_t stream) {
    if (n < 1 || n > MAX_BATCH) return cudaErrorInvalidValue;
    cudaError_t e = launch_any(cases[0]->prec, cases, n, static_cast<const CUtensorMap *>(maps),
                               shape, grid, stream, nullptr);
    if (e == cudaSuccess)
        for (int c = 0; c < n; ++c) cases[c]->cur = 1 - cases[c]->cur;
    return e;
}

cudaError_t launch_step_tma(Lattice &L) {
    Lattice *one = &L;
    return launch_step_batch(&one, 1, L.tmaps, 0, 0, L.stream);
}

}  // namespace mclbm
