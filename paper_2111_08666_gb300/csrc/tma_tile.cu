// Fused stream-collide-force kernel, 2-D tiles staged by TMA (default for
// the FP32 and deviation storages), in a persistent form that serves one
// lattice or a batch of lattices.
//
// A CTA walks a work list of (lattice, TX x TY tile) items.  For each tile,
// one elected thread copies the tile and its 3-node ring, all direction
// planes at once, into shared memory with a 3-D tensor copy, and the tile's
// work table with a bulk copy; both complete on one mbarrier (waits
// bounded).  The ghost columns and rows of the layouts make the ring one
// rectangular box even at periodic edges.
//
// The work table of a tile is built once per geometry and boundary mode
// (build_tables_kernel) and lists, as packed 32-bit entries: the tile's
// fluid nodes, the other fluid nodes of the density frame (tile + 2-node
// ring: the 2-ring, and periodic images in ragged edge tiles), and the
// non-fluid nodes of the 1-ring, each with the fluid/solid pattern of its 8
// neighbours.  So the step needs no geometry of its own and no branches on
// it.  From shared memory:
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

// Columns [0, store_cols) of a population row go by the tensor store: the
// row up to the last whole 16-byte chunk that ends inside the lattice.
__host__ __device__ constexpr int store_cols(int hx, int nx, int elem_bytes) {
    return (hx + nx) / (16 / elem_bytes) * (16 / elem_bytes);
}

namespace {

// ---------------------------------------------------------------------------
// Work tables.  Per tile: a 4-word header (n_own, n_ring, n_solid, 0), then
// n_own + n_ring + n_solid entries:
//   fluid node of the tile   tx | ty << 6 | nonfluid << 12 | set3 << 20
//   ring pull                pos | nonfluid << 12 | set3 << 20
//   ring non-fluid node      pos | code << 12 | fluid << 20
// pos = row * (TX + 4) + column in the density frame, whose origin is the
// node (x0 - 2, y0 - 2).  Bit i-1 of nonfluid (fluid) is set when the
// neighbour x + e_i is not fluid (is fluid).  set3 bit 0: x = 0 of a lattice
// with open ends, bit 1: x = nx - 1 of one.  Every frame position holds at
// most one entry, so a table never exceeds 4 + frame words.
// ---------------------------------------------------------------------------
constexpr uint32_t SET3_BITS = 3u << 20;
constexpr uint32_t AT_IN = 1u << 20, AT_OUT = 2u << 20;

template <int TX, int TY>
struct TableShape {
    static constexpr int DXW = TX + 4, DYH = TY + 4, N1 = DXW * DYH;
    static constexpr int words = (4 + N1 + 3) / 4 * 4;  // stride of one tile's table
    static_assert(N1 <= 4096 && TX <= 64 && TY <= 64, "entry fields too narrow");
};

int table_words(int tx, int ty) { return (4 + (tx + 4) * (ty + 4) + 3) / 4 * 4; }

// One warp per tile; entries appended in frame order (deterministic).
template <int TX, int TY>
__global__ void build_tables_kernel(Geometry g, const uint8_t *pad, int pad_rows, int open_x,
                                    int tiles_x, int ntiles, uint32_t *tab, int *max_words) {
    using TS = TableShape<TX, TY>;
    constexpr int DXW = TS::DXW, N1 = TS::N1;
    const int tile = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;  // whole warps leave together
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    // geometry code of lattice position (x, y) as the step sees it: pad row
    // y + HY, column GEO_HX + x (ghosts per the boundary mode); outside beyond
    auto code_at = [&](int x, int y) -> int {
        const int r = y + HY, col = GEO_HX + x;
        if (r < 0 || r >= pad_rows || col < 0 || col >= g.gpitch) return GEO_OUTSIDE;
        return pad[(long long)r * g.gpitch + col];
    };
    auto fluid_mask = [&](int x, int y) {
        uint32_t m = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if (code_at(x + ex(i), y + ey(i)) == GEO_FLUID) m |= 1u << (i - 1);
        return m;
    };
    auto set3 = [&](int x) -> uint32_t {
        return (open_x && x == 0 ? AT_IN : 0u) | (open_x && x == g.nx - 1 ? AT_OUT : 0u);
    };
    uint32_t *T = tab + (size_t)tile * TS::words;
    int n = 0;
    auto append = [&](bool flag, uint32_t e) {
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (flag) T[4 + n + __popc(m & ((1u << lane) - 1u))] = e;
        n += __popc(m);
    };
    for (int base = 0; base < TX * TY; base += 32) {
        const int k = base + lane;
        const int tx = k % TX, ty = k / TX, x = x0 + tx, y = y0 + ty;
        const bool f = k < TX * TY && x < g.nx && y < g.ny && code_at(x, y) == GEO_FLUID;
        append(f, f ? (uint32_t)tx | (uint32_t)ty << 6 | (~fluid_mask(x, y) & 0xffu) << 12 | set3(x)
                    : 0u);
    }
    const int n_own = n;
    for (int base = 0; base < N1; base += 32) {
        const int k = base + lane;
        const int dr = k / DXW, dc = k % DXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
        const bool own = dr >= 2 && dr < TY + 2 && dc >= 2 && dc < TX + 2 && x < g.nx && y < g.ny;
        const bool f = k < N1 && !own && code_at(x, y) == GEO_FLUID;
        append(f, f ? (uint32_t)k | (~fluid_mask(x, y) & 0xffu) << 12 | set3(x) : 0u);
    }
    const int n_ring = n - n_own;
    for (int base = 0; base < N1; base += 32) {
        const int k = base + lane;
        const int dr = k / DXW, dc = k % DXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
        const bool ring1 = dr >= 1 && dr <= TY + 2 && dc >= 1 && dc <= TX + 2;
        const int c = k < N1 && ring1 ? code_at(x, y) : GEO_FLUID;
        const bool f = c != GEO_FLUID;
        append(f, f ? (uint32_t)k | (uint32_t)c << 12 | fluid_mask(x, y) << 20 : 0u);
    }
    if (lane == 0) {
        T[0] = (uint32_t)n_own;
        T[1] = (uint32_t)n_ring;
        T[2] = (uint32_t)(n - n_own - n_ring);
        T[3] = 0;
        atomicMax(max_words, 4 + n);
    }
}

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
    static constexpr int DXW = TableShape<TX, TY>::DXW;  // density frame: tile + 2
    static constexpr int N1 = TableShape<TX, TY>::N1;
    static constexpr int TW = TableShape<TX, TY>::words;
    static constexpr size_t in_bytes = (size_t)NPL * PSTR * sizeof(S);
    static constexpr size_t out_off = (in_bytes + 127) / 128 * 128;
    static constexpr size_t out_bytes = (size_t)NPL * TY * TX * sizeof(S);
    static constexpr size_t rho_off = (out_off + out_bytes + 127) / 128 * 128;
    static constexpr size_t rho_bytes = (size_t)2 * N1 * sizeof(R);
    static constexpr size_t tab_off = (rho_off + rho_bytes + 127) / 128 * 128;  // two buffers
    static constexpr size_t tab_bytes = (size_t)2 * TW * 4;
    static constexpr size_t bar_off = tab_off + tab_bytes;
    static constexpr size_t total = bar_off + 8;
    static_assert((RXW * sizeof(S)) % 16 == 0, "tensor box rows must be whole 16-byte chunks");
    static_assert((TX * sizeof(S)) % 16 == 0, "store box rows must be whole 16-byte chunks");
    static_assert((TW * 4) % 16 == 0, "table copies must be whole 16-byte chunks");
    static_assert(HX >= 3, "halo must cover the stencil reach");
};

// The lattices of a launch; every lattice's arguments and tensor descriptors
// travel in the kernel parameters.  Sized by the number of lattices a launch
// may hold (1 or MAX_BATCH): the parameter block is copied at every launch,
// and a single lattice's launch stays small.
template <int N>
struct BatchArgs {
    CUtensorMap tin[N];   // input populations (whole padded array)
    CUtensorMap tout[N];  // output populations (extent ends inside the lattice)
    StepArgs a[N];
    const uint32_t *tab[N];
    int ncases, total;
    int tiles_x[N];
    int first[N + 1];     // first work item of each lattice
    int tab_words[N];     // table words copied per tile
};

// N = 1: the launch holds a single lattice (its arguments at fixed offsets)
template <class P, int TX, int TY, int N>
__global__ void __launch_bounds__(TX *TY, 2) tma_tile_kernel(const __grid_constant__ BatchArgs<N> b) {
    constexpr bool ONE = N == 1;
    using L = TileLayout<P, TX, TY>;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int NT = L::NT, HX = L::HX, RXW = L::RXW, PSTR = L::PSTR, DXW = L::DXW,
                  N1 = L::N1, TW = L::TW;

    extern __shared__ __align__(128) unsigned char smem[];
    const S *in = reinterpret_cast<const S *>(smem);
    S *out = reinterpret_cast<S *>(smem + L::out_off);
    R *rho = reinterpret_cast<R *>(smem + L::rho_off);
    uint32_t *tabs = reinterpret_cast<uint32_t *>(smem + L::tab_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);
    const int tid = threadIdx.x;

    auto case_of = [&](int w) -> int {
        if constexpr (ONE) {
            return 0;
        } else {
            int c = 0;
            while (c + 1 < b.ncases && w >= b.first[c + 1]) ++c;
            return c;
        }
    };

    // stage tile w: populations into the input buffer, work table into buffer tb
    auto issue = [&](int w, int tb) {
        const int c = case_of(w);
        const int t = w - b.first[c];
        const int x0 = (t % b.tiles_x[c]) * TX, y0 = (t / b.tiles_x[c]) * TY;
        const uint32_t tbytes = 4u * (uint32_t)b.tab_words[c];
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)L::in_bytes + tbytes);
        // element (x0 - HX, y0 - 3) is column x0, row y0 + HY - 3 in memory
        tma_load_3d(smem, &b.tin[c], x0, y0 + HY - 3, 0, bar);
        bulk_g2s(tabs + tb * TW, b.tab[c] + (size_t)t * TW, tbytes, bar);
    };

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if ((int)blockIdx.x >= b.total) return;
    if (tid == 0) issue(blockIdx.x, 0);

    uint32_t parity = 0;
    int tb = 0;
    for (int w = blockIdx.x; w < b.total; w += gridDim.x) {
        const int c = case_of(w);
        const StepArgs &a = b.a[c];
        const Geometry &g = a.g;
        const int t = w - b.first[c];
        const int x0 = (t % b.tiles_x[c]) * TX, y0 = (t / b.tiles_x[c]) * TY;

        const bool bad = !mbar_wait(bar, parity, a.wait_ns);
        if (__syncthreads_or(bad)) {
            if (tid == 0) {
                atomicExch(a.err, MCLBM_ERR_TIMEOUT);
                // give the outstanding copy a last, short chance to land
                mbar_wait(bar, parity, DRAIN_LIMIT_NS);
                bulk_wait_read();
            }
            return;
        }
        const uint32_t *T = tabs + tb * TW;
        const int n_own = (int)T[0], n_ring = (int)T[1], n_sol = (int)T[2];
        const uint32_t *E = T + 4;

        // population (plane, comp) of the staged node pos, w = its weight
        auto dec = [&](int plane, int comp, int pos, R w) -> R {
            R v = to_real(in[(comp * 9 + plane) * PSTR + pos]);
            if constexpr (P::ref) v += w * to_real(in[(18 + comp) * PSTR + pos]);
            return v;
        };
        // f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) where x - e_i is not fluid
        // (half-way bounce-back), then the open-end treatment (Sec. 2.3); the node sits at
        // staged row r, column cc, lattice column x and wrapped row y.  Where a
        // source lies beyond an open end the bounce-back value is a placeholder
        // that Set-3 replaces.
        auto pull = [&](int r, int cc, uint32_t e, int x, int y, R f[2][9]) {
            const uint32_t m = (e >> 12) & 0xffu;
            const int own = r * RXW + cc;
            f[0][0] = dec(0, 0, own, wgt<R>(0));
            f[1][0] = dec(0, 1, own, wgt<R>(0));
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const bool sb = (m >> (opp(i) - 1)) & 1u;
                const int pos = sb ? own : own - ey(i) * RXW - ex(i);
                const int pl = sb ? opp(i) : i;
                f[0][i] = dec(pl, 0, pos, wgt<R>(i));
                f[1][i] = dec(pl, 1, pos, wgt<R>(i));
            }
            if (e & SET3_BITS)
                apply_open_bc<R>(a, x, y, [&](int comp, int i) { return dec(i, comp, own, wgt<R>(i)); },
                              f);
        };

        // ---- A: densities of the ring's fluid nodes and of the tile's own ------
        // Thread t pulls tile node t (t < n_own); ring entries go first to the
        // threads without a tile node (entry j to thread n_own + j mod NT), so
        // that most threads pull once.
        for (int k = tid - n_own + (tid < n_own ? NT : 0); k < n_ring; k += NT) {
            const uint32_t e = E[n_own + k];
            const int pos = (int)(e & 0xfffu);
            const int dr = pos / DXW, dc = pos - dr * DXW;
            R f[2][9];
            pull(dr + 1, dc - 2 + HX, e, x0 - 2 + dc, wrap(y0 - 2 + dr, g.ny), f);
            R r1 = 0, r2 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                r1 += f[0][i];
                r2 += f[1][i];
            }
            rho[pos] = r1;
            rho[N1 + pos] = r2;
        }
        // each thread pulls at most one tile node and keeps its populations
        // in registers for the collision
        const bool have = tid < n_own;
        const uint32_t me = have ? E[tid] : 0u;
        const int tx = (int)(me & 63u), ty = (int)((me >> 6) & 63u);
        R f[2][9];
        R rho1 = 0, rho2 = 0;
        if (have) {
            pull(ty + 3, tx + HX, me, x0 + tx, y0 + ty, f);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                rho1 += f[0][i];
                rho2 += f[1][i];
            }
            rho[(ty + 2) * DXW + tx + 2] = rho1;
            rho[N1 + (ty + 2) * DXW + tx + 2] = rho2;
        }
        __syncthreads();
        // the staged input has been read: bring in the next tile meanwhile
        if (tid == 0 && w + (int)gridDim.x < b.total) issue(w + gridDim.x, tb ^ 1);

        // ---- B: virtual solid densities on the 1-ring (zero outside) -----------
        const uint32_t *Es = E + n_own + n_ring;
        for (int k = tid; k < n_sol; k += NT) {
            const uint32_t e = Es[k];
            const int pos = (int)(e & 0xfffu);
            const int code = (int)((e >> 12) & 0xffu);
            const uint32_t fm = e >> 20;
            R n1s = 0, n2s = 0, den = 0;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if ((fm >> (i - 1)) & 1u) {
                    const R w8 = wgt<R>(i);
                    const int q = pos + ey(i) * DXW + ex(i);
                    n1s += w8 * rho[q];
                    n2s += w8 * rho[N1 + q];
                    den += w8;
                }
            }
            R s1 = 0, s2 = 0;
            if (den > R(0) && code != GEO_OUTSIDE) {
                const R inv = R(1) / den;
                s1 = chi_at<R>(g, 2 * code) * n1s * inv;
                s2 = chi_at<R>(g, 2 * code + 1) * n2s * inv;
            }
            rho[pos] = s1;
            rho[N1 + pos] = s2;
        }
        // the previous tile's output copy must have read the output buffer
        if (tid == 0) bulk_wait_read();
        __syncthreads();

        // ---- C: collision of the tile's fluid nodes --------------------------------
        if (have) {
            const int x = x0 + tx, y = y0 + ty;
            const int dpos = (ty + 2) * DXW + tx + 2;
            const uint32_t m = (me >> 12) & 0xffu;
            R fx1, fy1, fx2, fy2;
            if (me & SET3_BITS) {
                // Sec. 2.1: a neighbour beyond an open end is replaced by the
                // one in the opposite direction
                const bool mir_in = me & AT_IN, mir_out = me & AT_OUT;
                node_force<R, false>(a.p, rho1, rho2,
                                     [&](int i, uint8_t &code, R &s1, R &s2) {
                                         const bool mir = (mir_in && ex(i) < 0) || (mir_out && ex(i) > 0);
                                         const int d = ey(i) * DXW + ex(i);
                                         const int q = mir ? dpos - d : dpos + d;
                                         const uint32_t bit = mir ? (m >> (opp(i) - 1)) : (m >> (i - 1));
                                         code = (bit & 1u) ? 1 : GEO_FLUID;
                                         s1 = rho[q];
                                         s2 = rho[N1 + q];
                                     },
                                     fx1, fy1, fx2, fy2);
            } else {
                node_force<R, false>(a.p, rho1, rho2,
                                     [&](int i, uint8_t &code, R &s1, R &s2) {
                                         const int q = dpos + ey(i) * DXW + ex(i);
                                         code = ((m >> (i - 1)) & 1u) ? 1 : GEO_FLUID;
                                         s1 = rho[q];
                                         s2 = rho[N1 + q];
                                     },
                                     fx1, fy1, fx2, fy2);
            }
            R omega, ux, uy;
            node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
            collide<R>(a.p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
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
        tb ^= 1;
    }
    if (tid == 0) bulk_wait_read();
}

// ---------------------------------------------------------------------------
// Host side: tensor descriptors, work tables and launch.
// ---------------------------------------------------------------------------
static_assert(sizeof(BatchArgs<MAX_BATCH>) < 32000, "batch arguments must fit the kernel parameter space");

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

int tiles_of(const Lattice &L, const TileShape &sh) {
    return ((L.nx + sh.tx - 1) / sh.tx) * ((L.ny + sh.ty - 1) / sh.ty);
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
// [3] output into buffer 1
constexpr int MAPS_PER_CASE = 4;

template <class P, int TX, int TY, int N>
int resident_slots() {
    using Lay = TileLayout<P, TX, TY>;
    static int slots = 0;
    if (slots == 0) {
        if (cudaFuncSetAttribute(tma_tile_kernel<P, TX, TY, N>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Lay::total) != cudaSuccess)
            return 0;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_tile_kernel<P, TX, TY, N>,
                                                      TX * TY, Lay::total);
        slots = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
    }
    return slots;
}

// fill the parameter block of n lattices and launch
template <class P, int TX, int TY, int N>
cudaError_t launch_args(Lattice *const *cases, int n, const CUtensorMap *maps, int shape, int grid,
                        int slots, cudaStream_t stream) {
    using Lay = TileLayout<P, TX, TY>;
    static BatchArgs<N> b;  // host staging of the parameter block
    std::memset(&b, 0, sizeof(b));
    b.ncases = n;
    int total = 0;
    for (int c = 0; c < n; ++c) {
        const Lattice &L = *cases[c];
        if (!L.tab[shape] || L.tab_words[shape] < 4) return cudaErrorInvalidValue;
        b.tiles_x[c] = (L.nx + TX - 1) / TX;
        b.first[c] = total;
        total += b.tiles_x[c] * ((L.ny + TY - 1) / TY);
        b.tab[c] = L.tab[shape];
        b.tab_words[c] = L.tab_words[shape];
        StepArgs &a = b.a[c];
        a.g = L.geometry();
        a.p = L.p;
        a.p.round_fp32();
        a.fin = L.f[L.cur];
        a.fout = L.f[1 - L.cur];
        a.d5 = L.d5;
        a.err = L.err;
        a.wait_ns = L.wait_ns;
        a.rows_per_cta = 0;
        const CUtensorMap *m = maps + MAPS_PER_CASE * c;
        b.tin[c] = m[2 * L.cur];               // read the current buffer
        b.tout[c] = m[2 * (1 - L.cur) + 1];    // store into the other one
    }
    b.first[n] = total;
    b.total = total;
    const int g = grid > 0 ? (grid < total ? grid : total) : (slots < total ? slots : total);
    tma_tile_kernel<P, TX, TY, N><<<g, TX * TY, Lay::total, stream>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <class P, int TX, int TY>
cudaError_t launch_cfg(Lattice *const *cases, int n, const CUtensorMap *maps, int shape, int grid,
                       cudaStream_t stream, int *slots_out) {
    const bool one = n == 1;
    const int slots = one ? resident_slots<P, TX, TY, 1>() : resident_slots<P, TX, TY, MAX_BATCH>();
    if (slots == 0) {
        const cudaError_t e = cudaGetLastError();
        return e != cudaSuccess ? e : cudaErrorUnknown;
    }
    if (slots_out) *slots_out = slots;
    if (!cases) return cudaSuccess;  // query only
    if (one) return launch_args<P, TX, TY, 1>(cases, n, maps, shape, grid, slots, stream);
    return launch_args<P, TX, TY, MAX_BATCH>(cases, n, maps, shape, grid, slots, stream);
}

template <class P>
cudaError_t launch_prec(Lattice *const *cases, int n, const CUtensorMap *maps, int shape,
                        int grid, cudaStream_t stream, int *slots) {
    constexpr bool dev32 = std::is_same<P, P32D>::value;
    if (shape == 1) return launch_cfg<P, 32, 8>(cases, n, maps, shape, grid, stream, slots);
    return launch_cfg<P, 32, dev32 ? 12 : 16>(cases, n, maps, shape, grid, stream, slots);
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

template <int TX, int TY>
cudaError_t launch_build(const Lattice &L, int shape) {
    const int tiles_x = (L.nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((L.ny + TY - 1) / TY);
    const int blocks = (ntiles + 3) / 4;  // four warps (tiles) per block
    build_tables_kernel<TX, TY><<<blocks, 128, 0, L.stream>>>(
        L.geometry(), L.geo_pad, L.geo_pad_rows, L.p.open_x, tiles_x, ntiles, L.tab[shape],
        L.tab_max + shape);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

// Descriptors of one lattice for a tile shape (MAPS_PER_CASE of them).
int encode_tile_maps(const Lattice &L, int shape, void *out) {
    CUtensorMap *maps = static_cast<CUtensorMap *>(out);
    const TileShape sh = shape_of(L.prec, shape);
    EncodeTiledFn enc = encode_fn();
    if (sh.tx == 0 || !enc) return fail(MCLBM_ERR_STATE, "TMA descriptors not available");
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
    return MCLBM_OK;
}

bool tma_supported(const Lattice &L) { return L.tmaps != nullptr; }

int tma_prepare(Lattice &L) {
    if (shape_of(L.prec).tx == 0 || !encode_fn() || !L.geo_pad) return MCLBM_OK;  // other kernels serve
    for (int s = 0; s < 2; ++s) {
        const TileShape sh = shape_of(L.prec, s);
        const size_t bytes = (size_t)tiles_of(L, sh) * table_words(sh.tx, sh.ty) * 4;
        if (cudaMalloc((void **)&L.tab[s], bytes) != cudaSuccess ||
            cudaMemsetAsync(L.tab[s], 0, bytes, L.stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(MCLBM_ERR_NOMEM, "device allocation of the work tables failed");
        }
        L.device_bytes += bytes;
    }
    if (cudaMalloc((void **)&L.tab_max, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCLBM_ERR_NOMEM, "device allocation failed");
    }
    CUtensorMap *maps = new (std::nothrow) CUtensorMap[2 * MAPS_PER_CASE];
    if (!maps) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    for (int s = 0; s < 2; ++s)
        if (int rc = encode_tile_maps(L, s, maps + s * MAPS_PER_CASE)) {
            delete[] maps;
            return rc;
        }
    L.tmaps = maps;
    return MCLBM_OK;
}

// (Re)build the work tables of both tile shapes for the current geometry
// ghosts and boundary mode, and read back the largest table of each.
int tma_build_tables(Lattice &L) {
    if (!L.tab[0] || !L.tab[1] || !L.tab_max) return MCLBM_OK;
    cudaError_t e = cudaMemsetAsync(L.tab_max, 0, 2 * sizeof(int), L.stream);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
        const TileShape sh = shape_of(L.prec, s);
        if (sh.ty == 16) e = launch_build<32, 16>(L, s);
        else if (sh.ty == 12) e = launch_build<32, 12>(L, s);
        else e = launch_build<32, 8>(L, s);
    }
    int mx[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mx, L.tab_max, sizeof(mx), cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "work tables of the tile kernel");
    for (int s = 0; s < 2; ++s) L.tab_words[s] = (mx[s] + 3) / 4 * 4;
    return MCLBM_OK;
}

void tma_release(Lattice &L) {
    delete[] static_cast<CUtensorMap *>(L.tmaps);
    L.tmaps = nullptr;
    for (int s = 0; s < 2; ++s) {
        cudaFree(L.tab[s]);
        L.tab[s] = nullptr;
    }
    cudaFree(L.tab_max);
    L.tab_max = nullptr;
}

size_t tile_maps_bytes() { return MAPS_PER_CASE * sizeof(CUtensorMap); }

int tile_maps_for(const Lattice &L, int shape, void *out) { return encode_tile_maps(L, shape, out); }

int batch_slots(mclbm_precision p, int shape) {
    int slots = 0;
    launch_any(p, nullptr, 2, nullptr, shape, 0, 0, &slots);
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
    const int s = L.tile_shape;
    return launch_step_batch(&one, 1, static_cast<const CUtensorMap *>(L.tmaps) + s * MAPS_PER_CASE,
                             s, 0, L.stream);
}

}  // namespace mclbm
