// Fluid-only step (kernel 4): the populations of the fluid nodes only, so
// that a step reads and writes 2 x 9 x 2 populations per fluid node and no
// solid node costs memory traffic.
//
// Tiles: the lattice is cut into bands of TY rows (12 for shape 0, 16 for
// shape 1), each band into tiles of at most 32 columns holding at most as
// many fluid nodes as the CTA has compute threads (256 or 384), so that a
// tile of a sparse region is wider than one of an open region.  A tile is
// narrowed further where its staged set or its table would not fit the
// shared memory of the target number of CTAs per SM (three or two).
//
// Storage: fs[b] = [nfp][planes] (a node's populations contiguous, so that
// a range of nodes is one bulk copy), the fluid nodes tile by tile (bands
// top to bottom, tiles left to right); inside a tile in border bands of
// width 3 -- top-left corner, top edge, top-right corner, right edge,
// bottom-right corner, bottom edge, bottom-left corner, left edge -- then
// the interior, each band padded to a 16-byte multiple.  A neighbour's halo
// band is then one or two contiguous ranges of its block.
//
// Per tile, built on the host from the geometry and validated against every
// buffer bound before the kernel may run:
//   copy record  the ranges (source, length, destination, in 16-byte units) whose
//                bulk copies stage the tile's own block and the fluid nodes
//                of its 3-node ring, all planes, into shared memory
//   table        the tile's origin, its work lists (own nodes with their
//                block index, ring pulls, ring non-fluid nodes) and the
//                staged slot of every position of the staged frame
// The step per tile: stage (bulk copies on one mbarrier), then the phases
// of the dense tile kernel, reading staged nodes through the slot map --
// pull + Set-3 + densities (Eq. 3), virtual solid densities (Eqs. 16-17),
// forces (Eqs. 12-15), tau_s, u (Eqs. 6-9), collision (Eqs. 1, 2, 11) --
// and one bulk store per plane of the tile's block.  Periodic edges need no
// ghost copies: a ring node across an edge is staged from its own tile.
//
// The dense buffers stay the interchange format of the library; the two
// layouts are converted lazily (dense_to_sparse / sparse_to_dense).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "async_copy.cuh"
#include "lbm_device.cuh"

namespace mclbm {

namespace {

constexpr int STX = 32;                  // largest tile width
constexpr int SFW = STX + 6;             // staged frame: tile + 3-node ring
constexpr int SDXW = STX + 4;            // density frame: tile + 2-node ring
constexpr int MAXR = 24;                 // ranges per tile (own block included)
constexpr int REC_WORDS = 4 + 3 * MAXR;  // copy record: n, bytes, own_len, start, ranges
constexpr int HDR = 8;                   // table header words
constexpr uint32_t SET3 = 3u << 20, IN_BIT = 1u << 20, OUT_BIT = 2u << 20;
static_assert((REC_WORDS * 4) % 16 == 0, "copy records are copied in 16-byte chunks");

// Band height TY -> compute threads (= most fluid nodes of a tile) and
// resident CTAs per SM the shared memory is budgeted for.
constexpr int threads_for(int ty) { return ty == 16 ? 384 : 256; }
constexpr int ctas_for(int ty) { return ty == 16 ? 2 : 3; }
// Shared memory of one CTA: 228 KB per SM, 1 KB of it reserved per CTA.
constexpr size_t smem_budget(int ty) { return (size_t)233472 / ctas_for(ty) - 1024; }

constexpr size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
// bytes of the shared-memory layout for scap staged slots of node_bytes
// each, tabw table words and density frame sn1 (regions in this order)
constexpr size_t smem_bytes(int scap, int node_bytes, int tabw, int sn1) {
    return round_up(round_up(round_up((size_t)scap * node_bytes, 128) * 2 + (size_t)4 * sn1 * 4, 128) +
                        (size_t)2 * tabw * 4 + REC_WORDS * 4,
                    16) +
           32;
}

template <class P, int STY>
struct SLayout {
    using S = typename P::store_t;
    using R = typename P::real_t;
    static constexpr int NT = threads_for(STY);
    static constexpr int SFH = STY + 6, SN1 = SDXW * (STY + 4);
    static_assert(SFW * SFH < 65535, "frame positions are 16-bit");
    static constexpr int NPL = P::planes, NB = NPL * (int)sizeof(S);
    // slots per 16-byte multiple (a node is NPL * sizeof(S) = 72 or 40 bytes)
    static constexpr int Q = 16 / (NB & 15 ? (NB & 15) : 16);
    static constexpr int OCAP = (NT + 9 * (Q - 1) + Q - 1) / Q * Q;  // own block
    // table: header, own + ring + ring non-fluid entries (disjoint positions
    // of the density frame), then the staged slot of every frame position
    // (16 bits each): the most a tile can need
    static constexpr int TABW = (HDR + SN1 + (SFW * SFH + 1) / 2 + 3) / 4 * 4;
    // the builder's table limit: work lists of up to 7/4 entries per
    // compute thread (a tile that needs more is narrowed), so that the
    // staged set keeps the rest of the budget
    static constexpr int TAB_CAP = std::min(TABW, (HDR + NT * 7 / 4 + (SFW * SFH + 1) / 2 + 3) / 4 * 4);
    // staged slots: the most (a multiple of 16) that fits the budget next to
    // TAB_CAP; the two stages [slot][plane] hold the tile being computed and
    // the next one in flight, and a stage's own block also receives the
    // tile's output
    static constexpr int scap_fit(int c) {
        return c <= 16 || smem_bytes(c, NB, TAB_CAP, SN1) <= smem_budget(STY) ? c : scap_fit(c - 16);
    }
    static constexpr int SCAP = scap_fit(((int)(smem_budget(STY) / 2 / NB) + 15) / 16 * 16);
    static constexpr size_t total = smem_bytes(SCAP, NB, TAB_CAP, SN1);
    static_assert(total <= smem_budget(STY), "shared memory of the target CTAs per SM");
    static_assert(SCAP >= OCAP + 16, "a tile's own block fits the stage");
    static_assert(OCAP <= 1023, "own-block index is 10 bits");
    static_assert(SCAP * NPL < 65535, "staged element offsets are 16-bit");
    static_assert((TABW * 4) % 16 == 0 && (Q * NPL * sizeof(S)) % 16 == 0, "bulk copy granularity");
};

}  // namespace

// kernel 4 serves FP32 and the 16-bit deviation storages (FP32 deviation
// storage, 20 planes of 4 bytes, does not fit two CTAs per SM)
bool sparse_precision(mclbm_precision p) {
    return p == MCLBM_FP32 || p == MCLBM_FP16_DEV || p == MCLBM_BF16_DEV;
}

namespace {

int table_capacity(mclbm_precision p, int sty) {
    if (sty == 12) return p == MCLBM_FP32 ? SLayout<P32, 12>::TAB_CAP : SLayout<P16D, 12>::TAB_CAP;
    return p == MCLBM_FP32 ? SLayout<P32, 16>::TAB_CAP : SLayout<P16D, 16>::TAB_CAP;
}
int staged_capacity(mclbm_precision p, int sty) {
    if (sty == 12) return p == MCLBM_FP32 ? SLayout<P32, 12>::SCAP : SLayout<P16D, 12>::SCAP;
    return p == MCLBM_FP32 ? SLayout<P32, 16>::SCAP : SLayout<P16D, 16>::SCAP;
}

// The lattices of a launch (1, or up to MAX_BATCH for a batch).
template <int N>
struct SArgs {
    StepArgs a[N];
    const void *fin[N];  // [nfp][planes]
    void *fout[N];
    const uint32_t *tab[N];   // [tiles][tab_words]
    const uint32_t *rec[N];   // [tiles][REC_WORDS]
    int tab_words[N];
    int first[N + 1];         // first work item of each lattice
    int ncases, total, tab_stride;
    // shared-memory layout, sized by the largest tile of the launch
    uint32_t stage_bytes, rho_off, tab_off, rec_off, bar_off;
};

// offsets of the shared-memory regions for staged slots scap (per stage)
// and table words tabw; returns the total bytes
template <class P, int STY, int N>
size_t smem_layout(int scap, int tabw, SArgs<N> &s) {
    constexpr int SN1 = SDXW * (STY + 4);
    using S = typename P::store_t;
    using R = typename P::real_t;
    auto up = [](size_t v, size_t a) { return (v + a - 1) / a * a; };
    s.stage_bytes = (uint32_t)up((size_t)scap * P::planes * sizeof(S), 128);
    s.rho_off = 2 * s.stage_bytes;
    s.tab_off = (uint32_t)up(s.rho_off + (size_t)4 * SN1 * sizeof(R), 128);  // two density buffers
    s.rec_off = (uint32_t)(s.tab_off + (size_t)2 * tabw * 4);
    s.bar_off = (uint32_t)up(s.rec_off + REC_WORDS * 4, 16);
    return s.bar_off + 32;  // mbarriers full[2], done[2]
}

// bulk store shared -> global with an L2 cache policy for the written lines
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes, uint64_t policy) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes), "l"(policy)
                 : "memory");
}

// The two components of a stored value sit side by side in the fluid-only
// layout (plane 2 i + comp for population i, 18 + comp for the reference
// densities of the deviation storages), so that one 8-byte (FP32) or
// 4-byte (16-bit) shared-memory access moves both.
__device__ __forceinline__ float2 pair_load(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 pair_load(const __half *p) {
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
__device__ __forceinline__ float2 pair_load(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
__device__ __forceinline__ void pair_store(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
__device__ __forceinline__ void pair_store(__half *p, float a, float b) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void pair_store(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
// dense plane (comp * 9 + i, or 18 + comp) of fluid-only plane k
__host__ __device__ __forceinline__ int dense_plane(int k) { return k < 18 ? (k & 1) * 9 + (k >> 1) : k; }

// named barrier `id` over `count` threads, and the same with an OR vote
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_or(bool v, int id, int count) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// CM: collision chosen at compile time (0 SRT of Eq. 1, 1 MRT) for a
// single lattice, by each case's flag (2) in a batch
template <class P, int STY, int N, int CM>
__global__ void __launch_bounds__(threads_for(STY) + 32, ctas_for(STY)) sparse_kernel(const __grid_constant__ SArgs<N> s) {
    using L = SLayout<P, STY>;
    constexpr int SN1 = L::SN1;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int NT = L::NT, NPL = L::NPL;
    // NT compute threads, then one producer warp: it stages tiles into two
    // stages ahead of the compute warps and stores their output, and meets
    // them only on mbarriers (full[k]: stage k staged; done[k]: stage k's
    // tile computed), never on their barriers (named barrier 1, NT threads)
    constexpr int PW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    auto stage = [&](int k) { return reinterpret_cast<S *>(smem + (size_t)k * s.stage_bytes); };
    static_assert(sizeof(R) == 4, "the fluid-only kernel computes in FP32");
    // two density buffers of [SN1] (rho1, rho2) pairs
    float2 *rho0 = reinterpret_cast<float2 *>(smem + s.rho_off);
    uint32_t *tabs = reinterpret_cast<uint32_t *>(smem + s.tab_off);
    uint32_t *rec = reinterpret_cast<uint32_t *>(smem + s.rec_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + s.bar_off);
    uint64_t *done = full + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the case of work item w; a thread's queries mostly move forward (its
    // tiles are w = blockIdx.x + m * gridDim.x), so the search starts at the
    // case of its previous query
    int c_hint = 0;
    auto case_of = [&](int w) -> int {
        if constexpr (N == 1) {
            return 0;
        } else {
            int c = w >= s.first[c_hint] ? c_hint : 0;
            while (c + 1 < s.ncases && w >= s.first[c + 1]) ++c;
            c_hint = c;
            return c;
        }
    };

    // L2 policies of the copy warp (made where used, so that no register
    // holds them across the tile loop): the per-tile tables and copy records
    // (read every step, about 6 % of a step's bytes) are kept in L2 across
    // steps; the output block is not read again before the next step has
    // streamed the whole lattice, so its lines go first.
    // copy warp: start the copy of tile w's record into shared memory
    auto fetch_record = [&](int w) {
        const int c = case_of(w);
        if (lane < REC_WORDS / 4) {
            const uint32_t *src = s.rec[c] + (size_t)(w - s.first[c]) * REC_WORDS + 4 * lane;
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                             smem_u32(rec + 4 * lane)),
                         "l"(src), "l"(policy_evict_last())
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // copy warp: stage tile w (record already in shared memory) into stage
    // and table buffer k, completing on mbarrier k
    auto issue = [&](int w, int k) {
        const int c = case_of(w);
        const S *fin = static_cast<const S *>(s.fin[c]);
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        const int nr = (int)rec[0];
        const uint32_t tbytes = 4u * (uint32_t)s.tab_words[c];
        S *dst_stage = stage(k);
        fence_proxy_async();
        if (lane == 0) {
            mbar_expect_tx(&full[k], rec[1] + tbytes);
            bulk_g2s_hint(tabs + k * s.tab_stride, s.tab[c] + (size_t)(w - s.first[c]) * s.tab_words[c],
                          tbytes, &full[k], policy_evict_last());
        }
        __syncwarp();
        for (int r = lane; r < nr; r += 32) {
            // source, length and destination in 16-byte units
            const uint32_t src = rec[4 + 3 * r], len = rec[5 + 3 * r], dst = rec[6 + 3 * r];
            bulk_g2s(reinterpret_cast<unsigned char *>(dst_stage) + (size_t)dst * 16,
                     reinterpret_cast<const unsigned char *>(fin) + (size_t)src * 16, len * 16u, &full[k]);
        }
        __syncwarp();
    };

    // A single-lattice launch follows the previous step programmatically:
    // the next step's grid may start as soon as the hardware allows, its
    // CTAs set up and fetch their first copy record (static) while this one
    // drains, and wait for the previous grid before touching the populations
    // (griddepcontrol.wait: that grid complete, its writes visible).
    // Without that launch attribute both instructions are no-ops.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&done[0], NT / 32);
        mbar_init(&done[1], NT / 32);
        fence_mbar_init();
    }
    __syncthreads();
    if ((int)blockIdx.x >= s.total) return;
    const int ntiles = (s.total - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    // (the test hook stages nothing: the first tile's wait runs out)
    const bool copies = !s.a[case_of(blockIdx.x)].test_no_copy;

    if (warp == PW) {
        // ---- producer: tile m of this CTA lives in stage m & 1 --------------------
        if (!copies) return;
        auto tile = [&](int m) { return (int)blockIdx.x + m * (int)gridDim.x; };
        // wait until tile m has been computed, then store its output (the
        // own block of its stage; length and start in table words 4 and 5)
        auto store = [&](int m) -> bool {
            const int km = m & 1, c = case_of(tile(m));
            if (!mbar_wait(&done[km], (uint32_t)(m >> 1) & 1u, s.a[c].wait_ns)) return false;
            const uint32_t *T = tabs + km * s.tab_stride;
            const uint32_t own_len = T[4], start = T[5];
            if (lane == 0 && own_len > 0)
                bulk_s2g(static_cast<S *>(s.fout[c]) + (size_t)start * NPL, stage(km),
                         own_len * (uint32_t)(NPL * sizeof(S)), policy_evict_first());
            bulk_commit();
            return true;
        };
        bool ok = true;
        int issued = 0;
        fetch_record(tile(0));
        asm volatile("griddepcontrol.wait;" ::: "memory");
        for (int m = 0; m < ntiles && ok; ++m) {
            if (m >= 2) {
                // stage m & 1 still holds tile m - 2: store it and wait until
                // the store has read the stage
                ok = store(m - 2);
                if (!ok) break;
                bulk_wait_read();
            }
            issue(tile(m), m & 1);
            ++issued;
            if (m + 1 < ntiles) fetch_record(tile(m + 1));
        }
        for (int m = ntiles > 2 ? ntiles - 2 : 0; m < ntiles && ok; ++m) ok = store(m);
        bulk_wait_read();
        if (!ok) {
            // a wait ran out: report it, and give the copies in flight a
            // bounded time to land before the shared memory is released
            const StepArgs &a = s.a[case_of(blockIdx.x)];
            const uint64_t drain = a.wait_ns < DRAIN_LIMIT_NS ? a.wait_ns : DRAIN_LIMIT_NS;
            if (lane == 0) atomicExch(a.err, MCLBM_ERR_TIMEOUT);
            for (int m = issued > 2 ? issued - 2 : 0; m < issued; ++m)
                mbar_wait(&full[m & 1], (uint32_t)(m >> 1) & 1u, drain);
        }
        return;
    }

    // ---- compute warps ----------------------------------------------------------
    // Tile n lives in stage n & 1 and densities buffer n & 1.  Per tile:
    //   X: collision (C) of tile n, then the pulls and densities (A) of
    //      tile n + 1 -- the threads without a node in C take the ring pulls
    //      of A, so that the two phases share one barrier;
    //   B: virtual solid densities of tile n + 1.
    // A thread keeps its own node's populations in registers from A to C.
    // A: pull + Set-3 + densities (Eq. 3) of tile w in stage k: the ring
    // entries from the last thread down, the own node of thread tid
    auto phase_a = [&](int w, int k, R f[2][9], R &rho1, R &rho2) {
        const StepArgs &a = s.a[case_of(w)];
        const S *stg = stage(k);
        float2 *rho = rho0 + k * SN1;
        const uint32_t *T = tabs + k * s.tab_stride;
        const int n_own = (int)T[0], n_ring = (int)T[1], n_sol = (int)T[2];
        const int x0 = (int)T[6], y0 = (int)T[7];  // the tile's origin
        const uint32_t *E = T + HDR;
        // staged element offset (slot x planes) of every frame position (0
        // where nothing is staged)
        const uint16_t *slot_of = reinterpret_cast<const uint16_t *>(E + n_own + n_ring + n_sol);
        // population (plane, comp) of the staged node at element offset
        // off, and both components of a plane at once
        auto val = [&](int plane, int comp, int off, R wt) -> R {
            R v = to_real(stg[off + 2 * plane + comp]);
            if constexpr (P::ref) v += wt * to_real(stg[off + 18 + comp]);
            return v;
        };
        auto val2 = [&](int plane, int off, R wt, R &v0, R &v1) {
            float2 v = pair_load(stg + off + 2 * plane);
            if constexpr (P::ref) {
                const float2 r = pair_load(stg + off + 18);
                v.x += wt * r.x;
                v.y += wt * r.y;
            }
            v0 = v.x;
            v1 = v.y;
        };
        // f_i = f*_i(x - e_i), or the node's own f*_opp(i) where x - e_i is
        // not fluid (half-way bounce-back), then the open-end treatment
        // (Sec. 2.3)
        auto pull = [&](int fpos, int ooff, uint32_t e, int x, int y, R g9[2][9]) {
            const uint32_t m = (e >> 12) & 0xffu;
            val2(0, ooff, wgt<R>(0), g9[0][0], g9[1][0]);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const bool sb = (m >> (opp(i) - 1)) & 1u;
                const int off = sb ? ooff : (int)slot_of[fpos - ey(i) * SFW - ex(i)];
                const int pl = sb ? opp(i) : i;
                val2(pl, off, wgt<R>(i), g9[0][i], g9[1][i]);
            }
            if (e & SET3)
                apply_open_bc<R>(a, x, y, [&](int comp, int i) { return val(i, comp, ooff, wgt<R>(i)); }, g9);
        };
        for (int kk = NT - 1 - tid; kk < n_ring; kk += NT) {
            const uint32_t e = E[n_own + kk];
            const int pos = (int)(e & 0xfffu);
            const int dr = pos / SDXW, dc = pos - dr * SDXW;
            const int fpos = (dr + 1) * SFW + dc + 1;
            R fr[2][9];
            pull(fpos, slot_of[fpos], e, x0 - 2 + dc, wrap(y0 - 2 + dr, a.g.ny), fr);
            R r1 = 0, r2 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                r1 += fr[0][i];
                r2 += fr[1][i];
            }
            rho[pos] = make_float2(r1, r2);
        }
        if (tid < n_own) {
            const uint32_t me = E[tid];
            const int tx = (int)(me & 63u), ty = (int)((me >> 6) & 63u), bidx = (int)(me >> 22);
            pull((ty + 3) * SFW + tx + 3, bidx * NPL, me, x0 + tx, y0 + ty, f);
            rho1 = 0;
            rho2 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                rho1 += f[0][i];
                rho2 += f[1][i];
            }
            rho[(ty + 2) * SDXW + tx + 2] = make_float2(rho1, rho2);
        }
    };
    // B: virtual solid densities (Eqs. 16-17) on the 1-ring (zero outside),
    // times G_ads / G_coh where G_coh != 0: the force stencil of phase C
    // then weights every neighbour by G_coh w_i
    auto phase_b = [&](int w, int k) {
        const StepArgs &a = s.a[case_of(w)];
        const Geometry &g = a.g;
        const R scale = a.p.g_coh_f != 0.f ? R(a.p.ads_over_coh_f) : R(1);
        float2 *rho = rho0 + k * SN1;
        const uint32_t *T = tabs + k * s.tab_stride;
        const int n_own = (int)T[0], n_ring = (int)T[1], n_sol = (int)T[2];
        const uint32_t *Es = T + HDR + n_own + n_ring;
        for (int kk = tid; kk < n_sol; kk += NT) {
            const uint32_t e = Es[kk];
            const int pos = (int)(e & 0xfffu);
            const int code = (int)((e >> 12) & 0xffu);
            const uint32_t fm = e >> 20;
            R n1s = 0, n2s = 0, den = 0;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if ((fm >> (i - 1)) & 1u) {
                    const R w8 = wgt<R>(i);
                    const int q = pos + ey(i) * SDXW + ex(i);
                    const float2 r = rho[q];
                    n1s += w8 * r.x;
                    n2s += w8 * r.y;
                    den += w8;
                }
            }
            R s1 = 0, s2 = 0;
            if (den > R(0) && code != GEO_OUTSIDE) {
                const R inv = scale / den;
                s1 = chi_at<R>(g, 2 * code) * n1s * inv;
                s2 = chi_at<R>(g, 2 * code + 1) * n2s * inv;
            }
            rho[pos] = make_float2(s1, s2);
        }
    };
    // C: forces (Eqs. 12-15), tau_s and u (Eqs. 6-9) and the collision
    // (Eqs. 1, 2, 11) of the own node of thread tid in tile w; the output
    // goes to the stage's own block, then each warp hands the stage over
    auto phase_c = [&](int w, int k, R f[2][9], R rho1, R rho2) {
        const StepArgs &a = s.a[case_of(w)];
        const float2 *rho = rho0 + k * SN1;
        const uint32_t *T = tabs + k * s.tab_stride;
        if (tid < (int)T[0]) {
            const uint32_t me = T[HDR + tid];
            const int tx = (int)(me & 63u), ty = (int)((me >> 6) & 63u), bidx = (int)(me >> 22);
            const int dpos = (ty + 2) * SDXW + tx + 2;
            const uint32_t m = (me >> 12) & 0xffu;
            R fx1, fy1, fx2, fy2;
            // Eqs. 12-15 with one coupling: F^s = -rho^s G_coh sum_i w_i
            // psi'^sb(x + e_i) e_i + rho^s g, psi' the density of a fluid
            // neighbour or the scaled virtual density of a solid one; the
            // axis and diagonal differences of the 8 neighbours
            auto uniform_force = [&](auto nb) {
                float2 v[9];
#pragma unroll
                for (int i = 1; i < 9; ++i) v[i] = nb(i);
                const R gca = R(a.p.g_coh_f) * wgt<R>(1), gcd = R(a.p.g_coh_f) * wgt<R>(5);
                const R px = (v[5].x + v[8].x) - (v[6].x + v[7].x), py = (v[5].x + v[6].x) - (v[7].x + v[8].x);
                const R qx = (v[5].y + v[8].y) - (v[6].y + v[7].y), qy = (v[5].y + v[6].y) - (v[7].y + v[8].y);
                const R sx1 = gca * (v[1].y - v[3].y) + gcd * qx, sy1 = gca * (v[2].y - v[4].y) + gcd * qy;
                const R sx2 = gca * (v[1].x - v[3].x) + gcd * px, sy2 = gca * (v[2].x - v[4].x) + gcd * py;
                fx1 = rho1 * (R(a.p.gx_f) - sx1);
                fy1 = rho1 * (R(a.p.gy_f) - sy1);
                fx2 = rho2 * (R(a.p.gx_f) - sx2);
                fy2 = rho2 * (R(a.p.gy_f) - sy2);
            };
            if (a.p.g_coh_f != 0.f) {
                if (me & SET3) {
                    // Sec. 2.1: a neighbour beyond an open end is replaced by
                    // the one in the opposite direction
                    const bool mir_in = me & IN_BIT, mir_out = me & OUT_BIT;
                    uniform_force([&](int i) {
                        const bool mir = (mir_in && ex(i) < 0) || (mir_out && ex(i) > 0);
                        const int d = ey(i) * SDXW + ex(i);
                        return rho[mir ? dpos - d : dpos + d];
                    });
                } else {
                    uniform_force([&](int i) { return rho[dpos + ey(i) * SDXW + ex(i)]; });
                }
            } else if (me & SET3) {
                // Sec. 2.1: a neighbour beyond an open end is replaced by the
                // one in the opposite direction
                const bool mir_in = me & IN_BIT, mir_out = me & OUT_BIT;
                node_force<R, false>(a.p, rho1, rho2,
                                     [&](int i, uint8_t &code, R &s1, R &s2) {
                                         const bool mir = (mir_in && ex(i) < 0) || (mir_out && ex(i) > 0);
                                         const int d = ey(i) * SDXW + ex(i);
                                         const int q = mir ? dpos - d : dpos + d;
                                         const uint32_t bit = mir ? (m >> (opp(i) - 1)) : (m >> (i - 1));
                                         code = (bit & 1u) ? 1 : GEO_FLUID;
                                         const float2 r = rho[q];
                                         s1 = r.x;
                                         s2 = r.y;
                                     },
                                     fx1, fy1, fx2, fy2);
            } else {
                node_force<R, false>(a.p, rho1, rho2,
                                     [&](int i, uint8_t &code, R &s1, R &s2) {
                                         const int q = dpos + ey(i) * SDXW + ex(i);
                                         code = ((m >> (i - 1)) & 1u) ? 1 : GEO_FLUID;
                                         const float2 r = rho[q];
                                         s1 = r.x;
                                         s2 = r.y;
                                     },
                                     fx1, fy1, fx2, fy2);
            }
            R omega, ux, uy;
            node_velocity<R>(a.p, f, rho1, rho2, fx1 + fx2, fy1 + fy2, omega, ux, uy);
            collide<R, CM>(a.p, f, rho1, rho2, ux, uy, fx1, fy1, fx2, fy2, omega);
            S *o = stage(k) + bidx * NPL;
            if constexpr (P::ref) {
                const S h1 = from_real<S>(rho1), h2 = from_real<S>(rho2);
                o[18] = h1;
                o[19] = h2;  // the reference pair, rounded once and reused below
                const R q1 = to_real(h1), q2 = to_real(h2);
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    pair_store(o + 2 * i, f[0][i] - wgt<R>(i) * q1, f[1][i] - wgt<R>(i) * q2);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) pair_store(o + 2 * i, f[0][i], f[1][i]);
            }
        }
        // the output is in the stage: one arrival per warp hands it to the
        // producer's store
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[k]);
    };
    auto timed_out = [&](int w) {
        // the producer finds the tile never computed and reports it
        if (tid == 0) atomicExch(s.a[case_of(w)].err, MCLBM_ERR_TIMEOUT);
    };

    R f[2][9];
    R rho1 = 0, rho2 = 0;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    {
        const bool bad = !mbar_wait(&full[0], 0u, s.a[case_of(blockIdx.x)].wait_ns);
        if (!bad) phase_a(blockIdx.x, 0, f, rho1, rho2);
        if (bar_or(bad, 1, NT)) {
            timed_out(blockIdx.x);
            return;
        }
    }
    int n = 0;
    for (int w = blockIdx.x; w < s.total; w += gridDim.x, ++n) {
        const int st = n & 1;
        phase_b(w, st);
        bar_sync(1, NT);
        phase_c(w, st, f, rho1, rho2);
        const int wn = w + (int)gridDim.x;
        bool bad = false;
        if (wn < s.total) {
            bad = !mbar_wait(&full[st ^ 1], (uint32_t)((n + 1) >> 1) & 1u, s.a[case_of(wn)].wait_ns);
            if (!bad) phase_a(wn, st ^ 1, f, rho1, rho2);
        }
        if (bar_or(bad, 1, NT)) {
            timed_out(wn);
            return;
        }
    }
}

// dense <-> fluid-only conversion, one thread per (slot, plane)
template <class P>
__global__ void to_sparse_kernel(Geometry g, const typename P::store_t *f, typename P::store_t *fs,
                                 const int *snode, long long nfp) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfp * P::planes) return;
    const long long sl = k / P::planes;
    const int pl = (int)(k - sl * P::planes);
    const int node = snode[sl];
    typename P::store_t v = typename P::store_t(0.f);
    if (node >= 0) v = f[(long long)dense_plane(pl) * g.plane + site_of(g, node % g.nx, node / g.nx)];
    fs[k] = v;
}

template <class P>
__global__ void to_dense_kernel(Geometry g, const typename P::store_t *fs, typename P::store_t *f,
                                const int *snode, long long nfp) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfp * P::planes) return;
    const long long sl = k / P::planes;
    const int pl = (int)(k - sl * P::planes);
    const int node = snode[sl];
    if (node >= 0) f[(long long)dense_plane(pl) * g.plane + site_of(g, node % g.nx, node / g.nx)] = fs[k];
}

template <class F>
cudaError_t dispatch_prec(mclbm_precision p, F fn) {
    switch (p) {
        case MCLBM_FP32: return fn(P32{});
        case MCLBM_FP16_DEV: return fn(P16D{});
        case MCLBM_BF16_DEV: return fn(PB16D{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host: layout and tables
// ---------------------------------------------------------------------------
namespace {
int sparse_build(Lattice &L, int STY);
}

int sparse_prepare(Lattice &L, int STY) {
    if (!sparse_precision(L.prec) || !L.geo_pad) return MCLBM_OK;  // kernel 4 unavailable
    if (L.sparse_mode == L.ghost_key() && L.nfp > 0 && L.sparse_ty == STY) return MCLBM_OK;
    // a geometry whose tiles do not fit is not tiled again for the same
    // boundary mode and band height (the geometry itself never changes)
    const int key = L.ghost_key() * 64 + STY;
    if (L.sparse_fail_key == key)
        return fail(MCLBM_ERR_STATE, "fluid-only layout: the tiles of this lattice do not fit the staging capacity");
    const int rc = sparse_build(L, STY);
    if (rc == MCLBM_ERR_STATE) L.sparse_fail_key = key;
    return rc;
}

namespace {
// The geometry codes as the step sees them (ghosts per the boundary mode),
// for x in [-3, nx + 3) and y in [-3, ny + 3): the step's reach (own nodes
// need forces from the 1-ring, virtual solid densities from the 2-ring,
// pulls from the 3-ring).
struct HostGeo {
    int nx, ny;
    const uint8_t *code;  // (ny + 6) rows of nx + 6, row y + 3, column x + 3
    int at(int x, int y) const {
        if (x < -3 || x >= nx + 3 || y < -3 || y >= ny + 3) return GEO_OUTSIDE;
        return code[(size_t)(y + 3) * (nx + 6) + (x + 3)];
    }
};

// The fluid-only layout of a lattice, built on the host from its geometry.
struct HostLayout {
    long long nfp = 0;
    std::vector<int> snode;    // [nfp] lattice node y * nx + x of each slot, -1 padding
    std::vector<uint32_t> tab;  // [ntiles][tab_words]
    std::vector<uint32_t> rec;  // [ntiles][REC_WORDS]
    int tab_words = 0, ntiles = 0, attempts = 0;
    long long max_own = 0, max_stage = 0;
};

// Tiles, blocks, tables and copy records for bands of STY rows (nodes of
// planes x store_bytes; Q slots make a 16-byte multiple).
int build_layout(const HostGeo &g, int STY, mclbm_precision prec, int planes, int store_bytes, int Q, bool open_x,
                 HostLayout &out) {
    const int SFH = STY + 6, SN1 = SDXW * (STY + 4);
    const int nx = g.nx, ny = g.ny;
    const int NB = planes * store_bytes;  // bytes of a node
    const int NT = threads_for(STY);
    const int tabcap = table_capacity(prec, STY), scap = staged_capacity(prec, STY);
    auto fluid_mask = [&](int x, int y) {
        uint32_t m = 0;
        for (int i = 1; i < 9; ++i)
            if (g.at(x + ex(i), y + ey(i)) == GEO_FLUID) m |= 1u << (i - 1);
        return m;
    };
    auto set3 = [&](int x) -> uint32_t {
        return (open_x && x == 0 ? IN_BIT : 0u) | (open_x && x == nx - 1 ? OUT_BIT : 0u);
    };
    // border band of in-tile position (tx, ty) against the tile's extent
    // (tw, th), so that what a neighbour stages stays contiguous
    auto band = [&](int tx, int ty, int tw, int th) {
        const bool l = tx < 3, r = tx >= tw - 3, t = ty < 3, b = ty >= th - 3;
        if (t && l) return 0;
        if (t && !r) return 1;
        if (t) return 2;
        if (r && !b) return 3;
        if (r) return 4;
        if (b && !l) return 5;
        if (b) return 6;
        if (l) return 7;
        return 8;
    };
    struct Tile {
        int x0, y0, w, h;
    };
    // What tile (x0, y0, tw, th) computes, from the geometry alone.  Only
    // what the tile's own nodes read is computed: the densities or virtual
    // solid densities of their 8 neighbours (forces, Eqs. 12-15; the
    // open-end mirror reads the opposite neighbour, also one of the 8), the
    // fluid neighbours of those solid neighbours (Eq. 17), and the
    // populations those densities pull.  Positions of the density frame:
    // own (1), neighbour of an own node (2), density needed (4).  Returns
    // the ring and non-fluid entries, the own block (lattice nodes in band
    // order, -1 padding) and the staged frame positions outside the tile.
    struct Work {
        std::vector<int> blk;
        std::vector<uint32_t> ring, sol;
        std::vector<int> need;  // frame positions r * SFW + c
        int n_own = 0;
    };
    std::vector<uint8_t> mark_buf((size_t)SN1), pulled_buf((size_t)SFW * SFH);
    auto tile_work = [&](const Tile &tl, Work &W) {
        const int x0 = tl.x0, y0 = tl.y0, tw = tl.w, th = tl.h;
        W.blk.clear();
        W.ring.clear();
        W.sol.clear();
        W.need.clear();
        W.n_own = 0;
        for (int bnd = 0; bnd < 9; ++bnd) {
            for (int ty = 0; ty < th; ++ty)
                for (int tx = 0; tx < tw; ++tx) {
                    if (band(tx, ty, tw, th) != bnd) continue;
                    if (g.at(x0 + tx, y0 + ty) == GEO_FLUID) {
                        W.blk.push_back((y0 + ty) * nx + x0 + tx);
                        ++W.n_own;
                    }
                }
            while (W.blk.size() % Q) W.blk.push_back(-1);
        }
        std::vector<uint8_t> &mark = mark_buf;
        std::fill(mark.begin(), mark.end(), (uint8_t)0);
        auto dpos = [&](int x, int y) { return (y - y0 + 2) * SDXW + (x - x0 + 2); };
        for (int n : W.blk) {
            if (n < 0) continue;
            const int x = n % nx, y = n / nx;
            mark[(size_t)dpos(x, y)] |= 1;
            for (int d = 1; d < 9; ++d) mark[(size_t)dpos(x + ex(d), y + ey(d))] |= 2;
        }
        for (int k = 0; k < SN1; ++k) {
            const int dr = k / SDXW, dc = k % SDXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
            if (!(mark[k] & 2)) continue;
            const int c = g.at(x, y);
            if (c == GEO_FLUID) {
                mark[k] |= 4;
                continue;
            }
            const uint32_t fm = fluid_mask(x, y);
            W.sol.push_back((uint32_t)k | (uint32_t)c << 12 | fm << 20);
            if (c == GEO_OUTSIDE) continue;  // zero: its neighbours are not read
            for (int d = 1; d < 9; ++d)
                if ((fm >> (d - 1)) & 1u) mark[(size_t)(k + ey(d) * SDXW + ex(d))] |= 4;
        }
        // the ring's densities, and the staged frame positions they and the
        // own nodes pull from (fluid sources outside the tile's own block)
        std::vector<uint8_t> &pulled = pulled_buf;
        std::fill(pulled.begin(), pulled.end(), (uint8_t)0);
        auto mark_sources = [&](int x, int y) {
            for (int d = 1; d < 9; ++d) {
                const int sx = x - ex(d), sy = y - ey(d);
                if (g.at(sx, sy) == GEO_FLUID) pulled[(size_t)(sy - y0 + 3) * SFW + (sx - x0 + 3)] = 1;
            }
        };
        for (int k = 0; k < SN1; ++k) {
            const int dr = k / SDXW, dc = k % SDXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
            if (mark[k] & 1) {
                mark_sources(x, y);
                continue;
            }
            if (!(mark[k] & 4)) continue;
            W.ring.push_back((uint32_t)k | (~fluid_mask(x, y) & 0xffu) << 12 | set3(x));
            mark_sources(x, y);
            // and the node itself: its bounce-back and its open-end
            // treatment read its own populations, which no other pulled node
            // may stage
            pulled[(size_t)(y - y0 + 3) * SFW + (x - x0 + 3)] = 1;
        }
        for (int r = 0; r < SFH; ++r)
            for (int c = 0; c < SFW; ++c) {
                const int x = x0 - 3 + c, y = y0 - 3 + r;
                const bool in_tile = x >= x0 && x < x0 + tw && y >= y0 && y < y0 + th;
                if (!in_tile && pulled[(size_t)r * SFW + c]) W.need.push_back(r * SFW + c);
            }
    };
    auto words_of = [&](const Work &W) {
        return (long long)HDR + W.n_own + (long long)W.ring.size() + (long long)W.sol.size() + (SFW * SFH + 1) / 2;
    };

    // 1. tiles: every band of STY rows cut from the left into the widest
    // tiles (at most STX columns) whose own nodes fit the compute threads
    // and whose table and staged set fit their capacities.  The staged
    // ranges are padded to 16-byte multiples once the slots are known; the
    // padding each tile needed is remembered per column of its band
    // (padc), and a later attempt reserves the largest value under a
    // candidate tile, so that an attempt after an overflow converges.
    std::vector<Tile> tiles;
    std::vector<Work> works;
    const int nbands = (ny + STY - 1) / STY;
    // first guess of the padding: twice the rounding of a full record (at
    // most 15 bytes at either end of each of MAXR ranges)
    std::vector<int> padc((size_t)nbands * nx, 2 * ((MAXR * 30 + NB - 1) / NB));
    std::vector<int> col;
    Work scratch;
    auto partition = [&]() -> bool {
        tiles.clear();
        works.clear();
        col.assign((size_t)nx, 0);
        for (int y0 = 0; y0 < ny; y0 += STY) {
            const int th = std::min(STY, ny - y0);
            for (int x = 0; x < nx; ++x) {
                col[(size_t)x] = 0;
                for (int ty = 0; ty < th; ++ty) col[(size_t)x] += g.at(x, y0 + ty) == GEO_FLUID;
            }
            for (int x0 = 0; x0 < nx;) {
                int w = std::min(STX, nx - x0);
                const int *pb = &padc[(size_t)(y0 / STY) * nx];
                auto fluid = [&](int width) {
                    int n = 0;
                    for (int x = x0; x < x0 + width; ++x) n += col[(size_t)x];
                    return n;
                };
                while (w > 1 && fluid(w) > NT) --w;
                Work &W = scratch;
                for (;; --w) {
                    if (w < 1) return false;
                    const int pad = *std::max_element(pb + x0, pb + x0 + w);
                    tile_work(Tile{x0, y0, w, th}, W);
                    if (W.n_own <= NT && words_of(W) <= tabcap &&
                        (long long)W.blk.size() + (long long)W.need.size() + pad <= scap)
                        break;
                }
                tiles.push_back(Tile{x0, y0, w, th});
                works.push_back(W);
                x0 += w;
            }
        }
        return true;
    };

    std::vector<long long> start;
    std::vector<int> gidx, snode;
    std::vector<std::vector<uint32_t>> tabs;
    std::vector<uint32_t> recs;
    long long nfp = 0;
    int maxw = HDR;
    long long max_own = Q, max_stage = Q;
    for (int attempt = 0;; ++attempt) {
        out.attempts = attempt + 1;
        if (attempt > 32 || !partition())
            return fail(MCLBM_ERR_STATE, "fluid-only layout: no tiling fits the staging capacity");
        const int ntiles = (int)tiles.size();
        // 2. blocks: own fluid nodes of every tile in band order, bands padded
        start.assign((size_t)ntiles + 1, 0);
        for (int t = 0; t < ntiles; ++t) start[(size_t)t + 1] = start[(size_t)t] + (long long)works[(size_t)t].blk.size();
        nfp = std::max<long long>(start[(size_t)ntiles], Q);
        if (nfp >= (1LL << 31)) return fail(MCLBM_ERR_ARG, "lattice too large for the fluid-only layout");
        gidx.assign((size_t)nx * ny, -1);
        snode.assign((size_t)nfp, -1);
        for (int t = 0; t < ntiles; ++t) {
            const std::vector<int> &B = works[(size_t)t].blk;
            for (size_t i = 0; i < B.size(); ++i) {
                snode[(size_t)(start[(size_t)t] + (long long)i)] = B[i];
                if (B[i] >= 0) gidx[(size_t)B[i]] = (int)(start[(size_t)t] + (long long)i);
            }
        }
        auto src_of = [&](int x, int y) -> int {  // slot of lattice position (x, y), wrapped
            if (x < 0 || x >= nx) x = ((x % nx) + nx) % nx;
            if (y < 0 || y >= ny) y = ((y % ny) + ny) % ny;
            return gidx[(size_t)y * nx + x];
        };

        // 3. tables and copy records
        tabs.assign((size_t)ntiles, {});
        recs.assign((size_t)ntiles * REC_WORDS, 0);
        maxw = HDR;
        max_own = Q;
        max_stage = Q;
        bool overflow = false;  // a tile's padded ranges overflowed the stage
        for (int t = 0; t < ntiles; ++t) {
            const Tile &tl = tiles[(size_t)t];
            const Work &W = works[(size_t)t];
            const int x0 = tl.x0, y0 = tl.y0;
            std::vector<uint32_t> own;
            std::vector<uint16_t> smap((size_t)SFW * SFH, 0);
            for (size_t i = 0; i < W.blk.size(); ++i) {
                const int n = W.blk[i];
                if (n < 0) continue;
                const int x = n % nx, y = n / nx;
                own.push_back((uint32_t)(x - x0) | (uint32_t)(y - y0) << 6 | (~fluid_mask(x, y) & 0xffu) << 12 |
                              set3(x) | (uint32_t)i << 22);
                smap[(size_t)(y - y0 + 3) * SFW + (x - x0 + 3)] = (uint16_t)(i * planes);
            }
            // ring nodes to stage: pulled fluid positions outside the own block
            std::vector<std::pair<int, int>> need;  // (slot, frame position)
            for (int fp : W.need) {
                const int gsl = src_of(x0 - 3 + fp % SFW, y0 - 3 + fp / SFW);
                if (gsl < 0) return fail(MCLBM_ERR_STATE, "fluid-only layout: ring node without a slot");
                need.push_back({gsl, fp});
            }
            std::sort(need.begin(), need.end());
            // ranges: the own block first, then runs of the ring's slots, in
            // 16-byte units (a run starts and ends on the 16-byte boundaries
            // around its first and last node, so that at most 15 bytes at
            // either end are copied for nothing).  Runs closer than `gap`
            // slots are merged (the slots between are copied too); the gap
            // grows until the record holds the tile's ranges.
            const long long own_len = (long long)W.blk.size();
            uint32_t *R = &recs[(size_t)t * REC_WORDS];
            int nr = 0;
            long long bytes = 0, cursor = 0;  // bytes: staged so far
            auto add_range = [&](long long src, long long len, long long dst) {  // 16-byte units
                if (nr >= MAXR) return false;
                R[4 + 3 * nr] = (uint32_t)src;
                R[5 + 3 * nr] = (uint32_t)len;
                R[6 + 3 * nr] = (uint32_t)dst;
                ++nr;
                bytes += 16 * len;
                return true;
            };
            const long long cap_bytes = (long long)scap * NB;
            auto make_ranges = [&](long long gap, long long cap) {
                nr = 0;
                bytes = 0;
                bool fits = own_len == 0 || add_range(start[(size_t)t] * NB / 16, own_len * NB / 16, 0);
                cursor = own_len * NB;
                size_t i = 0;
                while (fits && i < need.size()) {
                    size_t j = i;
                    while (j + 1 < need.size() && need[j + 1].first - need[j].first <= gap) ++j;
                    const long long a = (long long)need[i].first * NB / 16 * 16;
                    const long long b = ((long long)(need[j].first + 1) * NB + 15) / 16 * 16;
                    if (b > nfp * NB || cursor + (b - a) > cap) return false;
                    for (size_t k = i; k <= j; ++k)
                        smap[(size_t)need[k].second] =
                            (uint16_t)((cursor + (long long)need[k].first * NB - a) / store_bytes);
                    fits = add_range(a / 16, (b - a) / 16, cursor / 16);
                    cursor += b - a;
                    i = j + 1;
                }
                return fits;
            };
            bool ok = false;
            for (long long gap = 1; !ok && gap <= 4 * (long long)nfp; gap *= 2) ok = make_ranges(gap, cap_bytes);
            // remember the padding (slots) under the tile's columns; where
            // the ranges overflow, take it at the smallest gap a record can
            // hold, and raise the reserve at least by one, so that the tile
            // narrows
            const long long base = own_len + (long long)need.size();
            auto pad_slots = [&]() { return (int)std::max<long long>(0, (cursor - base * NB + NB - 1) / NB); };
            int *pc = &padc[(size_t)(y0 / STY) * nx];
            if (!ok) {
                int padded = -1;
                for (long long gap = 1; padded < 0 && gap <= 4 * (long long)nfp; gap *= 2)
                    if (make_ranges(gap, 1LL << 40)) padded = pad_slots();
                const int seen = *std::max_element(pc + x0, pc + x0 + tl.w);
                const int need_pad = std::max(padded, seen + 1);
                if (tl.w <= 1 && base + need_pad > scap)
                    return fail(MCLBM_ERR_STATE, "fluid-only layout: a one-column tile exceeds the stage");
                for (int x = x0; x < x0 + tl.w; ++x) pc[x] = std::max(pc[x], need_pad);
                overflow = true;
                continue;
            }
            for (int x = x0; x < x0 + tl.w; ++x) pc[x] = std::max(pc[x], pad_slots());
            const long long words = words_of(W);
            if (words > tabcap || (int)own.size() > NT || cursor / store_bytes > 65535)
                return fail(MCLBM_ERR_STATE, "fluid-only layout: tile " + std::to_string(t) +
                                                 " exceeds the staging capacity");
            max_own = std::max(max_own, own_len);
            max_stage = std::max(max_stage, (cursor + NB - 1) / NB);
            R[0] = (uint32_t)nr;
            R[1] = (uint32_t)bytes;
            R[2] = (uint32_t)own_len;
            R[3] = (uint32_t)start[(size_t)t];
            std::vector<uint32_t> &T = tabs[(size_t)t];
            T.assign(HDR, 0);
            T[0] = (uint32_t)own.size();
            T[1] = (uint32_t)W.ring.size();
            T[2] = (uint32_t)W.sol.size();
            T[3] = 0;
            T[4] = (uint32_t)own_len;
            T[5] = (uint32_t)start[(size_t)t];
            T[6] = (uint32_t)x0;
            T[7] = (uint32_t)y0;
            T.insert(T.end(), own.begin(), own.end());
            T.insert(T.end(), W.ring.begin(), W.ring.end());
            T.insert(T.end(), W.sol.begin(), W.sol.end());
            for (size_t k = 0; k < smap.size(); k += 2)
                T.push_back((uint32_t)smap[k] | (k + 1 < smap.size() ? (uint32_t)smap[k + 1] << 16 : 0u));
            maxw = std::max(maxw, (int)T.size());
        }
        if (!overflow) break;
    }
    const int ntiles = (int)tiles.size();
    const int tab_words = (maxw + 3) / 4 * 4;
    if (tab_words > tabcap) return fail(MCLBM_ERR_STATE, "fluid-only layout: tables too large");
    out.tab.assign((size_t)ntiles * tab_words, 0);
    for (int t = 0; t < ntiles; ++t)
        std::copy(tabs[(size_t)t].begin(), tabs[(size_t)t].end(), out.tab.begin() + (size_t)t * tab_words);
    out.nfp = nfp;
    out.snode = std::move(snode);
    out.rec = std::move(recs);
    out.tab_words = tab_words;
    out.ntiles = ntiles;
    out.max_own = max_own;
    out.max_stage = max_stage;
    return MCLBM_OK;
}

// Host self-check of a layout against the geometry: every invariant the
// step kernel relies on.  Returns 0, 1 + the first failing tile, or -1
// (the blocks do not hold every fluid node exactly once).
int check_layout(const HostGeo &g, int STY, int planes, int store_bytes, const HostLayout &H, int scap, int tabcap) {
    const int nx = g.nx, ny = g.ny, NT = threads_for(STY);
    const int SFH = STY + 6, SN1 = SDXW * (STY + 4);
    std::vector<int> gidx((size_t)nx * ny, -1);
    for (long long k = 0; k < H.nfp; ++k) {
        const int n = H.snode[(size_t)k];
        if (n < 0) continue;
        if (n >= nx * ny || gidx[(size_t)n] >= 0 || g.at(n % nx, n / nx) != GEO_FLUID) return -1;
        gidx[(size_t)n] = (int)k;
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            if (g.at(x, y) == GEO_FLUID && gidx[(size_t)y * nx + x] < 0) return -1;
    auto wrapped = [&](int x, int y) {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        return gidx[(size_t)y * nx + x];
    };
    if (H.tab_words > tabcap || H.max_stage > scap) return 1;
    for (int t = 0; t < H.ntiles; ++t) {
        const uint32_t *T = &H.tab[(size_t)t * H.tab_words];
        const uint32_t *R = &H.rec[(size_t)t * REC_WORDS];
        const int n_own = (int)T[0], n_ring = (int)T[1], n_sol = (int)T[2];
        const long long own_len = T[4], start = T[5];
        const int x0 = (int)T[6], y0 = (int)T[7];
        if (n_own > NT || HDR + n_own + n_ring + n_sol + (SFW * SFH + 1) / 2 > H.tab_words) return t + 1;
        if ((long long)R[2] != own_len || (long long)R[3] != start) return t + 1;
        // the stage as the copies fill it: (destination, source, length) in
        // bytes, disjoint, within the stage and the population buffer
        const long long NB = (long long)planes * store_bytes;
        struct Rg {
            long long dst, src, len;
        };
        std::vector<Rg> rg;
        const int nr = (int)R[0];
        if (nr < 1 && own_len > 0) return t + 1;
        long long bytes = 0;
        for (int r = 0; r < nr; ++r) {
            const Rg q{16LL * R[6 + 3 * r], 16LL * R[4 + 3 * r], 16LL * R[5 + 3 * r]};
            if (q.src + q.len > H.nfp * NB || q.dst + q.len > (long long)scap * NB ||
                (r == 0 && own_len > 0 && (q.src != start * NB || q.dst != 0 || q.len != own_len * NB)))
                return t + 1;
            for (const Rg &o : rg)
                if (q.dst < o.dst + o.len && o.dst < q.dst + q.len) return t + 1;
            rg.push_back(q);
            bytes += q.len;
        }
        if ((long long)R[1] != bytes) return t + 1;
        const uint32_t *E = T + HDR;
        const uint16_t *smap = reinterpret_cast<const uint16_t *>(E + n_own + n_ring + n_sol);
        // global slot of the node staged at frame position fp (-1: none, or
        // not a whole node of one copy)
        auto slot_at = [&](int fp) -> long long {
            const long long eb = (long long)smap[fp] * store_bytes;
            if (eb % 4) return -1;
            for (const Rg &q : rg)
                if (eb >= q.dst && eb + NB <= q.dst + q.len) {
                    const long long gb = q.src + (eb - q.dst);
                    return gb % NB ? -1 : gb / NB;
                }
            return -1;
        };
        std::vector<uint8_t> kind((size_t)SN1, 0);  // 1 own, 2 ring, 3 non-fluid
        // pulls of the node at frame position fp, lattice (x, y): every
        // fluid source must be staged at its frame position
        auto nonfluid_mask = [&](int x, int y) {
            uint32_t m = 0;
            for (int i = 1; i < 9; ++i)
                if (g.at(x + ex(i), y + ey(i)) != GEO_FLUID) m |= 1u << (i - 1);
            return m;
        };
        auto pulls_ok = [&](int fp, int x, int y) {
            for (int i = 1; i < 9; ++i) {
                const int sx = x - ex(i), sy = y - ey(i);
                if (g.at(sx, sy) != GEO_FLUID) continue;  // bounce-back: the node's own populations
                const long long sl = slot_at(fp - ey(i) * SFW - ex(i));
                if (sl < 0 || sl != wrapped(sx, sy)) return false;
            }
            return true;
        };
        for (int k = 0; k < n_own; ++k) {
            const uint32_t me = E[k];
            const int tx = (int)(me & 63u), ty = (int)((me >> 6) & 63u), bidx = (int)(me >> 22);
            const int x = x0 + tx, y = y0 + ty;
            if (x >= nx || y >= ny || bidx >= own_len || H.snode[(size_t)(start + bidx)] != y * nx + x) return t + 1;
            const int fp = (ty + 3) * SFW + tx + 3, dp = (ty + 2) * SDXW + tx + 2;
            if (slot_at(fp) != start + bidx || !pulls_ok(fp, x, y) || kind[(size_t)dp] ||
                ((me >> 12) & 0xffu) != nonfluid_mask(x, y))
                return t + 1;
            kind[(size_t)dp] = 1;
        }
        for (int k = 0; k < n_ring; ++k) {
            const int pos = (int)(E[n_own + k] & 0xfffu);
            if (pos >= SN1 || kind[(size_t)pos]) return t + 1;
            const int dr = pos / SDXW, dc = pos % SDXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
            const int fp = (dr + 1) * SFW + dc + 1;
            if (g.at(x, y) != GEO_FLUID || slot_at(fp) != wrapped(x, y) || !pulls_ok(fp, x, y) ||
                ((E[n_own + k] >> 12) & 0xffu) != nonfluid_mask(x, y))
                return t + 1;
            kind[(size_t)pos] = 2;
        }
        for (int k = 0; k < n_sol; ++k) {
            const uint32_t e = E[n_own + n_ring + k];
            const int pos = (int)(e & 0xfffu);
            if (pos >= SN1 || kind[(size_t)pos]) return t + 1;
            const int dr = pos / SDXW, dc = pos % SDXW;
            if (g.at(x0 - 2 + dc, y0 - 2 + dr) == GEO_FLUID || (int)((e >> 12) & 0xffu) != g.at(x0 - 2 + dc, y0 - 2 + dr))
                return t + 1;
            kind[(size_t)pos] = 3;
        }
        // what phases B and C read: every neighbour of an own node has a
        // density (own or ring) or a virtual density (non-fluid entry); every
        // fluid neighbour of a non-fluid entry inside the lattice has one too
        for (int k = 0; k < n_own; ++k) {
            const uint32_t me = E[k];
            const int dp = ((int)((me >> 6) & 63u) + 2) * SDXW + (int)(me & 63u) + 2;
            for (int i = 1; i < 9; ++i)
                if (!kind[(size_t)(dp + ey(i) * SDXW + ex(i))]) return t + 1;
        }
        for (int k = 0; k < n_sol; ++k) {
            const uint32_t e = E[n_own + n_ring + k];
            const int pos = (int)(e & 0xfffu);
            if (((e >> 12) & 0xffu) == GEO_OUTSIDE) continue;
            for (int i = 1; i < 9; ++i) {
                const int dr = pos / SDXW + ey(i), dc = pos % SDXW + ex(i);
                const bool fluid = g.at(x0 - 2 + dc, y0 - 2 + dr) == GEO_FLUID;
                if (((e >> 20 >> (i - 1)) & 1u) != (fluid ? 1u : 0u)) return t + 1;
                if (fluid && (dr < 0 || dr >= STY + 4 || dc < 0 || dc >= SDXW ||
                              (kind[(size_t)(dr * SDXW + dc)] != 1 && kind[(size_t)(dr * SDXW + dc)] != 2)))
                    return t + 1;
            }
        }
    }
    return 0;
}

int sparse_build(Lattice &L, int STY) {
    if (L.nfp > 0 && L.sparse_ty != STY) {
        // another slot order: bring the state back to the dense buffers first
        if (int rc = sparse_to_dense(L)) return rc;
        L.sparse_state = 0;
        L.sparse_mode = -1;
    }
    const int nx = L.nx, ny = L.ny;
    const int node_bytes = L.planes * (int)L.store_bytes;
    const int Q = 16 / ((node_bytes & 15) ? (node_bytes & 15) : 16);  // slots per 16-byte multiple
    if ((Q * node_bytes) % 16) return MCLBM_OK;  // no 16-byte multiple of nodes: kernel 4 unavailable
    const int planes = L.planes;
    std::vector<uint8_t> pad((size_t)L.geo_pad_rows * L.gpitch);
    cudaError_t e = cudaMemcpyAsync(pad.data(), L.geo_pad, pad.size(), cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "geometry read-back (fluid-only layout)");
    std::vector<uint8_t> codes((size_t)(ny + 6) * (nx + 6));
    for (int y = -3; y < ny + 3; ++y)
        for (int x = -3; x < nx + 3; ++x) {
            const int r = y + HY, col = GEO_HX + x;
            const bool in = r >= 0 && r < L.geo_pad_rows && col >= 0 && col < L.gpitch;
            codes[(size_t)(y + 3) * (nx + 6) + (x + 3)] = in ? pad[(size_t)r * L.gpitch + col] : (uint8_t)GEO_OUTSIDE;
        }
    HostLayout H;
    if (int rc = build_layout(HostGeo{nx, ny, codes.data()}, STY, L.prec, planes, (int)L.store_bytes, Q,
                              L.p.open_x != 0, H))
        return rc;
    const long long nfp = H.nfp;
    const std::vector<int> &snode = H.snode;
    const std::vector<uint32_t> &flat = H.tab, &recs = H.rec;
    const int tab_words = H.tab_words, ntiles = H.ntiles;
    const long long max_own = H.max_own, max_stage = H.max_stage;

    // 3. device buffers (the populations only when the slot count changed)
    auto realloc = [&](void **p, size_t bytes) -> cudaError_t {
        cudaFree(*p);
        *p = nullptr;
        return cudaMalloc(p, bytes);
    };
    if (L.nfp != nfp || L.sparse_ty != STY) {
        for (int b = 0; b < 2 && e == cudaSuccess; ++b)
            e = realloc(&L.fs[b], (size_t)planes * nfp * L.store_bytes);
        if (e == cudaSuccess) e = realloc((void **)&L.snode, (size_t)nfp * sizeof(int));
        L.sparse_state = 0;
    }
    if (e == cudaSuccess) e = realloc((void **)&L.stab, flat.size() * 4);
    if (e == cudaSuccess) e = realloc((void **)&L.scopy, recs.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.snode, snode.data(), snode.size() * sizeof(int),
                                              cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.stab, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.scopy, recs.data(), recs.size() * 4, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        L.nfp = 0;
        return cuda_fail(e, "fluid-only layout buffers");
    }
    L.nfp = nfp;
    L.stab_words = tab_words;
    L.sparse_ty = STY;
    L.stiles = ntiles;
    L.socap = (int)max_own;
    L.sscap = (int)((max_stage + 15) / 16 * 16);
    L.sparse_mode = L.ghost_key();
    return MCLBM_OK;
}
}  // namespace

int sparse_layout_check(int nx, int ny, const uint8_t *codes, mclbm_precision prec, int tile_shape, bool open_x,
                        int64_t out[8]) {
    if (!sparse_precision(prec)) return fail(MCLBM_ERR_ARG, "the fluid-only kernel does not serve this precision");
    const int STY = tile_shape == 1 ? 16 : 12;
    const int planes = prec == MCLBM_FP32 ? 18 : 20, store_bytes = prec == MCLBM_FP32 ? 4 : 2;
    const int node_bytes = planes * store_bytes;
    const int Q = 16 / ((node_bytes & 15) ? (node_bytes & 15) : 16);
    const HostGeo g{nx, ny, codes};
    HostLayout H;
    if (int rc = build_layout(g, STY, prec, planes, store_bytes, Q, open_x, H)) return rc;
    const int scap = staged_capacity(prec, STY), tabcap = table_capacity(prec, STY);
    const long long sscap = (H.max_stage + 15) / 16 * 16;
    out[0] = H.ntiles;
    out[1] = H.nfp;
    out[2] = H.max_stage;
    out[3] = H.tab_words;
    out[4] = H.attempts;
    out[5] = H.max_own;
    out[6] = (int64_t)smem_bytes((int)sscap, node_bytes, H.tab_words, SDXW * (STY + 4));
    out[7] = check_layout(g, STY, planes, store_bytes, H, scap, tabcap);
    return MCLBM_OK;
}

void sparse_release(Lattice &L) {
    for (int b = 0; b < 2; ++b) {
        cudaFree(L.fs[b]);
        L.fs[b] = nullptr;
    }
    cudaFree(L.stab);
    cudaFree(L.scopy);
    cudaFree(L.snode);
    L.stab = nullptr;
    L.scopy = nullptr;
    L.snode = nullptr;
    L.nfp = 0;
}

int dense_to_sparse(Lattice &L) {
    if (L.sparse_state != 0) return MCLBM_OK;
    if (L.nfp <= 0) return fail(MCLBM_ERR_STATE, "the fluid-only layout is not prepared");
    const Geometry g = L.geometry();
    cudaError_t e = dispatch_prec(L.prec, [&](auto tag) {
        using P = decltype(tag);
        const long long n = L.nfp * P::planes;
        to_sparse_kernel<P><<<(unsigned)((n + 255) / 256), 256, 0, L.stream>>>(
            g, static_cast<const typename P::store_t *>(L.f[L.cur]), static_cast<typename P::store_t *>(L.fs[0]),
            L.snode, L.nfp);
        count_launch();
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return cuda_fail(e, "dense to fluid-only conversion");
    L.scur = 0;
    L.sparse_state = 2;
    return MCLBM_OK;
}

int sparse_to_dense(Lattice &L) {
    if (L.sparse_state != 1) return MCLBM_OK;
    const Geometry g = L.geometry();
    cudaError_t e = dispatch_prec(L.prec, [&](auto tag) {
        using P = decltype(tag);
        const long long n = L.nfp * P::planes;
        to_dense_kernel<P><<<(unsigned)((n + 255) / 256), 256, 0, L.stream>>>(
            g, static_cast<const typename P::store_t *>(L.fs[L.scur]), static_cast<typename P::store_t *>(L.f[L.cur]),
            L.snode, L.nfp);
        count_launch();
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return cuda_fail(e, "fluid-only to dense conversion");
    L.sparse_state = 2;
    L.pop_ghosts_stale = true;  // rebuilt before the next dense step
    return MCLBM_OK;
}

namespace {
// one launch advancing lattices cases[0..n) by one step (all share the
// precision, the tile height and have their fluid-only state current)
template <class P, int STY, int N, int CM>
cudaError_t launch_sparse(Lattice *const *cases, int n, int grid, cudaStream_t stream, int *slots_out) {
    using Lay = SLayout<P, STY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sparse_kernel<P, STY, N, CM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Lay::total);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    static SArgs<N> s;  // host staging of the parameter block
    std::memset(&s, 0, sizeof(s));
    int scap = 16, tabw = 4, total = 0;
    for (int c = 0; c < n; ++c) {
        Lattice &L = *cases[c];
        if (L.nfp <= 0 || L.sparse_ty != STY || L.sparse_state == 0) return cudaErrorInvalidValue;
        scap = std::max(scap, L.sscap);
        tabw = std::max(tabw, L.stab_words);
        s.a[c].g = L.geometry();
        s.a[c].p = L.p;
        s.a[c].p.round_fp32();
        s.a[c].d5 = L.d5;
        s.a[c].err = L.err;
        s.a[c].wait_ns = L.wait_ns;
        s.a[c].test_no_copy = L.test_no_copy;
        s.fin[c] = L.fs[L.scur];
        s.fout[c] = L.fs[1 - L.scur];
        s.tab[c] = L.stab;
        s.rec[c] = L.scopy;
        s.tab_words[c] = L.stab_words;
        s.first[c] = total;
        total += L.stiles;
    }
    s.first[n] = total;
    s.ncases = n;
    s.total = total;
    s.tab_stride = tabw;
    const size_t bytes = smem_layout<P, STY, N>(scap, tabw, s);
    if (bytes > Lay::total) return cudaErrorInvalidValue;
    // resident CTAs per SM for this size (cached per size)
    static size_t last_bytes = 0;
    static int slots = 0;
    if (bytes != last_bytes) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_kernel<P, STY, N, CM>, Lay::NT + 32, bytes);
        slots = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
        last_bytes = bytes;
    }
    if (slots_out) *slots_out = slots;
    const int g = grid > 0 ? std::min(grid, total) : std::min(slots, total);
    cudaError_t e;
    if (N == 1) {
        // one lattice: programmatic dependent launch (the kernel orders its
        // accesses with griddepcontrol), so that this step's grid starts
        // while the previous one drains
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)g);
        cfg.blockDim = dim3(Lay::NT + 32);  // NT compute threads and the producer warp
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, sparse_kernel<P, STY, N, CM>, s);
    } else {
        // NT compute threads and the producer warp
        sparse_kernel<P, STY, N, CM><<<g, Lay::NT + 32, bytes, stream>>>(s);
        e = cudaGetLastError();
    }
    count_launch();
    if (e == cudaSuccess)
        for (int c = 0; c < n; ++c) {
            cases[c]->scur = 1 - cases[c]->scur;
            cases[c]->sparse_state = 1;
        }
    return e;
}
}  // namespace

cudaError_t launch_step_sparse(Lattice &L) {
    Lattice *one = &L;
    return dispatch_prec(L.prec, [&](auto tag) {
        using P = decltype(tag);
        if (L.p.mrt)
            return L.sparse_ty == 12 ? launch_sparse<P, 12, 1, 1>(&one, 1, 0, L.stream, nullptr)
                                    : launch_sparse<P, 16, 1, 1>(&one, 1, 0, L.stream, nullptr);
        return L.sparse_ty == 12 ? launch_sparse<P, 12, 1, 0>(&one, 1, 0, L.stream, nullptr)
                                : launch_sparse<P, 16, 1, 0>(&one, 1, 0, L.stream, nullptr);
    });
}

cudaError_t launch_step_sparse_batch(Lattice *const *cases, int n, int grid, cudaStream_t stream) {
    if (n < 1 || n > MAX_BATCH) return cudaErrorInvalidValue;
    const int ty = cases[0]->sparse_ty;
    return dispatch_prec(cases[0]->prec, [&](auto tag) {
        using P = decltype(tag);
        return ty == 12 ? launch_sparse<P, 12, MAX_BATCH, 2>(cases, n, grid, stream, nullptr)
                       : launch_sparse<P, 16, MAX_BATCH, 2>(cases, n, grid, stream, nullptr);
    });
}

}  // namespace mclbm
