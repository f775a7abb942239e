// Fluid-only step (kernel 4): the populations of the fluid nodes only, so
// that a step reads and writes 2 x 9 x 2 populations per fluid node and no
// solid node costs memory traffic.
//
// Storage: fs[b] = [nfp][planes] (a node's populations contiguous, so that
// a range of nodes is one bulk copy), the fluid nodes tile by tile (TX x TY
// tiles in row-major order); inside a tile in border bands of width 3 --
// top-left corner, top edge, top-right corner, right edge, bottom-right
// corner, bottom edge, bottom-left corner, left edge -- then the interior,
// each band padded to a 16-byte multiple.  A neighbour's halo band is then
// one or two contiguous ranges of its block.
//
// Per tile, built on the host from the geometry and validated against every
// buffer bound before the kernel may run:
//   copy record  the ranges (source slot, length, destination slot) whose
//                bulk copies stage the tile's own block and the fluid nodes
//                of its 3-node ring, all planes, into shared memory
//   table        the work lists of the dense tile kernel (own nodes with
//                their block index, ring pulls, ring non-fluid nodes) and
//                the staged slot of every position of the staged frame
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

constexpr int STX = 32;                  // tile width; height 8 (shape 0) or 12 (shape 1)
constexpr int SFW = STX + 6;             // staged frame: tile + 3-node ring
constexpr int SDXW = STX + 4;            // density frame: tile + 2-node ring
constexpr int MAXR = 24;                 // ranges per tile (own block included)
constexpr int REC_WORDS = 4 + 3 * MAXR;  // copy record: n, bytes, own_len, start, ranges
constexpr int HDR = 8;                   // table header words
constexpr uint32_t SET3 = 3u << 20, IN_BIT = 1u << 20, OUT_BIT = 2u << 20;
static_assert((REC_WORDS * 4) % 16 == 0, "copy records are copied in 16-byte chunks");

template <class P, int STY>
struct SLayout {
    using S = typename P::store_t;
    using R = typename P::real_t;
    static constexpr int SFH = STY + 6, SN1 = SDXW * (STY + 4);
    static_assert(SFW * SFH < 65535, "frame positions are 16-bit");
    static constexpr int NPL = P::planes;
    // slots per 16-byte multiple (a node is NPL * sizeof(S) = 72 or 40 bytes)
    static constexpr int Q = 16 / ((NPL * (int)sizeof(S)) & 15 ? ((NPL * (int)sizeof(S)) & 15) : 16);
    static constexpr int OCAP = (STX * STY + 9 * (Q - 1) + Q - 1) / Q * Q;  // own block
    // staged slots: the own block, the ring's nodes (at most the staged
    // frame outside the tile) and the 16-byte rounding of every range
    static constexpr int SCAP = (OCAP + SFW * SFH - STX * STY + 2 * MAXR * (Q - 1) + 15) / 16 * 16;
    // table: header, own + ring + ring non-fluid entries (disjoint positions
    // of the density frame), then the staged slot of every frame position
    // (16 bits each)
    static constexpr int TABW = (HDR + SN1 + (SFW * SFH + 1) / 2 + 3) / 4 * 4;
    // two stages [slot][plane]: the tile being computed and the next one
    // in flight; a stage's own block also receives the tile's output
    static constexpr size_t stg_bytes = ((size_t)SCAP * NPL * sizeof(S) + 127) / 128 * 128;
    static constexpr size_t rho_off = 2 * stg_bytes;
    static constexpr size_t rho_bytes = (size_t)4 * SN1 * sizeof(R);  // two buffers of (rho1, rho2) pairs
    static constexpr size_t tab_off = (rho_off + rho_bytes + 127) / 128 * 128;  // two buffers
    static constexpr size_t tab_bytes = (size_t)2 * TABW * 4;
    static constexpr size_t rec_off = tab_off + tab_bytes;
    static constexpr size_t bar_off = (rec_off + REC_WORDS * 4 + 15) / 16 * 16;
    static constexpr size_t total = bar_off + 32;  // mbarriers full[2], done[2]
    static_assert(OCAP <= 1023, "own-block index is 10 bits");
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
    if (sty == 8) return p == MCLBM_FP32 ? SLayout<P32, 8>::TABW : SLayout<P16D, 8>::TABW;
    return p == MCLBM_FP32 ? SLayout<P32, 12>::TABW : SLayout<P16D, 12>::TABW;
}
int staged_capacity(mclbm_precision p, int sty) {
    if (sty == 8) return p == MCLBM_FP32 ? SLayout<P32, 8>::SCAP : SLayout<P16D, 8>::SCAP;
    return p == MCLBM_FP32 ? SLayout<P32, 12>::SCAP : SLayout<P16D, 12>::SCAP;
}

// The lattices of a launch (1, or up to MAX_BATCH for a batch).
template <int N>
struct SArgs {
    StepArgs a[N];
    const void *fin[N];  // [nfp][planes]
    void *fout[N];
    const uint32_t *tab[N];   // [tiles][tab_words]
    const uint32_t *rec[N];   // [tiles][REC_WORDS]
    int tab_words[N], tiles_x[N];
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
__global__ void __launch_bounds__(STX *STY + 32, STY == 8 ? 3 : 2) sparse_kernel(const __grid_constant__ SArgs<N> s) {
    using L = SLayout<P, STY>;
    constexpr int SN1 = L::SN1;
    using S = typename P::store_t;
    using R = typename P::real_t;
    constexpr int NT = STX * STY, NPL = L::NPL;
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
            const uint32_t src = rec[4 + 3 * r], len = rec[5 + 3 * r], dst = rec[6 + 3 * r];
            bulk_g2s(dst_stage + (size_t)dst * NPL, fin + (size_t)src * NPL, len * (uint32_t)(NPL * sizeof(S)),
                     &full[k]);
        }
        __syncwarp();
    };

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
    auto tile_xy = [&](int w, int &c, int &x0, int &y0) {
        c = case_of(w);
        const int t = w - s.first[c];
        x0 = (t % s.tiles_x[c]) * STX;
        y0 = (t / s.tiles_x[c]) * STY;
    };
    // A: pull + Set-3 + densities (Eq. 3) of tile w in stage k: the ring
    // entries from the last thread down, the own node of thread tid
    auto phase_a = [&](int w, int k, R f[2][9], R &rho1, R &rho2) {
        int c, x0, y0;
        tile_xy(w, c, x0, y0);
        const StepArgs &a = s.a[c];
        const S *stg = stage(k);
        float2 *rho = rho0 + k * SN1;
        const uint32_t *T = tabs + k * s.tab_stride;
        const int n_own = (int)T[0], n_ring = (int)T[1], n_sol = (int)T[2];
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
    // B: virtual solid densities (Eqs. 16-17) on the 1-ring (zero outside)
    auto phase_b = [&](int w, int k) {
        const Geometry &g = s.a[case_of(w)].g;
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
                const R inv = R(1) / den;
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
            if (me & SET3) {
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
int sparse_prepare(Lattice &L, int STY) {
    if (!sparse_precision(L.prec) || !L.geo_pad) return MCLBM_OK;  // kernel 4 unavailable
    if (L.sparse_mode == L.ghost_key() && L.nfp > 0 && L.sparse_ty == STY) return MCLBM_OK;
    if (L.nfp > 0 && L.sparse_ty != STY) {
        // another slot order: bring the state back to the dense buffers first
        if (int rc = sparse_to_dense(L)) return rc;
        L.sparse_state = 0;
        L.sparse_mode = -1;
    }
    const int SFH = STY + 6, SN1 = SDXW * (STY + 4);
    const int nx = L.nx, ny = L.ny;
    const int node_bytes = L.planes * (int)L.store_bytes;
    const int Q = 16 / ((node_bytes & 15) ? (node_bytes & 15) : 16);  // slots per 16-byte multiple
    if ((Q * node_bytes) % 16) return MCLBM_OK;  // no 16-byte multiple of nodes: kernel 4 unavailable
    const int planes = L.planes;
    std::vector<uint8_t> pad((size_t)L.geo_pad_rows * L.gpitch);
    cudaError_t e = cudaMemcpyAsync(pad.data(), L.geo_pad, pad.size(), cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "geometry read-back (fluid-only layout)");
    // the geometry as the step sees it (ghosts per the boundary mode), up to
    // 3 nodes past an edge: the step's reach (own nodes need forces from the
    // 1-ring, virtual solid densities from the 2-ring, pulls from the 3-ring)
    auto code_at = [&](int x, int y) -> int {
        if (x < -3 || x >= nx + 3 || y < -3 || y >= ny + 3) return GEO_OUTSIDE;
        const int r = y + HY, col = GEO_HX + x;
        if (r < 0 || r >= L.geo_pad_rows || col < 0 || col >= L.gpitch) return GEO_OUTSIDE;
        return pad[(size_t)r * L.gpitch + col];
    };
    const int tiles_x = (nx + STX - 1) / STX, tiles_y = (ny + STY - 1) / STY;
    const int ntiles = tiles_x * tiles_y;
    const bool open_x = L.p.open_x != 0;

    // 1. blocks: own fluid nodes of every tile in band order, bands padded
    std::vector<long long> start(ntiles + 1, 0);
    std::vector<std::vector<int>> blk(ntiles);  // node y*nx+x per slot, -1 padding
    // bands against the tile's extent inside the lattice (ragged edge tiles
    // are narrower), so that what a neighbour stages stays contiguous
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
    for (int t = 0; t < ntiles; ++t) {
        const int x0 = (t % tiles_x) * STX, y0 = (t / tiles_x) * STY;
        std::vector<int> &B = blk[t];
        const int tw = std::min(STX, nx - x0), th = std::min(STY, ny - y0);
        for (int bnd = 0; bnd < 9; ++bnd) {
            for (int ty = 0; ty < th; ++ty)
                for (int tx = 0; tx < tw; ++tx) {
                    const int x = x0 + tx, y = y0 + ty;
                    if (band(tx, ty, tw, th) != bnd) continue;
                    if (code_at(x, y) == GEO_FLUID) B.push_back(y * nx + x);
                }
            while (B.size() % Q) B.push_back(-1);
        }
        start[t + 1] = start[t] + (long long)B.size();
    }
    const long long nfp = std::max<long long>(start[ntiles], Q);
    if (nfp >= (1LL << 31)) return fail(MCLBM_ERR_ARG, "lattice too large for the fluid-only layout");
    std::vector<int> gidx((size_t)nx * ny, -1), snode((size_t)nfp, -1), bpos((size_t)nx * ny, -1);
    for (int t = 0; t < ntiles; ++t)
        for (size_t i = 0; i < blk[t].size(); ++i) {
            const int n = blk[t][i];
            snode[(size_t)(start[t] + (long long)i)] = n;
            if (n >= 0) {
                gidx[n] = (int)(start[t] + (long long)i);
                bpos[n] = (int)i;
            }
        }
    auto src_of = [&](int x, int y) -> int {  // slot of lattice position (x, y), wrapped
        if (x < 0 || x >= nx) x = ((x % nx) + nx) % nx;
        if (y < 0 || y >= ny) y = ((y % ny) + ny) % ny;
        return gidx[(size_t)y * nx + x];
    };
    auto fluid_mask = [&](int x, int y) {
        uint32_t m = 0;
        for (int i = 1; i < 9; ++i)
            if (code_at(x + ex(i), y + ey(i)) == GEO_FLUID) m |= 1u << (i - 1);
        return m;
    };
    auto set3 = [&](int x) -> uint32_t {
        return (open_x && x == 0 ? IN_BIT : 0u) | (open_x && x == nx - 1 ? OUT_BIT : 0u);
    };

    // 2. tables and copy records
    const int tabcap = table_capacity(L.prec, STY), scap = staged_capacity(L.prec, STY);
    std::vector<std::vector<uint32_t>> tabs(ntiles);
    std::vector<uint32_t> recs((size_t)ntiles * REC_WORDS, 0);
    int maxw = HDR;
    long long max_own = Q, max_stage = Q;
    for (int t = 0; t < ntiles; ++t) {
        const int x0 = (t % tiles_x) * STX, y0 = (t / tiles_x) * STY;
        std::vector<uint32_t> own, ring, sol;
        std::vector<uint16_t> smap((size_t)SFW * SFH, 0);
        // Only what the tile's own nodes read is computed: the densities or
        // virtual solid densities of their 8 neighbours (forces, Eqs. 12-15;
        // the open-end mirror reads the opposite neighbour, also one of the
        // 8), the fluid neighbours of those solid neighbours (Eq. 17), and
        // the populations those densities pull.  Positions of the density
        // frame: own (1), neighbour of an own node (2), density needed (4).
        std::vector<uint8_t> mark((size_t)SN1, 0);
        auto dpos = [&](int x, int y) { return (y - y0 + 2) * SDXW + (x - x0 + 2); };
        for (size_t i = 0; i < blk[t].size(); ++i) {
            const int n = blk[t][i];
            if (n < 0) continue;
            const int x = n % nx, y = n / nx;
            own.push_back((uint32_t)(x - x0) | (uint32_t)(y - y0) << 6 | (~fluid_mask(x, y) & 0xffu) << 12 |
                          set3(x) | (uint32_t)i << 22);
            smap[(size_t)(y - y0 + 3) * SFW + (x - x0 + 3)] = (uint16_t)(i * planes);
            mark[(size_t)dpos(x, y)] |= 1;
            for (int d = 1; d < 9; ++d) mark[(size_t)dpos(x + ex(d), y + ey(d))] |= 2;
        }
        for (int k = 0; k < SN1; ++k) {
            const int dr = k / SDXW, dc = k % SDXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
            if (!(mark[k] & 2)) continue;
            const int c = code_at(x, y);
            if (c == GEO_FLUID) {
                mark[k] |= 4;
                continue;
            }
            const uint32_t fm = fluid_mask(x, y);
            sol.push_back((uint32_t)k | (uint32_t)c << 12 | fm << 20);
            if (c == GEO_OUTSIDE) continue;  // zero: its neighbours are not read
            for (int d = 1; d < 9; ++d)
                if ((fm >> (d - 1)) & 1u) mark[(size_t)(k + ey(d) * SDXW + ex(d))] |= 4;
        }
        // the ring's densities, and the staged frame positions they and the
        // own nodes pull from (fluid sources outside the tile's own block)
        std::vector<uint8_t> pulled((size_t)SFW * SFH, 0);
        auto mark_sources = [&](int x, int y) {
            for (int d = 1; d < 9; ++d) {
                const int sx = x - ex(d), sy = y - ey(d);
                if (code_at(sx, sy) == GEO_FLUID) pulled[(size_t)(sy - y0 + 3) * SFW + (sx - x0 + 3)] = 1;
            }
        };
        for (int k = 0; k < SN1; ++k) {
            const int dr = k / SDXW, dc = k % SDXW, x = x0 - 2 + dc, y = y0 - 2 + dr;
            if (mark[k] & 1) {
                mark_sources(x, y);
                continue;
            }
            if (!(mark[k] & 4)) continue;
            ring.push_back((uint32_t)k | (~fluid_mask(x, y) & 0xffu) << 12 | set3(x));
            mark_sources(x, y);
        }
        // ring nodes to stage: pulled fluid positions outside the own block
        std::vector<std::pair<int, int>> need;  // (slot, frame position)
        for (int r = 0; r < SFH; ++r)
            for (int c = 0; c < SFW; ++c) {
                const int x = x0 - 3 + c, y = y0 - 3 + r;
                const bool in_tile = x >= x0 && x < x0 + STX && y >= y0 && y < y0 + STY && x < nx && y < ny;
                if (in_tile || !pulled[(size_t)r * SFW + c]) continue;
                const int gsl = src_of(x, y);
                if (gsl < 0) return fail(MCLBM_ERR_STATE, "fluid-only layout: ring node without a slot");
                need.push_back({gsl, r * SFW + c});
            }
        std::sort(need.begin(), need.end());
        // ranges: the own block first, then runs of the ring's slots.  Runs
        // closer than `gap` slots are merged (the slots between are copied
        // too); the gap grows until the record holds the tile's ranges.
        const long long own_len = (long long)blk[t].size();
        uint32_t *R = &recs[(size_t)t * REC_WORDS];
        int nr = 0;
        long long bytes = 0, cursor = 0;
        auto add_range = [&](long long src, long long len, long long dst) {
            if (nr >= MAXR) return false;
            R[4 + 3 * nr] = (uint32_t)src;
            R[5 + 3 * nr] = (uint32_t)len;
            R[6 + 3 * nr] = (uint32_t)dst;
            ++nr;
            bytes += len * planes * (long long)L.store_bytes;
            return true;
        };
        bool ok = false;
        for (long long gap = Q; !ok && gap <= 4 * (long long)nfp; gap *= 2) {
            nr = 0;
            bytes = 0;
            ok = own_len == 0 || add_range(start[t], own_len, 0);
            cursor = own_len;
            size_t i = 0;
            while (ok && i < need.size()) {
                const long long a = need[i].first / Q * Q;
                size_t j = i;
                while (j + 1 < need.size() && need[j + 1].first - need[j].first <= gap) ++j;
                const long long b = (need[j].first / Q + 1) * Q;  // exclusive, 16-byte multiple
                if (b > nfp || cursor + (b - a) > scap) {
                    ok = false;
                    break;
                }
                for (size_t k = i; k <= j; ++k)
                    smap[(size_t)need[k].second] = (uint16_t)((cursor + need[k].first - a) * planes);
                ok = add_range(a, b - a, cursor);
                cursor += b - a;
                i = j + 1;
            }
        }
        const long long words = HDR + (long long)own.size() + ring.size() + sol.size() + (smap.size() + 1) / 2;
        if (!ok || words > tabcap || own.size() > (size_t)STX * STY || cursor * planes > 65535)
            return fail(MCLBM_ERR_STATE, "fluid-only layout: tile " + std::to_string(t) +
                                             " exceeds the staging capacity");
        max_own = std::max(max_own, own_len);
        max_stage = std::max(max_stage, cursor);
        R[0] = (uint32_t)nr;
        R[1] = (uint32_t)bytes;
        R[2] = (uint32_t)own_len;
        R[3] = (uint32_t)start[t];
        std::vector<uint32_t> &T = tabs[t];
        T.assign(HDR, 0);
        T[0] = (uint32_t)own.size();
        T[1] = (uint32_t)ring.size();
        T[2] = (uint32_t)sol.size();
        T[3] = 0;
        T[4] = (uint32_t)own_len;
        T[5] = (uint32_t)start[t];
        T.insert(T.end(), own.begin(), own.end());
        T.insert(T.end(), ring.begin(), ring.end());
        T.insert(T.end(), sol.begin(), sol.end());
        for (size_t k = 0; k < smap.size(); k += 2)
            T.push_back((uint32_t)smap[k] | (k + 1 < smap.size() ? (uint32_t)smap[k + 1] << 16 : 0u));
        maxw = std::max(maxw, (int)T.size());
    }
    const int tab_words = (maxw + 3) / 4 * 4;
    if (tab_words > tabcap) return fail(MCLBM_ERR_STATE, "fluid-only layout: tables too large");
    std::vector<uint32_t> flat((size_t)ntiles * tab_words, 0);
    for (int t = 0; t < ntiles; ++t) std::copy(tabs[t].begin(), tabs[t].end(), flat.begin() + (size_t)t * tab_words);

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
    L.socap = (int)max_own;
    L.sscap = (int)((max_stage + 15) / 16 * 16);
    L.sparse_mode = L.ghost_key();
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
        s.tiles_x[c] = (L.nx + STX - 1) / STX;
        s.first[c] = total;
        total += s.tiles_x[c] * ((L.ny + STY - 1) / STY);
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_kernel<P, STY, N, CM>, STX * STY + 32, bytes);
        slots = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
        last_bytes = bytes;
    }
    if (slots_out) *slots_out = slots;
    const int g = grid > 0 ? std::min(grid, total) : std::min(slots, total);
    // STX * STY compute threads and the producer warp
    sparse_kernel<P, STY, N, CM><<<g, STX * STY + 32, bytes, stream>>>(s);
    count_launch();
    cudaError_t e = cudaGetLastError();
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
            return L.sparse_ty == 8 ? launch_sparse<P, 8, 1, 1>(&one, 1, 0, L.stream, nullptr)
                                    : launch_sparse<P, 12, 1, 1>(&one, 1, 0, L.stream, nullptr);
        return L.sparse_ty == 8 ? launch_sparse<P, 8, 1, 0>(&one, 1, 0, L.stream, nullptr)
                                : launch_sparse<P, 12, 1, 0>(&one, 1, 0, L.stream, nullptr);
    });
}

cudaError_t launch_step_sparse_batch(Lattice *const *cases, int n, int grid, cudaStream_t stream) {
    if (n < 1 || n > MAX_BATCH) return cudaErrorInvalidValue;
    const int ty = cases[0]->sparse_ty;
    return dispatch_prec(cases[0]->prec, [&](auto tag) {
        using P = decltype(tag);
        return ty == 8 ? launch_sparse<P, 8, MAX_BATCH, 2>(cases, n, grid, stream, nullptr)
                       : launch_sparse<P, 12, MAX_BATCH, 2>(cases, n, grid, stream, nullptr);
    });
}

}  // namespace mclbm
