// Internal declarations of the CUDA library: D2Q9 constants, storage
// precisions, memory layout, the lattice object and the kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "mclbm.h"

namespace mclbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (Sec. 2.1).  Written as constexpr functions so that unrolled
// loops fold them into immediates.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <class R>
__host__ __device__ constexpr R wgt(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

// Geometry code of a node: 0 fluid, 1..254 solid with wettability-table
// index, 255 outside the domain (beyond a non-periodic edge).
constexpr uint8_t GEO_FLUID = 0;
constexpr uint8_t GEO_OUTSIDE = 255;
constexpr int MAX_XI_VALUES = 254;
// Geometry rows carry 16 ghost columns on each side; column x sits at byte
// GEO_HX + x of its row.
constexpr int GEO_HX = 16;

// ---------------------------------------------------------------------------
// Storage precisions.  Populations are stored as S and computed in R.  With
// REF the store holds, per node and component, a reference density rho_hat
// (the node's own density rounded to S) and the deviations
// d_i = f_i - w_i rho_hat from that rest equilibrium; f_i = w_i rho_hat + d_i.
// ---------------------------------------------------------------------------
template <class S, class R, bool REF>
struct Prec {
    using store_t = S;
    using real_t = R;
    static constexpr bool ref = REF;
    static constexpr int planes = REF ? 20 : 18;
    // ghost columns per side of a population row: at least 3 (the deepest
    // stencil reach) and a whole 16-byte chunk
    static constexpr int hx = sizeof(S) >= 4 ? 4 : 16 / (int)sizeof(S);
};
using P64 = Prec<double, double, false>;
using P32 = Prec<float, float, false>;
using P32D = Prec<float, float, true>;
using P16D = Prec<__half, float, true>;
using PB16D = Prec<__nv_bfloat16, float, true>;

__device__ __forceinline__ float to_real(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_real(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_real(float v) { return v; }
__device__ __forceinline__ double to_real(double v) { return v; }
template <class S> __device__ __forceinline__ S from_real(float v);
template <> __device__ __forceinline__ float from_real<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_real<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <class S> __device__ __forceinline__ S from_real(double v) { return (S)v; }

// ---------------------------------------------------------------------------
// Physical and boundary parameters of a lattice, passed by value to kernels.
// ---------------------------------------------------------------------------
struct Params {
    double nu1 = 1.0 / 6.0, nu2 = 1.0 / 6.0;
    double g_coh = 3.5, g_ads = 3.5;
    double gx = 0.0, gy = 0.0;
    double rho_in1 = -1.0, rho_out2 = -1.0;
    int open_x = 0;      // pressure boundaries on at x = 0 and x = nx-1
    int periodic_y = 0;  // else rows 0 and ny-1 must be solid
    int vel_shift = 1;   // u carries F/2
    int bc_set = 3;      // inlet/outlet treatment of Sec. 2.3: Set-1, -2 or -3
    double rho_in2 = 0.0, rho_out1 = 0.0;  // Set-1: the other component's densities
    int mrt = 0;         // 0: SRT collision of Eq. 1; 1: multiple-relaxation-time variant
    double s_e = 0.0, s_eps = 0.0, s_q = 0.0;  // MRT rates (0: 1/tau_s; s_q -1: 8(2-w)/(8-w))
    // the same values rounded to FP32 once on the host: the FP32 kernels
    // read these rather than converting from FP64 at every node (such a
    // conversion occupies the narrow FP64 pipe)
    float nu1_f = 0, nu2_f = 0, g_coh_f = 0, g_ads_f = 0, gx_f = 0, gy_f = 0;
    float rho_in1_f = 0, rho_out2_f = 0, rho_in2_f = 0, rho_out1_f = 0;
    float s_e_f = 0, s_eps_f = 0, s_q_f = 0;
    // G_ads / G_coh (0 where G_coh = 0), for the fluid-only step, which
    // stores the virtual solid densities scaled by it so that its force
    // stencil has one coupling for all 8 neighbours
    float ads_over_coh_f = 0;
    void round_fp32() {
        ads_over_coh_f = g_coh != 0 ? (float)(g_ads / g_coh) : 0.f;
        nu1_f = (float)nu1;
        nu2_f = (float)nu2;
        g_coh_f = (float)g_coh;
        g_ads_f = (float)g_ads;
        gx_f = (float)gx;
        gy_f = (float)gy;
        rho_in1_f = (float)rho_in1;
        rho_out2_f = (float)rho_out2;
        rho_in2_f = (float)rho_in2;
        rho_out1_f = (float)rho_out1;
        s_e_f = (float)s_e;
        s_eps_f = (float)s_eps;
        s_q_f = (float)s_q;
    }
};

// A parameter in the arithmetic type R: the FP64 value, or its FP32 copy.
template <class R> __device__ __forceinline__ R par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

// Memory layout shared by every kernel.  Population (c, i, y, x) lives at
// f[(c*9 + i) * plane + (y + HY) * pitch + hx + x]; columns -hx..-1 and
// nx..nx+hx-1 are ghost copies of the opposite edge when x is periodic, and
// rows -HY..-1 and ny..ny+HY-1 likewise when y is periodic, so that a tile
// and its 3-node ring are always one rectangular box.  Reference densities
// (REF precisions) are planes 18 and 19.  pitch and plane are odd multiples
// of 128 bytes so that the direction planes and rows do not alias in the
// caches.
constexpr int HY = 3;

struct Geometry {
    int nx, ny;
    int pitch;                 // population row stride, elements
    int hx;                    // column of x = 0 within a population row
    long long plane;           // population plane stride, elements (ny + 2 HY rows)
    int gpitch;                // geometry row stride, bytes
    const uint8_t *geo;        // [ny][gpitch], column x at GEO_HX + x
    const double *chi;         // [256][2] (1 + xi, 1 - xi) by code, in FP64
    const float *chi_f;        // the same table rounded to FP32
};

// wetting factor k of the chi table in the arithmetic type R
template <class R> __device__ __forceinline__ R chi_at(const Geometry &g, int k);
template <> __device__ __forceinline__ double chi_at<double>(const Geometry &g, int k) {
    return g.chi[k];
}
template <> __device__ __forceinline__ float chi_at<float>(const Geometry &g, int k) {
    return g.chi_f[k];
}

struct StepArgs {
    Geometry g;
    Params p;
    const void *fin;           // post-collision state of step t
    void *fout;                // post-collision state of step t+1
    const void *d5;            // [6][ny] (real type): component 1's outlet f_{3,6,7} (Eq. 26),
                               // component 2's inlet f_{1,5,8} (Eq. 27), frozen at initialisation
    int *err;                  // device error word (bounded waits)
    int rows_per_cta;          // strip kernel: rows of one CTA
    unsigned long long wait_ns = 1000000000ull;  // limit of every bounded wait of the staging kernels
    int test_no_copy = 0;      // test hook: the fluid-only kernel issues no staging copies
};

// strip width (columns per CTA) of the row-sweeping kernel
constexpr int SWEEP_W = 128;

// ---------------------------------------------------------------------------
// The lattice object behind the opaque handle of the C ABI.
// ---------------------------------------------------------------------------
struct Lattice {
    int nx = 0, ny = 0;
    int pitch = 0, hx = 0, gpitch = 0;
    long long plane = 0;
    int planes = 18;
    mclbm_precision prec = MCLBM_FP32;
    size_t store_bytes = 4;    // bytes per stored population
    size_t real_bytes = 4;     // bytes of the math type
    Params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    uint8_t *geo = nullptr;    // [ny][gpitch]
    uint8_t *geo_pad = nullptr;  // [geo_pad_rows][gpitch]: rows -HY.. of the geometry,
    int geo_pad_rows = 0;        // ghost rows per the y mode, outside beyond
    int ghost_mode = -1;       // boundary mode the ghosts were built for
    double *chi = nullptr;     // [256][2]
    float *chi_f = nullptr;    // [256][2], rounded to FP32
    void *f[2] = {nullptr, nullptr};  // ping-pong population buffers
    int cur = 0;               // index of the buffer holding the state
    void *d5 = nullptr;        // [6][ny] real type (see StepArgs::d5)
    int *err = nullptr;        // device error word
    double *diag_partial = nullptr;   // scratch of the diagnostics reduction
    int diag_blocks = 0;
    double *diag_out = nullptr;       // [8] device
    double *host_diag = nullptr;      // [8] pinned
    unsigned long long *bad_flag = nullptr;  // device: divergence count
    unsigned long long *blend_count = nullptr;  // device: nodes replaced by the last blend
    int64_t diag_every = 0;
    uint64_t wait_ns = 1000000000ull;  // bounded-wait limit of the staging kernels (1 s)
    int test_no_copy = 0;      // MCLBM_FLAG_TEST_NO_COPY
    int64_t kernel = 0;        // 0 auto, 1 tile kernel, 2 strip kernel
    int64_t steps = 0;
    size_t device_bytes = 0;
    bool boundary_rows_solid = false;
    bool initialised = false;
    void *tmaps = nullptr;     // host copies of the TMA descriptors (tile kernel), both shapes
    int tile_shape = 0;        // tile shape of the tile kernel (0 or 1)
    // work tables of the tile kernel, per tile shape: for every tile a
    // header and the packed entries of its fluid nodes, ring pulls and ring
    // solids; rebuilt with the ghosts whenever the boundary mode changes
    uint32_t *tab[2] = {nullptr, nullptr};
    int tab_words[2] = {0, 0};  // words copied per tile (largest table, 16-byte multiple)
    int *tab_max = nullptr;     // device scratch of the table build
    // fluid-only step (kernel 4): populations of the fluid nodes only, tile by
    // tile; the dense buffers stay the interchange format and the two are
    // converted lazily
    void *fs[2] = {nullptr, nullptr};  // [planes][nfp] each
    long long nfp = 0;                 // fluid slots (padded), 0 = kernel 4 unavailable
    int scur = 0;
    int sparse_state = 0;              // 0 dense current, 1 fluid-only current, 2 both
    bool pop_ghosts_stale = false;     // dense ghost copies need rebuilding
    int sparse_mode = -1;              // boundary mode the sparse tables were built for
    uint32_t *stab = nullptr;          // per-tile tables of kernel 4
    int stab_words = 0;                // words per tile table (stride and copy size)
    int socap = 0, sscap = 0;          // largest own block and staged set of any tile
    int sparse_ty = 0;                 // band height of the layout (12 or 16)
    int stiles = 0;                    // tiles of the layout
    int sparse_fail_key = -1;          // (boundary mode, band height) that could not be tiled
    uint32_t *scopy = nullptr;         // per-tile copy records of kernel 4
    int *snode = nullptr;              // [nfp]: lattice node y * nx + x of each slot, -1 padding
    uint64_t version = 0;      // bumped whenever a parameter changes
    int ghost_key() const { return p.open_x * 2 + p.periodic_y; }
    Geometry geometry() const {
        return Geometry{nx, ny, pitch, hx, plane, gpitch, geo, chi, chi_f};
    }
};

// status helpers (capi.cu)
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
void count_launch(int n = 1);
int lattice_prepare_step(Lattice &L);  // checks and ghost refresh before stepping (capi.cu)
int check_ready(Lattice &L);           // initialised, walls where y is not periodic
int refresh_ghosts(Lattice &L);        // ghosts and tables for the current boundary mode
int dense_current(Lattice &L);         // the dense buffers current, with their ghost copies

// launchers (step.cu, sweep.cu, fields.cu); return cudaError_t of the launch
cudaError_t launch_step_tile(Lattice &L, int tile_cfg);
cudaError_t launch_step_sweep(Lattice &L);
bool sweep_supported(const Lattice &L);
cudaError_t launch_step_tma(Lattice &L);
bool tma_supported(const Lattice &L);
int tma_prepare(Lattice &L);      // builds the TMA descriptors; MCLBM_OK or error
int tma_build_tables(Lattice &L); // work tables for the current boundary mode (synchronises)
// fluid-only step (sparse.cu)
bool sparse_precision(mclbm_precision p);
int sparse_prepare(Lattice &L, int band_height);  // layout and tables (bands of 12 or 16 rows)
// host only: build and check the layout of a geometry given as codes over
// [-3, nx + 3) x [-3, ny + 3) (capi: mclbm_fluid_layout_check)
int sparse_layout_check(int nx, int ny, const uint8_t *codes, mclbm_precision prec, int tile_shape, bool open_x,
                        int64_t out[8]);
cudaError_t launch_step_sparse(Lattice &L);
// one launch over several lattices (fluid-only state current, same tile height)
cudaError_t launch_step_sparse_batch(Lattice *const *cases, int n, int grid, cudaStream_t stream);
int sparse_to_dense(Lattice &L);      // make the dense buffers current (no-op if they are)
int dense_to_sparse(Lattice &L);      // make the fluid-only buffers current
void sparse_release(Lattice &L);
void tma_release(Lattice &L);
// batched persistent launch over several lattices (tma_tile.cu)
constexpr int MAX_BATCH = 32;
size_t tile_maps_bytes();         // bytes of the 4 descriptors of one lattice
int tile_maps_for(const Lattice &L, int shape, void *out);
cudaError_t launch_step_batch(Lattice *const *cases, int n, const void *maps, int shape, int grid,
                              cudaStream_t stream);
int batch_slots(mclbm_precision p, int shape);
cudaError_t launch_geo_ghosts(Lattice &L);
cudaError_t launch_init_equilibrium(Lattice &L, const double *rho1, const double *rho2);
cudaError_t launch_phase_densities(Lattice &L, const float *phi, double hi, double lo, double *r1,
                                   double *r2);
cudaError_t launch_blend_phase(Lattice &L, const float *phi, double hi, double lo, double flip,
                               unsigned long long *changed);
cudaError_t launch_set_populations(Lattice &L, const double *f);
cudaError_t launch_get_populations(Lattice &L, double *f);
cudaError_t launch_diagnostics(Lattice &L);
cudaError_t launch_density(Lattice &L, int comp, double *out);
cudaError_t launch_pressure(Lattice &L, double *out);
cudaError_t launch_phase(Lattice &L, float *out);
cudaError_t launch_velocity(Lattice &L, double *ux, double *uy, void *scratch);
size_t velocity_scratch_bytes(const Lattice &L);
int diag_blocks_for(const Lattice &L);

}  // namespace mclbm

// the opaque handle type of the C ABI is the lattice object itself
struct mclbm_lattice : public mclbm::Lattice {};
