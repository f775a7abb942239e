/*
 * mclbm.h - C ABI of the GB300 two-component pseudopotential lattice
 * Boltzmann library (improved multicomponent Shan-Chen model of Sedahmed,
 * Coelho and Warda, arXiv:2111.08666).
 *
 * The library advances a two-component D2Q9 lattice over a 2-D porous
 * medium: component densities and pseudopotentials, inter-component cohesion
 * (Eq. 13) and improved-virtual-solid-density adhesion (Eqs. 15-17), the
 * modified explicit-forcing BGK collision with a system relaxation time
 * (Eqs. 1, 2, 6, 8, 11), streaming with half-way bounce-back, and the Set-3
 * inlet/outlet pressure boundaries (Sec. 2.3, Eqs. 18-28).
 *
 * Conventions shared by every call:
 *  - Lattice arrays are row-major [ny][nx]; x is the flow direction, the
 *    inlet is column x = 0 and the outlet column x = nx-1.  Populations are
 *    [2][9][ny][nx]: component (0 = component 1, 1 = component 2), direction
 *    i of Sec. 2.1 (e_0..e_8 = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
 *    (-1,-1) (1,-1)), row, column.
 *  - Lattice units throughout (dx = dt = 1, c_s^2 = 1/3).
 *  - Every call returns MCLBM_OK (0) or a negative error code; on error
 *    mclbm_last_error() gives a message (thread-local, valid until the next
 *    failing call on the same thread).  No call throws or aborts.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Buffers
 *    the library fills may be host memory (pageable or pinned) or device
 *    memory; the library tells them apart with cudaPointerGetAttributes.
 *  - Work is enqueued on the lattice's CUDA stream.  mclbm_step returns
 *    before the GPU finishes; the read-outs synchronise that stream.
 *  - The library owns all device memory of a lattice and frees it in
 *    mclbm_destroy.  A lattice must not be used from two threads at once.
 */
#ifndef MCLBM_H
#define MCLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define MCLBM_OK 0
#define MCLBM_ERR_ARG (-1)      /* invalid argument (null, size, range) */
#define MCLBM_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define MCLBM_ERR_DIVERGED (-3) /* non-finite or negative density detected */
#define MCLBM_ERR_TIMEOUT (-4)  /* a bounded device-side wait ran out */
#define MCLBM_ERR_STATE (-5)    /* call not valid in the lattice's state */
#define MCLBM_ERR_NOMEM (-6)    /* device or host allocation failed */

/* Storage precision of the populations.  FP64 and FP32 store f_i.  The
 * deviation variants store, per node and component, a reference density
 * rho_hat (the node's density rounded to the storage type) and the
 * deviations f_i - w_i rho_hat from that rest equilibrium, in FP32, FP16 or
 * BF16, and compute in FP32.  Global reductions are FP64 in every variant. */
typedef enum {
    MCLBM_FP64 = 0,
    MCLBM_FP32 = 1,
    MCLBM_FP32_DEV = 2,
    MCLBM_FP16_DEV = 3,
    MCLBM_BF16_DEV = 4
} mclbm_precision;

/* Switches for mclbm_set_flag. */
typedef enum {
    /* 1: periodic in y.  0 (default): rows 0 and ny-1 must be solid walls. */
    MCLBM_FLAG_PERIODIC_Y = 0,
    /* 1 (default): the velocity in Eqs. 2 and 11 carries half the total
     * force, u = (sum_sigma sum_i e_i f_i + F/2) / rho, which the
     * (1 - 1/(2 tau_s)) prefactor of Eq. 1 needs for the momentum balance.
     * 0: the literal barycentric velocity of Eq. 8. */
    MCLBM_FLAG_VEL_SHIFT = 1,
    /* k > 0: every k steps mclbm_step runs the divergence check (non-finite
     * or negative density); a hit is reported by the next synchronising
     * call as MCLBM_ERR_DIVERGED.  0 (default): off. */
    MCLBM_FLAG_DIAG_EVERY = 2,
    /* Step kernel, all computing the same update: 0 (default) chooses 4
     * for FP32 and the 16-bit deviation storages, 3 for FP32 deviation
     * storage (or where 4 cannot stage a tile) and 1 for FP64; 1 the 2-D tile
     * kernel pulling straight from global memory; 2 the row-sweeping strip
     * kernel staging rows with bulk copies; 3 the 2-D tile kernel staging
     * the tile and its ring with one tensor copy (not for FP64); 4 the
     * fluid-only kernel: the populations of the fluid nodes only, tile by
     * tile, staged with bulk copies (FP32, FP16 and BF16 deviation storage;
     * the dense buffers are rebuilt whenever a read-out needs them). */
    MCLBM_FLAG_KERNEL = 3,
    /* Tile shape, same results either way.  Kernel 3: 0 (default) 32 x 16
     * nodes (32 x 12 for FP32_DEV), two CTAs per SM; 1: 32 x 8 nodes, three
     * CTAs per SM.  Kernel 4: bands of 12 rows (0, default; 256 compute
     * threads, three CTAs per SM) or 16 rows (1; 384 threads, two CTAs per
     * SM), cut into tiles of at most 32 columns and at most one fluid node
     * per compute thread (narrower where the staged tile would not fit). */
    MCLBM_FLAG_TILE_SHAPE = 4,
    /* Limit, in microseconds (1..10^7, default 10^6), of every wait of the
     * staging kernels (2, 3 and 4) for their asynchronous copies.  A wait
     * that runs out ends the launch and the next synchronising call returns
     * MCLBM_ERR_TIMEOUT; the lattice state is then not valid until it is
     * initialised again. */
    MCLBM_FLAG_WAIT_LIMIT_US = 5,
    /* Test hook, 0 by default: 1 makes kernel 4 issue no staging copies, so
     * that its first wait runs out and the step reports MCLBM_ERR_TIMEOUT.
     * It exercises the bounded-wait error path without a GPU fault. */
    MCLBM_FLAG_TEST_NO_COPY = 6
} mclbm_flag;

typedef struct mclbm_lattice mclbm_lattice;

/*
 * Create a lattice of nx * ny nodes (nx >= 3, ny >= 3).
 *   solid [ny][nx]  1 = solid node (phi = 1 of Eq. 16), 0 = fluid.
 *   xi    [ny][nx]  wettability parameter of Eq. 17 (chi^1 = 1 + xi,
 *                   chi^2 = 1 - xi), read at solid nodes only.  At most 254
 *                   distinct values over the solid nodes.  May be NULL
 *                   (xi = 0 everywhere, neutral wetting).
 *   prec            storage precision.
 *   cuda_stream     cudaStream_t to run on, or NULL for a stream the library
 *                   creates and owns.
 * Defaults: nu1 = nu2 = 1/6 (tau = 1), G_coh = G_ads = 3.5 (Sec. 2.1),
 * no body force, periodic x (no pressure boundaries), walls in y, velocity
 * shift on.  The populations start at zero: call mclbm_init_densities.
 */
int mclbm_create(int nx, int ny, const uint8_t *solid, const float *xi,
                 mclbm_precision prec, void *cuda_stream, mclbm_lattice **out);

/* Free the lattice and all its device memory.  NULL is accepted. */
int mclbm_destroy(mclbm_lattice *lat);

int mclbm_set_flag(mclbm_lattice *lat, int flag, int64_t value);

/* Kinematic viscosities of the components, Eq. 7 read as
 * nu = c_s^2 (tau - 1/2); they set the system relaxation time of Eq. 6. */
int mclbm_set_viscosity(mclbm_lattice *lat, double nu1, double nu2);

/* Cohesion strength G_coh (Eq. 13) and adhesion strength G_ads (Eq. 15);
 * the paper uses 3.5 for both (Sec. 2.2). */
int mclbm_set_coupling(mclbm_lattice *lat, double g_coh, double g_ads);

/* Body acceleration g: F^b,sigma = rho^sigma g (Eq. 12). */
int mclbm_set_body_force(mclbm_lattice *lat, double gx, double gy);

/* Pressure boundaries (Sec. 2.3): rho_in1 is the density of component 1
 * imposed at x = 0 (Eqs. 22-25), rho_out2 that of component 2 at x = nx-1
 * (Eqs. 18-21).  Either value < 0 switches the boundaries off and makes x
 * periodic.  The treatment of the other component at each end is chosen by
 * mclbm_set_bc (Set-3 by default). */
int mclbm_set_pressure_bc(mclbm_lattice *lat, double rho_in1, double rho_out2);

/* Inlet/outlet treatment of the other component (Sec. 2.3), in effect while
 * the pressure boundaries are on:
 *   bc_set 1 (Set-1): Zou-He for both components at both ends; component 2
 *            at x = 0 with density rho_in2 (Eqs. 22-25 with the component
 *            exchanged), component 1 at x = nx-1 with rho_out1 (Eqs. 18-21);
 *   bc_set 2 (Set-2): component 1's missing f_{3,6,7} at the outlet (Eq. 26)
 *            and component 2's missing f_{1,5,8} at the inlet (Eq. 27) keep
 *            the values they had at initialisation;
 *   bc_set 3 (Set-3, the paper's and the default): Eq. 26 at the outlet;
 *            at the inlet component 2 keeps its own post-collision
 *            f_{1,5,8} (Eq. 28).
 * rho_in2 and rho_out1 are read for Set-1 only.  The frozen values of Eqs.
 * 26-27 are recorded by every initialisation (mclbm_init_densities,
 * mclbm_init_from_phase, mclbm_set_populations).  Errors: MCLBM_ERR_ARG for
 * a set outside 1..3 or, with Set-1, densities that are not positive and
 * finite. */
int mclbm_set_bc(mclbm_lattice *lat, int bc_set, double rho_in2, double rho_out1);

/* Multiple-relaxation-time collision (not in the paper, which uses the SRT
 * of Eq. 1; offered for viscosity ratios beyond its runs).  on = 0 restores
 * Eq. 1.  With on = 1 the collision is
 *   f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M S^F
 * in the D2Q9 moment basis of Lallemand and Luo (rho, e, eps, j_x, q_x,
 * j_y, q_y, p_xx, p_xy), S = diag(-, s_e, s_eps, w, s_q, w, s_q, w, w) and
 * w = 1/tau_s from Eq. 6, f^eq of Eq. 2 and S^F of Eq. 11 with the same
 * velocity as the SRT.  Each rate lies in (0, 2), or is 0 for w (all three
 * 0: the SRT operator, up to rounding); s_q = -1 selects 8 (2 - w) / (8 - w),
 * which with s_e = s_eps = 0 makes half-way bounce-back exact for Poiseuille
 * flow at any tau.  Errors: MCLBM_ERR_ARG for a rate outside those values. */
int mclbm_set_mrt(mclbm_lattice *lat, int on, double s_e, double s_eps, double s_q);

/* The same boundaries given as pressures: Eq. 14 is inverted for the
 * majority density with the minority density held at 0.027 (the dissolved
 * density at G = 3.5, Sec. 3.2).  A negative pressure switches them off. */
int mclbm_set_pressure_bc_p(mclbm_lattice *lat, double p_in, double p_out);

/* Change the stream subsequent work is enqueued on (NULL: the library's
 * own stream). */
int mclbm_set_stream(mclbm_lattice *lat, void *cuda_stream);

/*
 * Initialise at rest from component densities rho1, rho2 [ny][nx] (host or
 * device, FP64): f_i = f_i^eq(rho^sigma, u = 0) of Eq. 2 on fluid nodes,
 * zero on solid nodes; the step counter restarts at 0.  The values taken by
 * component 1's f_3, f_6, f_7 on the outlet column are recorded as the
 * values Eq. 26 keeps there.
 */
int mclbm_init_densities(mclbm_lattice *lat, const double *rho1, const double *rho2);

/* Replace the post-collision populations by f [2][9][ny][nx] (FP64, host or
 * device).  Values on solid nodes are ignored.  Like mclbm_init_densities,
 * this records component 1's outlet f_3, f_6, f_7 for Eq. 26. */
int mclbm_set_populations(mclbm_lattice *lat, const double *f);

/* Copy the post-collision populations into f [2][9][ny][nx] (FP64, host or
 * device); zero on solid nodes.  Synchronises the stream. */
int mclbm_get_populations(mclbm_lattice *lat, double *f);

/*
 * Advance nsteps time steps of Eq. 1 with the fused kernel: pull streaming
 * with half-way bounce-back, Set-3 boundaries, moments (Eqs. 3-5), virtual
 * solid densities (Eqs. 16-17), forces (Eqs. 12-15 with the boundary-column
 * mirror of Sec. 2.1), system relaxation time and velocity (Eqs. 6-9), and
 * the forced BGK collision (Eqs. 1, 2, 11).  Asynchronous.  The fluid-only
 * kernel (4) launches each step as a programmatic dependent of the work
 * before it on the stream: its grid may start early, but it reads nothing
 * that earlier work writes (and writes nothing) until that work has
 * completed, so stream order holds for the caller's own kernels too.
 */
int mclbm_step(mclbm_lattice *lat, int64_t nsteps);

/* Wait for the lattice's stream; returns MCLBM_ERR_TIMEOUT if a bounded
 * wait inside the step kernel ran out (the state is then not valid), or
 * MCLBM_ERR_DIVERGED if the divergence check (MCLBM_FLAG_DIAG_EVERY) fired
 * since the last call. */
int mclbm_synchronize(mclbm_lattice *lat);

/* Component density rho^sigma (Eq. 3) of the current state, comp = 1 or 2,
 * into out [ny][nx] (FP64, host or device); zero on solid nodes. */
int mclbm_read_density(mclbm_lattice *lat, int comp, double *out);

/* Common velocity u = u^eq of the last collision (Eq. 9) into ux, uy
 * [ny][nx] (FP64, host or device); zero on solid nodes. */
int mclbm_read_velocity(mclbm_lattice *lat, double *ux, double *uy);

/* Pressure of Eq. 14, P = (rho1 + rho2)/3 + (G_coh/3) rho1 rho2, into
 * out [ny][nx] (FP64); zero on solid nodes. */
int mclbm_read_pressure(mclbm_lattice *lat, double *out);

/* Phase field (rho1 - rho2)/(rho1 + rho2) into out [ny][nx] (FP32); zero on
 * solid nodes. */
int mclbm_read_phase(mclbm_lattice *lat, float *out);

/*
 * All global diagnostics of the current state, reduced in FP64 (Sec. 4.2.1):
 *   out[0], out[1]  mass of component 1 and 2 over the fluid nodes
 *   out[2]          water saturation S_w by count: fluid nodes with
 *                   rho2 > rho1 over all fluid nodes
 *   out[3]          S_w by mass: sum rho2 / sum (rho1 + rho2)
 *   out[4], out[5]  P_in, P_out: mean of Eq. 14 over the fluid nodes of
 *                   column 0 (nx-1) more than 2 nodes in y from any solid
 *                   node of that column (NaN if there is none)
 *   out[6]          capillary pressure P_c = P_in - P_out
 *   out[7]          number of fluid nodes
 * out is host memory.  Synchronises the stream.
 */
int mclbm_diagnostics(mclbm_lattice *lat, double out[8]);

/* Conveniences over mclbm_diagnostics. */
int mclbm_saturation(mclbm_lattice *lat, double *sw_count, double *sw_mass);
int mclbm_capillary_pressure(mclbm_lattice *lat, double *pc, double *p_in, double *p_out);
int mclbm_mass(mclbm_lattice *lat, double out[2]);

/* Lattice facts: out[0] nx, out[1] ny, out[2] row pitch in elements,
 * out[3] precision, out[4] steps taken since initialisation, out[5] bytes
 * of device memory held. */
int mclbm_info(mclbm_lattice *lat, int64_t out[6]);

/*
 * mclbm_diagnostics without any allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc, or let a library call it
 * for them (a process whose device memory all comes from its own pool
 * allocator, a loop that must not allocate once running).
 *   f      [2][9][ny][nx] FP64 populations in device memory (the layout of
 *          mclbm_get_populations), owned by the caller
 *   solid  [ny][nx] uint8 in device memory, 1 = solid, owned by the caller
 *   g_coh  the cohesion strength that enters the boundary pressures, as in
 *          mclbm_diagnostics
 *   periodic_y  1 if rows wrap (affects which boundary nodes count as near
 *          a wall for P_in/P_out)
 *   out    [8] results as in mclbm_diagnostics, device or host memory
 *   cuda_stream  stream to run on (NULL: the legacy default stream)
 * The per-block partial sums live in a fixed array in the library's device
 * globals (64 KB per device, held until the process exits), which bounds the
 * lattice to at most 4194304 nodes; larger lattices are rejected with
 * MCLBM_ERR_ARG.  The caller guarantees the buffer sizes: f holds at least
 * 18 * nx * ny doubles, solid nx * ny bytes and out 8 doubles (the library
 * cannot check the extent of a raw pointer).  Allocates nothing.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so it should come before any stream capture.  All calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller.  With a device
 * output the call is asynchronous; with a host output it synchronises the
 * stream.
 */
int mclbm_diagnostics_noalloc(const double *f, const uint8_t *solid, int nx, int ny,
                              double g_coh, int periodic_y, double *out, void *cuda_stream);

/*
 * Batches: many independent lattices (porous-medium realisations or
 * wettability states of uneven sizes) advanced together, one persistent
 * launch per step over a work list of (lattice, tile) items, replayed from a
 * captured CUDA graph.  The paper runs one lattice at a time; batching is a
 * throughput feature of this library.  Every case computes exactly what
 * mclbm_step computes for it alone.
 */
typedef struct {
    int nx, ny;                 /* lattice size (as mclbm_create) */
    const uint8_t *solid;       /* [ny][nx] host, 1 = solid */
    const float *xi;            /* [ny][nx] host wettability, or NULL */
    double nu1, nu2;            /* viscosities (mclbm_set_viscosity) */
    double g_coh, g_ads;        /* coupling strengths (mclbm_set_coupling) */
    double gx, gy;              /* body acceleration */
    double rho_in1, rho_out2;   /* Set-3 densities; < 0: periodic x */
    int periodic_y;             /* 1: periodic y */
    const double *rho1, *rho2;  /* initial densities [ny][nx], or NULL */
} mclbm_case_desc;

typedef struct mclbm_batch mclbm_batch;

/* Create a batch of 1..32 cases in one storage precision (not FP64); the
 * library copies the host arrays.  cuda_stream as for mclbm_create. */
int mclbm_batch_create(int ncases, const mclbm_case_desc *cases, mclbm_precision prec,
                       void *cuda_stream, mclbm_batch **out);

/* Free the batch and all its lattices.  NULL is accepted. */
int mclbm_batch_destroy(mclbm_batch *b);

/* Borrow case k as a lattice handle for parameters and read-outs (valid
 * until the batch is destroyed; do not destroy it, and do not step it with
 * mclbm_step).  A parameter change makes the next batch step re-capture
 * its graph. */
int mclbm_batch_lattice(mclbm_batch *b, int k, mclbm_lattice **view);

/* Advance every case nsteps steps.  The first call times the candidate
 * kernels, tile shapes and grid sizes on its first steps (ordinary steps:
 * all candidates compute the same update, to rounding) and keeps the
 * fastest; steps then run in graph replays of 16 launches.  Asynchronous. */
int mclbm_batch_step(mclbm_batch *b, int64_t nsteps);

/* out[0] cases, out[1] total nodes, out[2] chosen step (0: tile kernel
 * 32 x 16 or 32 x 12, 1: tile kernel 32 x 8, 2: fluid-only kernel, 12-row
 * bands, 3: fluid-only kernel, 16-row bands; -1 not yet chosen), out[3] grid (0: one CTA
 * per resident slot, persistent; -1: one CTA per tile), out[4] steps per
 * graph replay, out[5] steps taken, out[6] resident CTA slots of the tile
 * kernel (0 for the fluid-only kernel), out[7] 1 if a graph is captured. */
int mclbm_batch_info(mclbm_batch *b, int64_t out[8]);

/* Milliseconds per step the tuner measured for its 6 candidates: the tile
 * kernel at shape 0 persistent, shape 0 one CTA per tile, shape 1
 * persistent, shape 1 one CTA per tile; the fluid-only kernel with bands of
 * 12 and of 16 rows (persistent).  -1 for a candidate not available. */
int mclbm_batch_tuning(mclbm_batch *b, double ms_per_step[6]);

/* Host only, no GPU needed: build the fluid-only layout of kernel 4 (its
 * tiles, slot blocks, work tables and copy records; Sec. 2.1 fixes what a
 * tile reads: pulls with half-way bounce-back, the 8-neighbour stencils of
 * Eqs. 12-15 and the weighted virtual densities of Eqs. 16-17) for a
 * geometry and check every invariant the step kernel relies on against it.
 * codes: (ny + 6) rows of nx + 6 bytes, row y + 3 and column x + 3 holding
 * the code of node (x, y) for x in [-3, nx + 3), y in [-3, ny + 3): 0
 * fluid, 255 outside the lattice, any other value a solid class (the ghost
 * rows and columns as the boundary mode makes them: copies of the opposite
 * edge where periodic).  Caller-owned, read only.  tile_shape as
 * MCLBM_FLAG_TILE_SHAPE; open_x marks the x ends open (Sec. 2.3).
 * out[0] tiles, out[1] fluid slots (padded), out[2] largest staged set
 * (slots), out[3] table words per tile, out[4] build attempts (a tile whose
 * padded copy ranges overflow the stage is narrowed and the layout
 * rebuilt), out[5] largest own block (slots), out[6] shared memory per CTA
 * (bytes), out[7] 0 if every check holds, 1 + the first failing tile, or
 * -1 if the blocks do not hold every fluid node exactly once.  Returns
 * MCLBM_ERR_ARG for a bad argument or a precision kernel 4 does not serve,
 * MCLBM_ERR_STATE if no tiling fits the staging capacity. */
int mclbm_fluid_layout_check(int nx, int ny, const uint8_t *codes, mclbm_precision prec, int tile_shape,
                             int open_x, int64_t out[8]);

/* Checkpoint: write the current state (populations as stored, the outlet
 * record of Eq. 26, the parameters and the step count) to a file, and read
 * it back into a lattice of the same size and precision; the restored run
 * continues bit for bit.  The file holds raw device bytes in this library
 * version's layout (same machine byte order). */
int mclbm_save(mclbm_lattice *lat, const char *path);
int mclbm_load(mclbm_lattice *lat, const char *path);

/* ------------------------------------------------------------------------
 * Learned warm start (an extension of the quasi-static protocol of
 * Sec. 4.2): a U-Net predicts the phase field of the next equilibrium.
 *
 * Network: levels L, base channels C0 (multiple of 32, at most 64),
 * C_l = C0 2^l.  Encoder level l: conv3x3 + ReLU twice = e_l, 2x2 average
 * pooling between levels.  Decoder level l = L-2..0: concat(e_l, nearest
 * 2x upsampling of d_(l+1)) with the skip first (d_(L-1) = e_(L-1)), conv3x3
 * + ReLU twice = d_l.  Head: 1x1 conv C0 -> 1, tanh.  Zero padding.
 *
 * Parameters: one flat FP32 vector in this order: enc0a, enc0b, ...,
 * enc(L-1)a, enc(L-1)b, dec(L-2)a, dec(L-2)b, ..., dec0a, dec0b, head; each
 * conv as weights [C_out][3][3][C_in] (head [1][1][1][C0]) then its bias
 * [C_out]; C_in of enc0a is 8 (channels 4..7 of the input are zero).
 *
 * Inputs x [B][H][W][4] (FP32, NHWC): solid indicator (1 solid, 0 fluid),
 * wettability xi (solid nodes, 0 elsewhere), current phase field
 * (rho1 - rho2)/(rho1 + rho2), pressure step.  Output phi [B][H][W] in
 * [-1, 1].  Loss: mean over the pixels with mask = 1 of (phi - target)^2.
 * H and W are multiples of 2^(L-1).  Arithmetic: BF16 operands on the
 * tensor cores with FP32 accumulation; FP32 master parameters and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * Buffers may be host or device memory.  Calls synchronise the network's
 * stream before returning.
 * ------------------------------------------------------------------------ */
typedef struct mclbm_unet mclbm_unet;

/* Network for batches up to max_batch of images up to max_h x max_w,
 * parameters zero until mclbm_unet_set_params.  cuda_stream NULL: own
 * stream.  Errors: MCLBM_ERR_ARG for levels outside 1..6, base not 32 or
 * 64 (or base 2^(levels-1) above 1024), sizes that are not positive
 * multiples of 2^(levels-1), or max_batch x max_h x max_w of 2^31 pixels or
 * more (pixel indices are 32-bit); MCLBM_ERR_NOMEM / MCLBM_ERR_CUDA when
 * the allocation fails. */
int mclbm_unet_create(int levels, int base, int max_batch, int max_h, int max_w, void *cuda_stream,
                      mclbm_unet **out);
int mclbm_unet_destroy(mclbm_unet *u);
int mclbm_unet_param_count(const mclbm_unet *u, int64_t *n);
/* Upper bound on the CTAs of the persistent row-tile kernels (convolution
 * and weight gradient, used for image widths that are multiples of 128); 0
 * (the default) sizes them to one wave of the GPU.  A small bound makes
 * every CTA walk many tiles, which lets a test cover the multi-tile
 * schedule on small images.  Results do not depend on it beyond the order
 * of the FP32 sums of the weight gradient.  Errors: MCLBM_ERR_ARG for a
 * NULL network or n < 0. */
int mclbm_unet_set_max_ctas(mclbm_unet *u, int n);
/* Weight-gradient kernel choice for image widths that are multiples of 128.
 * enable = 1 (the default): every layer takes the shared-tap kernel (the
 * nine taps of a 32-output-channel slice in one tensor-core product, dZ rows
 * kept in a ring down 128-pixel strips); enable = 0: every layer takes the
 * per-tap kernel (one product per tap).  The two give the same gradient up to the
 * order of the FP32 sums, which lets a test cross-check them.  Errors:
 * MCLBM_ERR_ARG for a NULL network or enable not 0 or 1. */
int mclbm_unet_set_shared_taps(mclbm_unet *u, int enable);
/* Copy the parameter vector in (resets the Adam moments) or out. */
int mclbm_unet_set_params(mclbm_unet *u, const float *theta);
int mclbm_unet_get_params(mclbm_unet *u, float *theta);
/* phi = network(x). */
int mclbm_unet_infer(mclbm_unet *u, int batch, int h, int w, const float *x, float *phi);
/* Loss and its gradient with respect to the parameters (no update); grad
 * may be NULL. */
int mclbm_unet_gradient(mclbm_unet *u, int batch, int h, int w, const float *x, const float *target,
                        const float *mask, double *loss, float *grad);
/* One Adam step with learning rate lr; *loss = the loss before the step. */
int mclbm_unet_train_step(mclbm_unet *u, int batch, int h, int w, const float *x, const float *target,
                          const float *mask, double lr, double *loss);

/* Initialise the lattice at rest from a phase field phi [ny][nx] (FP32,
 * host or device; read at fluid nodes): rho1 = rho_lo + (rho_hi -
 * rho_lo)(1 + phi)/2, rho2 = rho_lo + (rho_hi - rho_lo)(1 - phi)/2 with
 * rho_hi = 1 and rho_lo = 0.027 (the minority density of the separated
 * phases at G = 3.5, Sec. 3.1), phi clamped to [-1, 1]; then as
 * mclbm_init_densities. */
int mclbm_init_from_phase(mclbm_lattice *lat, const float *phi);

/*
 * Warm start in place (a quasi-static step of Sec. 4.2 started from a
 * predicted equilibrium): at every fluid node whose predicted phase field
 * phi_hat is on the other side of zero from the node's own phase (component
 * 1's side is rho1 > rho2) and |phi_hat| > flip, the populations are reset
 * to rest with the separated-phase densities of phi_hat, as in
 * mclbm_init_from_phase; every other node keeps its populations, and the
 * inlet/outlet records of Eqs. 26-27 are kept.
 *   phi_hat  [ny][nx] float, host or device, owned by the caller
 *   flip     in [0, 1)
 *   changed  receives the number of nodes reset (may be NULL)
 * The lattice must be initialised.  Synchronises the lattice's stream.
 */
int mclbm_blend_phase(mclbm_lattice *lat, const float *phi_hat, double flip, int64_t *changed);

/* Kernel launches enqueued by this library since it was loaded (all
 * lattices); used to count the GPU work inside a timed region. */
int64_t mclbm_launch_count(void);

const char *mclbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MCLBM_H */
