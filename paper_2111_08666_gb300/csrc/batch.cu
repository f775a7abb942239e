// Batched stepping of many independent lattices (porous-medium realisations
// or wettability states of uneven sizes) in one persistent launch per step,
// replayed from a captured CUDA graph, with the tile shape and the grid
// chosen by timing the candidates on the batch itself.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.cuh"

using namespace mclbm;

constexpr int NCAND = 6;

struct mclbm_batch {
    std::vector<mclbm_lattice *> cases;
    mclbm_precision prec = MCLBM_FP32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<unsigned char> maps[2];  // tensor descriptors per tile shape
    // chosen step (-1: not tuned yet): 0-3 the dense tile kernel (tile shape
    // 0 or 1, persistent or one CTA per tile), 4-5 the fluid-only kernel
    // (bands of 12 or 16 rows, persistent)
    int cand = -1;
    double tune_ms[NCAND] = {0, 0, 0, 0, 0, 0};
    cudaGraphExec_t graph = nullptr;
    int graph_parity = 0;
    uint64_t graph_version = ~0ull;
    int64_t steps = 0;
    int64_t total_nodes = 0;
};

namespace {

constexpr int GRAPH_STEPS = 16;  // even, so a replay leaves the buffer parity unchanged

uint64_t version_of(const mclbm_batch &b) {
    uint64_t v = 0;
    for (auto *L : b.cases) v = v * 1000003ull + L->version * 31ull + (uint64_t)L->ghost_key();
    return v;
}

bool fluid_cand(int cand) { return cand >= 4; }
int shape_of_cand(int cand) { return fluid_cand(cand) ? cand - 4 : cand / 2; }
int grid_of_cand(int cand) { return !fluid_cand(cand) && cand % 2 ? 1 << 30 : 0; }

// bring every case to the layout the step of candidate cand works on
int ensure_layout(mclbm_batch &b, int cand) {
    for (auto *L : b.cases) {
        if (fluid_cand(cand)) {
            if (int rc = sparse_prepare(*L, shape_of_cand(cand) == 1 ? 16 : 12)) return rc;
            if (L->nfp <= 0) return fail(MCLBM_ERR_STATE, "fluid-only layout unavailable for a case");
            if (int rc = dense_to_sparse(*L)) return rc;
        } else {
            if (int rc = dense_current(*L)) return rc;
        }
    }
    return MCLBM_OK;
}

int parity_of(const mclbm_batch &b, int cand) {
    return fluid_cand(cand) ? b.cases[0]->scur : b.cases[0]->cur;
}

// the launch of one step (layout already current)
cudaError_t launch_cand(mclbm_batch &b, int cand) {
    std::vector<Lattice *> ls(b.cases.begin(), b.cases.end());
    if (fluid_cand(cand)) return launch_step_sparse_batch(ls.data(), (int)ls.size(), 0, b.stream);
    const int shape = shape_of_cand(cand);
    cudaError_t e = launch_step_batch(ls.data(), (int)ls.size(), b.maps[shape].data(), shape,
                                      grid_of_cand(cand), b.stream);
    if (e == cudaSuccess)
        for (auto *L : b.cases) L->sparse_state = 0;
    return e;
}

int direct_step(mclbm_batch &b, int cand) {
    if (int rc = ensure_layout(b, cand)) return rc;
    cudaError_t e = launch_cand(b, cand);
    if (e != cudaSuccess) return cuda_fail(e, "batched step kernel");
    for (auto *L : b.cases) ++L->steps;
    ++b.steps;
    return MCLBM_OK;
}

void drop_graph(mclbm_batch &b) {
    if (b.graph) cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
}

// Time every candidate on a few real steps of the batch and keep the
// fastest.  The candidates compute the same update (to rounding), so the
// trial steps are ordinary steps of the simulation.  Returns steps used.
int autotune(mclbm_batch &b, int64_t budget, int *rc) {
    *rc = MCLBM_OK;
    const int reps = 4;  // timed steps per candidate (2 picked unevenly from run to run)
    if (budget < (int64_t)NCAND * (reps + 1)) {
        b.cand = 0;
        return 0;
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    int used = 0;
    double best = 1e300;
    for (int c = 0; c < NCAND && *rc == MCLBM_OK; ++c) {
        if (fluid_cand(c) && !sparse_precision(b.prec)) {
            b.tune_ms[c] = -1;
            continue;
        }
        if ((*rc = direct_step(b, c))) {  // warm-up (and layout conversion)
            if (fluid_cand(c)) {          // a geometry the fluid-only kernel cannot stage
                *rc = MCLBM_OK;
                b.tune_ms[c] = -1;
                continue;
            }
            break;
        }
        ++used;
        cudaEventRecord(t0, b.stream);
        for (int r = 0; r < reps && *rc == MCLBM_OK; ++r) {
            *rc = direct_step(b, c);
            ++used;
        }
        cudaEventRecord(t1, b.stream);
        cudaEventSynchronize(t1);
        float ms = 0;
        cudaEventElapsedTime(&ms, t0, t1);
        b.tune_ms[c] = ms / reps;
        if (ms < best) {
            best = ms;
            b.cand = c;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (b.cand < 0) b.cand = 0;
    return used;
}

int capture_graph(mclbm_batch &b) {
    drop_graph(b);
    if (int rc = ensure_layout(b, b.cand)) return rc;  // conversions are not captured
    const int64_t launches0 = mclbm_launch_count();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const int parity = parity_of(b, b.cand);
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < GRAPH_STEPS && le == cudaSuccess; ++s) le = launch_cand(b, b.cand);
    e = cudaStreamEndCapture(b.stream, &g);
    // the captured launches ran nothing yet: undo their bookkeeping
    count_launch((int)(launches0 - mclbm_launch_count()));
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        for (auto *L : b.cases) {
            if (fluid_cand(b.cand)) L->scur = parity;
            else L->cur = parity;
        }
        return cuda_fail(le != cudaSuccess ? le : e, "graph capture of the batched step");
    }
    e = cudaGraphInstantiate(&b.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b.graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    b.graph_parity = parity;
    b.graph_version = version_of(b);
    return MCLBM_OK;
}

void destroy_batch(mclbm_batch *b) {
    if (!b) return;
    drop_graph(*b);
    for (auto *L : b->cases) mclbm_destroy(L);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

int mclbm_batch_create(int ncases, const mclbm_case_desc *cases, mclbm_precision prec,
                       void *cuda_stream, mclbm_batch **out) {
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ncases < 1 || ncases > MAX_BATCH)
        return fail(MCLBM_ERR_ARG, "ncases must be 1.." + std::to_string(MAX_BATCH));
    if (!cases) return fail(MCLBM_ERR_ARG, "cases is NULL");
    if (prec == MCLBM_FP64) return fail(MCLBM_ERR_ARG, "the batched kernel has no FP64 variant");
    mclbm_batch *b = new (std::nothrow) mclbm_batch();
    if (!b) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    b->prec = prec;
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "cudaStreamCreate");
        }
        b->own_stream = true;
    }
    for (int k = 0; k < ncases; ++k) {
        const mclbm_case_desc &d = cases[k];
        mclbm_lattice *L = nullptr;
        int rc = mclbm_create(d.nx, d.ny, d.solid, d.xi, prec, b->stream, &L);
        if (!rc) rc = mclbm_set_viscosity(L, d.nu1, d.nu2);
        if (!rc) rc = mclbm_set_coupling(L, d.g_coh, d.g_ads);
        if (!rc) rc = mclbm_set_body_force(L, d.gx, d.gy);
        if (!rc) rc = mclbm_set_pressure_bc(L, d.rho_in1, d.rho_out2);
        if (!rc) rc = mclbm_set_flag(L, MCLBM_FLAG_PERIODIC_Y, d.periodic_y);
        if (!rc && d.rho1 && d.rho2) rc = mclbm_init_densities(L, d.rho1, d.rho2);
        if (L) b->cases.push_back(L);
        if (!rc && !L->tmaps) rc = fail(MCLBM_ERR_STATE, "TMA descriptors are not available");
        if (rc) {
            std::string msg = "case " + std::to_string(k) + ": " + mclbm_last_error();
            destroy_batch(b);
            return fail(rc, msg);
        }
        b->total_nodes += (int64_t)d.nx * d.ny;
    }
    for (int shape = 0; shape < 2; ++shape) {
        b->maps[shape].resize(tile_maps_bytes() * ncases);
        for (int k = 0; k < ncases; ++k) {
            if (int rc = tile_maps_for(*b->cases[k], shape, b->maps[shape].data() + k * tile_maps_bytes())) {
                destroy_batch(b);
                return rc;
            }
        }
    }
    *out = b;
    return MCLBM_OK;
}

int mclbm_batch_destroy(mclbm_batch *b) {
    if (!b) return MCLBM_OK;
    cudaStreamSynchronize(b->stream);
    destroy_batch(b);
    return MCLBM_OK;
}

int mclbm_batch_lattice(mclbm_batch *b, int k, mclbm_lattice **view) {
    if (!b || !view) return fail(MCLBM_ERR_ARG, "NULL argument");
    if (k < 0 || k >= (int)b->cases.size()) return fail(MCLBM_ERR_ARG, "case index out of range");
    *view = b->cases[k];
    return MCLBM_OK;
}

int mclbm_batch_step(mclbm_batch *b, int64_t nsteps) {
    if (!b) return fail(MCLBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return fail(MCLBM_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return MCLBM_OK;
    for (auto *L : b->cases) {
        if (int rc = check_ready(*L)) return rc;
        if (int rc = refresh_ghosts(*L)) return rc;
    }
    int64_t left = nsteps;
    if (b->cand < 0) {
        int rc = MCLBM_OK;
        left -= autotune(*b, left, &rc);
        if (rc) return rc;
    }
    if (int rc = ensure_layout(*b, b->cand)) return rc;
    const int parity = parity_of(*b, b->cand);
    for (auto *L : b->cases)
        if ((fluid_cand(b->cand) ? L->scur : L->cur) != parity)
            return fail(MCLBM_ERR_STATE, "the cases of a batch were stepped separately "
                                         "and are at different buffer parities");
    if (left >= 2 * GRAPH_STEPS) {
        if (!b->graph || b->graph_version != version_of(*b) || b->graph_parity != parity) {
            if (parity != b->graph_parity && b->graph && b->graph_version == version_of(*b)) {
                // one direct step brings the parity back to the captured one
                if (int rc = direct_step(*b, b->cand)) return rc;
                --left;
            } else if (int rc = capture_graph(*b)) {
                return rc;
            }
        }
        while (left >= GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            count_launch(GRAPH_STEPS);
            for (auto *L : b->cases) L->steps += GRAPH_STEPS;
            b->steps += GRAPH_STEPS;
            left -= GRAPH_STEPS;
        }
    }
    while (left-- > 0)
        if (int rc = direct_step(*b, b->cand)) return rc;
    return MCLBM_OK;
}

int mclbm_batch_info(mclbm_batch *b, int64_t out[8]) {
    if (!b || !out) return fail(MCLBM_ERR_ARG, "NULL argument");
    out[0] = (int64_t)b->cases.size();
    out[1] = b->total_nodes;
    const int cand = b->cand < 0 ? 0 : b->cand;
    out[2] = b->cand < 0 ? -1 : (fluid_cand(cand) ? 2 + shape_of_cand(cand) : shape_of_cand(cand));
    out[3] = grid_of_cand(cand) == 0 ? 0 : -1;
    out[4] = GRAPH_STEPS;
    out[5] = b->steps;
    out[6] = fluid_cand(cand) ? 0 : batch_slots(b->prec, shape_of_cand(cand));
    out[7] = b->graph ? 1 : 0;
    return MCLBM_OK;
}

int mclbm_batch_tuning(mclbm_batch *b, double ms_per_step[6]) {
    if (!b || !ms_per_step) return fail(MCLBM_ERR_ARG, "NULL argument");
    for (int k = 0; k < NCAND; ++k) ms_per_step[k] = b->tune_ms[k];
    return MCLBM_OK;
}

}  // extern "C"
