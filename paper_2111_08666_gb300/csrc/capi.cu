// The C ABI of include/mclbm.h: argument checks, device memory, host/device
// transfers, and the step loop.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbm.cuh"

namespace mclbm {

namespace {
thread_local std::string g_error;
std::atomic<long long> g_launches{0};

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A device view of a caller buffer: the buffer itself if it is device
// memory, else a temporary device copy (for inputs) or staging area.
struct DeviceView {
    void *ptr = nullptr;
    void *tmp = nullptr;
    ~DeviceView() {
        if (tmp) cudaFree(tmp);
    }
};

int view_in(Lattice &L, const void *src, size_t bytes, DeviceView &v) {
    if (is_device_ptr(src)) {
        v.ptr = const_cast<void *>(src);
        return MCLBM_OK;
    }
    cudaError_t e = cudaMalloc(&v.tmp, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(staging)");
    e = cudaMemcpyAsync(v.tmp, src, bytes, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(H2D)");
    v.ptr = v.tmp;
    return MCLBM_OK;
}

int view_out(void *dst, size_t bytes, DeviceView &v) {
    if (is_device_ptr(dst)) {
        v.ptr = dst;
        return MCLBM_OK;
    }
    cudaError_t e = cudaMalloc(&v.tmp, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(staging)");
    v.ptr = v.tmp;
    return MCLBM_OK;
}

// finish an output view: copy back to the host buffer if staged, and wait
int finish_out(Lattice &L, void *dst, size_t bytes, DeviceView &v) {
    cudaError_t e;
    if (v.tmp) {
        e = cudaMemcpyAsync(dst, v.tmp, bytes, cudaMemcpyDeviceToHost, L.stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
    e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return MCLBM_OK;
}

size_t store_bytes_of(mclbm_precision p) {
    switch (p) {
        case MCLBM_FP64: return 8;
        case MCLBM_FP32:
        case MCLBM_FP32_DEV: return 4;
        default: return 2;
    }
}

int check_lat(const Lattice *L) {
    if (!L) return fail(MCLBM_ERR_ARG, "lattice handle is NULL");
    return MCLBM_OK;
}

int make_current(const Lattice &L) {
    cudaError_t e = cudaSetDevice(L.device);
    return e == cudaSuccess ? MCLBM_OK : cuda_fail(e, "cudaSetDevice");
}

// Free the device and pinned memory of a lattice (not the object itself).
void release(Lattice *L) {
    if (!L) return;
    cudaSetDevice(L->device);
    cudaFree(L->geo);
    cudaFree(L->chi);
    cudaFree(L->chi_f);
    cudaFree(L->f[0]);
    cudaFree(L->f[1]);
    cudaFree(L->d5);
    cudaFree(L->diag_partial);
    cudaFree(L->diag_out);
    cudaFree(L->bad_flag);
    cudaFree(L->blend_count);
    cudaFree(L->err);
    cudaFree(L->geo_pad);
    tma_release(*L);
    sparse_release(*L);
    if (L->host_diag) cudaFreeHost(L->host_diag);
    if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
    L->own_stream = false;
}

int dev_alloc(Lattice &L, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MCLBM_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                         cudaGetErrorString(e));
    }
    L.device_bytes += bytes;
    return MCLBM_OK;
}

int run_diagnostics(Lattice &L, double out[8]) {
    if (int rc = sparse_to_dense(L)) return rc;
    cudaError_t e = launch_diagnostics(L);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics kernel");
    e = cudaMemcpyAsync(L.host_diag, L.diag_out, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                        L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(diagnostics)");
    e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    std::memcpy(out, L.host_diag, 8 * sizeof(double));
    return MCLBM_OK;
}

}  // namespace

int fail(int code, const std::string &msg) {
    g_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    return MCLBM_ERR_CUDA;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Rebuild the ghost columns and tables if the boundary mode changed since
// they were last built.
int refresh_ghosts(Lattice &L) {
    if (L.ghost_mode == L.ghost_key()) return MCLBM_OK;
    cudaError_t e = launch_geo_ghosts(L);
    if (e != cudaSuccess) return cuda_fail(e, "ghost columns");
    if (int rc = tma_build_tables(L)) return rc;
    L.ghost_mode = L.ghost_key();
    return MCLBM_OK;
}

int check_ready(Lattice &L) {
    if (!L.initialised)
        return fail(MCLBM_ERR_STATE, "populations not initialised: call mclbm_init_densities");
    if (!L.p.periodic_y && !L.boundary_rows_solid)
        return fail(MCLBM_ERR_ARG,
                    "rows 0 and ny-1 must be solid unless the lattice is periodic in y");
    return MCLBM_OK;
}

// the dense buffers current, with their ghost copies
int dense_current(Lattice &L) {
    if (int rc = sparse_to_dense(L)) return rc;
    if (L.pop_ghosts_stale && L.ghost_mode == L.ghost_key()) {
        cudaError_t e = launch_geo_ghosts(L);
        if (e != cudaSuccess) return cuda_fail(e, "ghost columns");
    }
    L.pop_ghosts_stale = false;
    return MCLBM_OK;
}

int lattice_prepare_step(Lattice &L) {
    if (int rc = check_ready(L)) return rc;
    if (int rc = dense_current(L)) return rc;
    if (int rc = refresh_ghosts(L)) return rc;
    L.sparse_state = 0;  // the batched kernel steps the dense buffers
    return MCLBM_OK;
}

}  // namespace mclbm

using namespace mclbm;


extern "C" {

const char *mclbm_last_error(void) { return g_error.c_str(); }

int64_t mclbm_launch_count(void) { return g_launches.load(); }

int mclbm_create(int nx, int ny, const uint8_t *solid, const float *xi, mclbm_precision prec,
                 void *cuda_stream, mclbm_lattice **out) {
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3) return fail(MCLBM_ERR_ARG, "nx and ny must be >= 3");
    if ((long long)nx * ny > (1LL << 31)) return fail(MCLBM_ERR_ARG, "lattice too large");
    if (!solid) return fail(MCLBM_ERR_ARG, "solid is NULL");
    if (prec < MCLBM_FP64 || prec > MCLBM_BF16_DEV) return fail(MCLBM_ERR_ARG, "bad precision");
    mclbm_lattice *L = new (std::nothrow) mclbm_lattice();
    if (!L) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&L->device);
    if (e != cudaSuccess) {
        delete L;
        return cuda_fail(e, "cudaGetDevice");
    }
    L->nx = nx;
    L->ny = ny;
    L->prec = prec;
    L->store_bytes = store_bytes_of(prec);
    L->real_bytes = prec == MCLBM_FP64 ? 8 : 4;
    L->planes = (prec == MCLBM_FP64 || prec == MCLBM_FP32) ? 18 : 20;
    L->hx = L->store_bytes >= 4 ? 4 : 16 / (int)L->store_bytes;
    {
        // rows: every strip's staged copy in bounds, 128-byte aligned, an odd
        // number of 128-byte lines; planes: an odd number of lines as well
        const long long sb = (long long)L->store_bytes;
        const long long cols = (long long)(nx + SWEEP_W - 1) / SWEEP_W * SWEEP_W + 2 * L->hx;
        long long row_bytes = (cols * sb + 127) / 128 * 128;
        if ((row_bytes / 128) % 2 == 0) row_bytes += 128;
        L->pitch = (int)(row_bytes / sb);
        long long plane_bytes = row_bytes * (ny + 2 * HY);
        if ((plane_bytes / 128) % 2 == 0) plane_bytes += 128;
        L->plane = plane_bytes / sb;
        L->gpitch = (int)(((long long)(nx + SWEEP_W - 1) / SWEEP_W * SWEEP_W + 2 * GEO_HX + 15) / 16 * 16);
    }

    // geometry codes and the wettability table (chi^1 = 1 + xi, chi^2 = 1 - xi)
    std::vector<uint8_t> geo((size_t)L->gpitch * ny, GEO_OUTSIDE);
    std::vector<double> chi(512, 1.0);
    std::map<uint32_t, int> codes;
    bool rows_solid = true;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t k = (size_t)y * nx + x;
            uint8_t c = GEO_FLUID;
            if (solid[k]) {
                const float v = xi ? xi[k] : 0.0f;
                if (!std::isfinite(v)) {
                    delete L;
                    return fail(MCLBM_ERR_ARG, "xi is not finite at a solid node");
                }
                uint32_t bits;
                std::memcpy(&bits, &v, 4);
                auto it = codes.find(bits);
                if (it == codes.end()) {
                    if ((int)codes.size() >= MAX_XI_VALUES) {
                        delete L;
                        return fail(MCLBM_ERR_ARG, "more than 254 distinct xi values on solid nodes");
                    }
                    const int code = 1 + (int)codes.size();
                    codes[bits] = code;
                    chi[2 * code] = 1.0 + (double)v;
                    chi[2 * code + 1] = 1.0 - (double)v;
                    c = (uint8_t)code;
                } else {
                    c = (uint8_t)it->second;
                }
            } else if (y == 0 || y == ny - 1) {
                rows_solid = false;
            }
            geo[(size_t)y * L->gpitch + GEO_HX + x] = c;
        }
    L->boundary_rows_solid = rows_solid;
    std::vector<float> chi_f(chi.begin(), chi.end());  // round to nearest, as on the device
    L->p.round_fp32();

    if (cuda_stream) {
        L->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete L;
            return cuda_fail(e, "cudaStreamCreate");
        }
        L->own_stream = true;
    }
    const size_t geo_bytes = (size_t)L->gpitch * ny;
    L->geo_pad_rows = ny + 2 * HY + 16;  // room for the deepest tile frame past the edge
    const size_t pop_bytes = (size_t)L->planes * (size_t)L->plane * L->store_bytes;
    int rc = MCLBM_OK;
    L->diag_blocks = diag_blocks_for(*L);
    if ((rc = dev_alloc(*L, (void **)&L->geo, geo_bytes)) ||
        (rc = dev_alloc(*L, (void **)&L->chi, 512 * sizeof(double))) ||
        (rc = dev_alloc(*L, (void **)&L->chi_f, 512 * sizeof(float))) ||
        (rc = dev_alloc(*L, &L->f[0], pop_bytes)) ||
        (rc = dev_alloc(*L, &L->f[1], pop_bytes)) ||
        (rc = dev_alloc(*L, (void **)&L->err, sizeof(int))) ||
        (rc = dev_alloc(*L, (void **)&L->geo_pad, (size_t)L->geo_pad_rows * L->gpitch)) ||
        (rc = dev_alloc(*L, &L->d5, 6 * (size_t)ny * L->real_bytes)) ||
        (rc = dev_alloc(*L, (void **)&L->diag_partial, (size_t)L->diag_blocks * 9 * sizeof(double))) ||
        (rc = dev_alloc(*L, (void **)&L->diag_out, 8 * sizeof(double))) ||
        (rc = dev_alloc(*L, (void **)&L->bad_flag, sizeof(unsigned long long)))) {
        release(L);
        delete L;
        return rc;
    }
    if ((rc = tma_prepare(*L))) {
        release(L);
        delete L;
        return rc;
    }
    e = cudaMallocHost((void **)&L->host_diag, 8 * sizeof(double));
    if (e != cudaSuccess) {
        release(L);
        delete L;
        return cuda_fail(e, "cudaMallocHost");
    }
    if ((e = cudaMemcpyAsync(L->geo, geo.data(), geo_bytes, cudaMemcpyHostToDevice, L->stream)) ||
        (e = cudaMemcpyAsync(L->chi, chi.data(), 512 * sizeof(double), cudaMemcpyHostToDevice,
                             L->stream)) ||
        (e = cudaMemcpyAsync(L->chi_f, chi_f.data(), 512 * sizeof(float), cudaMemcpyHostToDevice,
                             L->stream)) ||
        (e = cudaMemsetAsync(L->f[0], 0, pop_bytes, L->stream)) ||
        (e = cudaMemsetAsync(L->f[1], 0, pop_bytes, L->stream)) ||
        (e = cudaMemsetAsync(L->err, 0, sizeof(int), L->stream)) ||
        (e = cudaMemsetAsync(L->d5, 0, 6 * (size_t)ny * L->real_bytes, L->stream)) ||
        (e = cudaMemsetAsync(L->bad_flag, 0, sizeof(unsigned long long), L->stream)) ||
        (e = cudaStreamSynchronize(L->stream))) {
        release(L);
        delete L;
        return cuda_fail(e, "lattice upload");
    }
    *out = L;
    return MCLBM_OK;
}

int mclbm_destroy(mclbm_lattice *lat) {
    if (!lat) return MCLBM_OK;
    cudaSetDevice(lat->device);
    cudaStreamSynchronize(lat->stream);
    release(lat);
    delete lat;
    return MCLBM_OK;
}

// Band height of the fluid-only kernel: 12 rows by default (256 compute
// threads, three CTAs per SM: their warps fill each other's barrier waits),
// 16 rows for shape 1 (384 compute threads, two CTAs per SM).
static int sparse_height(const Lattice &L) { return L.tile_shape == 1 ? 16 : 12; }

int mclbm_set_flag(mclbm_lattice *lat, int flag, int64_t value) {
    if (int rc = check_lat(lat)) return rc;
    switch (flag) {
        case MCLBM_FLAG_PERIODIC_Y:
            lat->p.periodic_y = value ? 1 : 0;
            ++lat->version;
            return MCLBM_OK;
        case MCLBM_FLAG_VEL_SHIFT:
            lat->p.vel_shift = value ? 1 : 0;
            ++lat->version;
            return MCLBM_OK;
        case MCLBM_FLAG_KERNEL:
            if (value < 0 || value > 4) return fail(MCLBM_ERR_ARG, "kernel must be 0..4");
            lat->kernel = value;
            return MCLBM_OK;
        case MCLBM_FLAG_TILE_SHAPE:
            if (value < 0 || value > 1) return fail(MCLBM_ERR_ARG, "tile shape must be 0 or 1");
            lat->tile_shape = (int)value;
            return MCLBM_OK;
        case MCLBM_FLAG_DIAG_EVERY:
            if (value < 0) return fail(MCLBM_ERR_ARG, "diag_every must be >= 0");
            lat->diag_every = value;
            return MCLBM_OK;
        case MCLBM_FLAG_WAIT_LIMIT_US:
            if (value < 1 || value > 10000000)
                return fail(MCLBM_ERR_ARG, "the wait limit must be 1..10000000 microseconds");
            lat->wait_ns = (uint64_t)value * 1000ull;
            return MCLBM_OK;
        case MCLBM_FLAG_TEST_NO_COPY:
            lat->test_no_copy = value ? 1 : 0;
            return MCLBM_OK;
        default: return fail(MCLBM_ERR_ARG, "unknown flag " + std::to_string(flag));
    }
}

int mclbm_set_viscosity(mclbm_lattice *lat, double nu1, double nu2) {
    if (int rc = check_lat(lat)) return rc;
    if (!(nu1 > 0) || !(nu2 > 0) || !std::isfinite(nu1) || !std::isfinite(nu2))
        return fail(MCLBM_ERR_ARG, "viscosities must be positive and finite");
    lat->p.nu1 = nu1;
    lat->p.nu2 = nu2;
    lat->p.round_fp32();
    ++lat->version;
    return MCLBM_OK;
}

int mclbm_set_coupling(mclbm_lattice *lat, double g_coh, double g_ads) {
    if (int rc = check_lat(lat)) return rc;
    if (!std::isfinite(g_coh) || !std::isfinite(g_ads))
        return fail(MCLBM_ERR_ARG, "coupling strengths must be finite");
    lat->p.g_coh = g_coh;
    lat->p.g_ads = g_ads;
    lat->p.round_fp32();
    ++lat->version;
    return MCLBM_OK;
}

int mclbm_set_body_force(mclbm_lattice *lat, double gx, double gy) {
    if (int rc = check_lat(lat)) return rc;
    if (!std::isfinite(gx) || !std::isfinite(gy)) return fail(MCLBM_ERR_ARG, "g must be finite");
    lat->p.gx = gx;
    lat->p.gy = gy;
    lat->p.round_fp32();
    ++lat->version;
    return MCLBM_OK;
}

int mclbm_set_pressure_bc(mclbm_lattice *lat, double rho_in1, double rho_out2) {
    if (int rc = check_lat(lat)) return rc;
    if (!std::isfinite(rho_in1) || !std::isfinite(rho_out2))
        return fail(MCLBM_ERR_ARG, "boundary densities must be finite");
    ++lat->version;
    if (rho_in1 < 0 || rho_out2 < 0) {
        lat->p.open_x = 0;
        lat->p.rho_in1 = lat->p.rho_out2 = -1.0;
        lat->p.round_fp32();
        return MCLBM_OK;
    }
    if (rho_in1 == 0 || rho_out2 == 0)
        return fail(MCLBM_ERR_ARG, "boundary densities must be positive");
    lat->p.open_x = 1;
    lat->p.rho_in1 = rho_in1;
    lat->p.rho_out2 = rho_out2;
    lat->p.round_fp32();
    return MCLBM_OK;
}

int mclbm_set_bc(mclbm_lattice *lat, int bc_set, double rho_in2, double rho_out1) {
    if (int rc = check_lat(lat)) return rc;
    if (bc_set < 1 || bc_set > 3) return fail(MCLBM_ERR_ARG, "bc_set must be 1, 2 or 3");
    if (bc_set == 1 && !(std::isfinite(rho_in2) && std::isfinite(rho_out1) && rho_in2 > 0 && rho_out1 > 0))
        return fail(MCLBM_ERR_ARG, "Set-1 needs positive finite rho_in2 and rho_out1");
    ++lat->version;
    lat->p.bc_set = bc_set;
    lat->p.rho_in2 = bc_set == 1 ? rho_in2 : 0.0;
    lat->p.rho_out1 = bc_set == 1 ? rho_out1 : 0.0;
    lat->p.round_fp32();
    return MCLBM_OK;
}

int mclbm_set_mrt(mclbm_lattice *lat, int on, double s_e, double s_eps, double s_q) {
    if (int rc = check_lat(lat)) return rc;
    auto rate_ok = [](double s) { return s == 0.0 || (s > 0.0 && s < 2.0); };
    if (on && (!rate_ok(s_e) || !rate_ok(s_eps) || !(rate_ok(s_q) || s_q == -1.0)))
        return fail(MCLBM_ERR_ARG, "MRT rates must lie in (0, 2), or be 0 (1/tau_s); s_q may be -1");
    ++lat->version;
    lat->p.mrt = on ? 1 : 0;
    lat->p.s_e = on ? s_e : 0.0;
    lat->p.s_eps = on ? s_eps : 0.0;
    lat->p.s_q = on ? s_q : 0.0;
    lat->p.round_fp32();
    return MCLBM_OK;
}

int mclbm_set_pressure_bc_p(mclbm_lattice *lat, double p_in, double p_out) {
    if (int rc = check_lat(lat)) return rc;
    if (p_in < 0 || p_out < 0) return mclbm_set_pressure_bc(lat, -1.0, -1.0);
    // Eq. 14 with the minority density m = 0.027: P = (r + m)/3 + (G/3) r m
    const double m = 0.027, G = lat->p.g_coh;
    const double denom = (1.0 + G * m) / 3.0;
    const double r_in = (p_in - m / 3.0) / denom, r_out = (p_out - m / 3.0) / denom;
    if (!(r_in > 0) || !(r_out > 0))
        return fail(MCLBM_ERR_ARG, "pressure below the minority-only pressure");
    return mclbm_set_pressure_bc(lat, r_in, r_out);
}

int mclbm_set_stream(mclbm_lattice *lat, void *cuda_stream) {
    if (int rc = check_lat(lat)) return rc;
    cudaStreamSynchronize(lat->stream);
    if (lat->own_stream && !cuda_stream) return MCLBM_OK;
    if (lat->own_stream) {
        cudaStreamDestroy(lat->stream);
        lat->own_stream = false;
    }
    if (cuda_stream) {
        lat->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&lat->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        lat->own_stream = true;
    }
    return MCLBM_OK;
}

int mclbm_init_densities(mclbm_lattice *lat, const double *rho1, const double *rho2) {
    if (int rc = check_lat(lat)) return rc;
    if (!rho1 || !rho2) return fail(MCLBM_ERR_ARG, "rho1/rho2 is NULL");
    if (int rc = make_current(*lat)) return rc;
    const size_t bytes = (size_t)lat->nx * lat->ny * sizeof(double);
    DeviceView v1, v2;
    if (int rc = view_in(*lat, rho1, bytes, v1)) return rc;
    if (int rc = view_in(*lat, rho2, bytes, v2)) return rc;
    lat->ghost_mode = -1;
    if (int rc = refresh_ghosts(*lat)) return rc;
    cudaError_t e = launch_init_equilibrium(*lat, static_cast<const double *>(v1.ptr),
                                            static_cast<const double *>(v2.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    e = cudaStreamSynchronize(lat->stream);  // staging buffers are freed on return
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    lat->sparse_state = 0;
    lat->pop_ghosts_stale = false;
    lat->initialised = true;
    lat->steps = 0;
    return MCLBM_OK;
}

int mclbm_init_from_phase(mclbm_lattice *lat, const float *phi) {
    if (int rc = check_lat(lat)) return rc;
    if (!phi) return fail(MCLBM_ERR_ARG, "phi is NULL");
    if (int rc = make_current(*lat)) return rc;
    const size_t n = (size_t)lat->nx * lat->ny;
    DeviceView vp;
    if (int rc = view_in(*lat, phi, n * sizeof(float), vp)) return rc;
    double *r = nullptr;
    cudaError_t e = cudaMalloc((void **)&r, 2 * n * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(staging)");
    // rho_hi = 1, rho_lo = 0.027: the separated phases at G = 3.5 (Sec. 3.1)
    e = launch_phase_densities(*lat, static_cast<const float *>(vp.ptr), 1.0, 0.027, r, r + n);
    if (e == cudaSuccess) {
        lat->ghost_mode = -1;
        if (int rc = refresh_ghosts(*lat)) {
            cudaFree(r);
            return rc;
        }
        e = launch_init_equilibrium(*lat, r, r + n);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    cudaFree(r);
    if (e != cudaSuccess) return cuda_fail(e, "init from phase");
    lat->sparse_state = 0;
    lat->pop_ghosts_stale = false;
    lat->initialised = true;
    lat->steps = 0;
    return MCLBM_OK;
}

int mclbm_blend_phase(mclbm_lattice *lat, const float *phi_hat, double flip, int64_t *changed) {
    if (int rc = check_lat(lat)) return rc;
    if (!phi_hat) return fail(MCLBM_ERR_ARG, "phi_hat is NULL");
    if (!(flip >= 0.0) || !(flip < 1.0)) return fail(MCLBM_ERR_ARG, "flip must be in [0, 1)");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = check_ready(*lat)) return rc;
    const size_t n = (size_t)lat->nx * lat->ny;
    DeviceView vp;
    if (int rc = view_in(*lat, phi_hat, n * sizeof(float), vp)) return rc;
    cudaError_t e = cudaSuccess;
    if (!lat->blend_count) {
        e = cudaMalloc((void **)&lat->blend_count, sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(blend counter)");
    }
    if (int rc = dense_current(*lat)) return rc;
    e = cudaMemsetAsync(lat->blend_count, 0, sizeof(unsigned long long), lat->stream);
    // rho_hi = 1, rho_lo = 0.027: the separated phases at G = 3.5 (Sec. 3.1)
    if (e == cudaSuccess)
        e = launch_blend_phase(*lat, static_cast<const float *>(vp.ptr), 1.0, 0.027, flip, lat->blend_count);
    unsigned long long cnt = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&cnt, lat->blend_count, sizeof(cnt), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "warm-start blend");
    lat->sparse_state = 0;  // the dense buffers hold the state
    if (changed) *changed = (int64_t)cnt;
    return MCLBM_OK;
}

int mclbm_set_populations(mclbm_lattice *lat, const double *f) {
    if (int rc = check_lat(lat)) return rc;
    if (!f) return fail(MCLBM_ERR_ARG, "f is NULL");
    if (int rc = make_current(*lat)) return rc;
    DeviceView v;
    if (int rc = view_in(*lat, f, (size_t)18 * lat->nx * lat->ny * sizeof(double), v)) return rc;
    lat->ghost_mode = -1;
    if (int rc = refresh_ghosts(*lat)) return rc;
    cudaError_t e = launch_set_populations(*lat, static_cast<const double *>(v.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "import kernel");
    e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    lat->sparse_state = 0;
    lat->pop_ghosts_stale = false;
    lat->initialised = true;
    return MCLBM_OK;
}

int mclbm_get_populations(mclbm_lattice *lat, double *f) {
    if (int rc = check_lat(lat)) return rc;
    if (!f) return fail(MCLBM_ERR_ARG, "f is NULL");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    const size_t bytes = (size_t)18 * lat->nx * lat->ny * sizeof(double);
    DeviceView v;
    if (int rc = view_out(f, bytes, v)) return rc;
    cudaError_t e = launch_get_populations(*lat, static_cast<double *>(v.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "export kernel");
    return finish_out(*lat, f, bytes, v);
}

// Checkpoint file: header, Params, then the current population buffer and
// the frozen boundary records of Eqs. 26-27 as raw device bytes (bit-exact
// restore).  Version 2: Params carry the inlet/outlet treatment (Set-1/2/3).
namespace {
struct CheckpointHeader {
    char magic[8];
    int32_t version, nx, ny, prec;
    int64_t pop_bytes, d5_bytes, steps;
};
constexpr char CKPT_MAGIC[8] = {'M', 'C', 'L', 'B', 'M', 'C', 'K', '1'};
}  // namespace

int mclbm_save(mclbm_lattice *lat, const char *path) {
    if (int rc = check_lat(lat)) return rc;
    if (!path) return fail(MCLBM_ERR_ARG, "path is NULL");
    if (!lat->initialised) return fail(MCLBM_ERR_STATE, "nothing to save: lattice not initialised");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    CheckpointHeader h{};
    std::memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 2;
    h.nx = lat->nx;
    h.ny = lat->ny;
    h.prec = (int32_t)lat->prec;
    h.pop_bytes = (int64_t)lat->planes * lat->plane * (int64_t)lat->store_bytes;
    h.d5_bytes = 6 * (int64_t)lat->ny * (int64_t)lat->real_bytes;
    h.steps = lat->steps;
    std::vector<unsigned char> buf((size_t)(h.pop_bytes + h.d5_bytes));
    cudaError_t e = cudaMemcpyAsync(buf.data(), lat->f[lat->cur], (size_t)h.pop_bytes,
                                    cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf.data() + h.pop_bytes, lat->d5, (size_t)h.d5_bytes, cudaMemcpyDeviceToHost,
                            lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint read-back");
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(MCLBM_ERR_ARG, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(&lat->p, sizeof(Params), 1, fp) == 1 &&
              std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? MCLBM_OK : fail(MCLBM_ERR_ARG, std::string("write to ") + path + " failed");
}

int mclbm_load(mclbm_lattice *lat, const char *path) {
    if (int rc = check_lat(lat)) return rc;
    if (!path) return fail(MCLBM_ERR_ARG, "path is NULL");
    if (int rc = make_current(*lat)) return rc;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(MCLBM_ERR_ARG, std::string("cannot open ") + path);
    CheckpointHeader h{};
    Params p;
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::fread(&p, sizeof(Params), 1, fp) == 1;
    const int64_t pop_bytes = (int64_t)lat->planes * lat->plane * (int64_t)lat->store_bytes;
    const int64_t d5_bytes = 6 * (int64_t)lat->ny * (int64_t)lat->real_bytes;
    ok = ok && std::memcmp(h.magic, CKPT_MAGIC, 8) == 0 && h.version == 2;
    if (ok && (h.nx != lat->nx || h.ny != lat->ny || h.prec != (int32_t)lat->prec ||
               h.pop_bytes != pop_bytes || h.d5_bytes != d5_bytes)) {
        std::fclose(fp);
        return fail(MCLBM_ERR_ARG, "checkpoint is of another lattice size or precision");
    }
    std::vector<unsigned char> buf;
    if (ok) {
        buf.resize((size_t)(pop_bytes + d5_bytes));
        ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    }
    std::fclose(fp);
    if (!ok) return fail(MCLBM_ERR_ARG, std::string(path) + " is not a complete checkpoint");
    lat->cur = 0;
    cudaError_t e = cudaMemcpyAsync(lat->f[0], buf.data(), (size_t)pop_bytes, cudaMemcpyHostToDevice,
                                    lat->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lat->d5, buf.data() + pop_bytes, (size_t)d5_bytes, cudaMemcpyHostToDevice,
                            lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint upload");
    lat->sparse_state = 0;
    lat->pop_ghosts_stale = false;
    lat->p = p;
    lat->p.round_fp32();
    lat->steps = h.steps;
    lat->initialised = true;
    lat->ghost_mode = -1;  // boundary mode of the restored parameters
    ++lat->version;
    return MCLBM_OK;
}

int mclbm_step(mclbm_lattice *lat, int64_t nsteps) {
    if (int rc = check_lat(lat)) return rc;
    if (nsteps < 0) return fail(MCLBM_ERR_ARG, "nsteps < 0");
    if (int rc = check_ready(*lat)) return rc;
    if (int rc = make_current(*lat)) return rc;
    if (int rc = refresh_ghosts(*lat)) return rc;
    int which = (int)lat->kernel;
    if (which == 0) {
        // the fluid-only kernel where it serves this precision and geometry,
        // else the TMA tile kernel, else (FP64) the global-memory tile kernel
        which = tma_supported(*lat) ? 3 : 1;
        if (sparse_precision(lat->prec)) {
            if (sparse_prepare(*lat, sparse_height(*lat)) == MCLBM_OK && lat->nfp > 0) which = 4;
        }
    }
    if (which == 3 && !tma_supported(*lat))
        return fail(MCLBM_ERR_ARG, "the TMA tile kernel is not available for this precision");
    if (which == 2 && !sweep_supported(*lat))
        return fail(MCLBM_ERR_ARG, "the strip kernel is not available for this lattice");
    if (which == 4) {
        if (!sparse_precision(lat->prec))
            return fail(MCLBM_ERR_ARG, "the fluid-only kernel is not available for this precision");
        if (int rc = sparse_prepare(*lat, sparse_height(*lat))) return rc;
        if (int rc = dense_to_sparse(*lat)) return rc;
    } else if (nsteps > 0) {
        if (int rc = dense_current(*lat)) return rc;
    }
    for (int64_t t = 0; t < nsteps; ++t) {
        cudaError_t e = which == 4   ? launch_step_sparse(*lat)
                        : which == 3 ? launch_step_tma(*lat)
                        : which == 2 ? launch_step_sweep(*lat)
                                     : launch_step_tile(*lat, 0);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel");
        if (which != 4) lat->sparse_state = 0;
        ++lat->steps;
        if (lat->diag_every > 0 && lat->steps % lat->diag_every == 0) {
            if (int rc = sparse_to_dense(*lat)) return rc;
            e = launch_diagnostics(*lat);
            if (e != cudaSuccess) return cuda_fail(e, "divergence check");
        }
    }
    return MCLBM_OK;
}

int mclbm_synchronize(mclbm_lattice *lat) {
    if (int rc = check_lat(lat)) return rc;
    if (int rc = make_current(*lat)) return rc;
    cudaError_t e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int err = 0;
    e = cudaMemcpy(&err, lat->err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error word)");
    if (err) {
        cudaMemset(lat->err, 0, sizeof(err));
        return fail(err, "a bounded wait in the step kernel ran out; the state is not valid");
    }
    unsigned long long bad = 0;
    e = cudaMemcpy(&bad, lat->bad_flag, sizeof(bad), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(flag)");
    if (bad) {
        cudaMemset(lat->bad_flag, 0, sizeof(bad));
        return fail(MCLBM_ERR_DIVERGED, std::to_string(bad) +
                                            " node-checks saw a non-finite or negative density");
    }
    return MCLBM_OK;
}

int mclbm_read_density(mclbm_lattice *lat, int comp, double *out) {
    if (int rc = check_lat(lat)) return rc;
    if (comp != 1 && comp != 2) return fail(MCLBM_ERR_ARG, "comp must be 1 or 2");
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    const size_t bytes = (size_t)lat->nx * lat->ny * sizeof(double);
    DeviceView v;
    if (int rc = view_out(out, bytes, v)) return rc;
    cudaError_t e = launch_density(*lat, comp - 1, static_cast<double *>(v.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "density kernel");
    return finish_out(*lat, out, bytes, v);
}

int mclbm_read_pressure(mclbm_lattice *lat, double *out) {
    if (int rc = check_lat(lat)) return rc;
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    const size_t bytes = (size_t)lat->nx * lat->ny * sizeof(double);
    DeviceView v;
    if (int rc = view_out(out, bytes, v)) return rc;
    cudaError_t e = launch_pressure(*lat, static_cast<double *>(v.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "pressure kernel");
    return finish_out(*lat, out, bytes, v);
}

int mclbm_read_phase(mclbm_lattice *lat, float *out) {
    if (int rc = check_lat(lat)) return rc;
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    const size_t bytes = (size_t)lat->nx * lat->ny * sizeof(float);
    DeviceView v;
    if (int rc = view_out(out, bytes, v)) return rc;
    cudaError_t e = launch_phase(*lat, static_cast<float *>(v.ptr));
    if (e != cudaSuccess) return cuda_fail(e, "phase kernel");
    return finish_out(*lat, out, bytes, v);
}

int mclbm_read_velocity(mclbm_lattice *lat, double *ux, double *uy) {
    if (int rc = check_lat(lat)) return rc;
    if (!ux || !uy) return fail(MCLBM_ERR_ARG, "ux/uy is NULL");
    if (int rc = make_current(*lat)) return rc;
    if (int rc = sparse_to_dense(*lat)) return rc;
    const size_t bytes = (size_t)lat->nx * lat->ny * sizeof(double);
    DeviceView vx, vy;
    if (int rc = view_out(ux, bytes, vx)) return rc;
    if (int rc = view_out(uy, bytes, vy)) return rc;
    void *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, velocity_scratch_bytes(*lat));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(velocity scratch)");
    e = launch_velocity(*lat, static_cast<double *>(vx.ptr), static_cast<double *>(vy.ptr),
                        scratch);
    int rc = MCLBM_OK;
    if (e != cudaSuccess) rc = cuda_fail(e, "velocity kernels");
    if (rc == MCLBM_OK && vx.tmp) {
        e = cudaMemcpyAsync(ux, vx.tmp, bytes, cudaMemcpyDeviceToHost, lat->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
    if (rc == MCLBM_OK) rc = finish_out(*lat, uy, bytes, vy);
    else cudaStreamSynchronize(lat->stream);
    cudaFree(scratch);
    return rc;
}

int mclbm_diagnostics(mclbm_lattice *lat, double out[8]) {
    if (int rc = check_lat(lat)) return rc;
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    if (int rc = make_current(*lat)) return rc;
    return run_diagnostics(*lat, out);
}

int mclbm_saturation(mclbm_lattice *lat, double *sw_count, double *sw_mass) {
    double d[8];
    if (int rc = mclbm_diagnostics(lat, d)) return rc;
    if (sw_count) *sw_count = d[2];
    if (sw_mass) *sw_mass = d[3];
    return MCLBM_OK;
}

int mclbm_capillary_pressure(mclbm_lattice *lat, double *pc, double *p_in, double *p_out) {
    double d[8];
    if (int rc = mclbm_diagnostics(lat, d)) return rc;
    if (pc) *pc = d[6];
    if (p_in) *p_in = d[4];
    if (p_out) *p_out = d[5];
    return MCLBM_OK;
}

int mclbm_mass(mclbm_lattice *lat, double out[2]) {
    double d[8];
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    if (int rc = mclbm_diagnostics(lat, d)) return rc;
    out[0] = d[0];
    out[1] = d[1];
    return MCLBM_OK;
}

int mclbm_info(mclbm_lattice *lat, int64_t out[6]) {
    if (int rc = check_lat(lat)) return rc;
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    out[0] = lat->nx;
    out[1] = lat->ny;
    out[2] = lat->pitch;
    out[3] = lat->prec;
    out[4] = lat->steps;
    out[5] = (int64_t)lat->device_bytes;
    return MCLBM_OK;
}

int mclbm_fluid_layout_check(int nx, int ny, const uint8_t *codes, mclbm_precision prec, int tile_shape,
                             int open_x, int64_t out[8]) {
    if (nx < 1 || ny < 1 || (int64_t)nx * ny > (1LL << 30)) return fail(MCLBM_ERR_ARG, "lattice size out of range");
    if (!codes || !out) return fail(MCLBM_ERR_ARG, "codes or out is NULL");
    if (tile_shape != 0 && tile_shape != 1) return fail(MCLBM_ERR_ARG, "tile_shape must be 0 or 1");
    try {
        return sparse_layout_check(nx, ny, codes, prec, tile_shape, open_x != 0, out);
    } catch (const std::bad_alloc &) {
        return fail(MCLBM_ERR_NOMEM, "host memory for the layout check");
    }
}

}  // extern "C"
