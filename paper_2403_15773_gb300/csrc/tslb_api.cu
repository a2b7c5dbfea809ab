// Host side of the C ABI declared in include/tslb.h: contexts, argument
// checking, workspace layout, state I/O, graph-captured time stepping, FP64
// sums and checkpoints.  All compute runs in the kernels of tslb_step.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "tslb.h"
#include "tslb_internal.h"

using tslb::StepParams;

struct tslb_ctx {
    StepParams p;
    int storage = 0;
    size_t elem = 4;
    int device = 0;
    long long N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    void* buf[2] = {nullptr, nullptr};
    float* staging = nullptr;
    double* partials = nullptr;
    double* result = nullptr;
    long long* tdev = nullptr;
    int cur = 0;
    int64_t t = 0;
    bool have_state = false;
    int nparts = 0;
    bool parts_valid = false;
    int graph_steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int check_every = 0;
    int64_t since_check = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_init_err;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t state, staging, partials, result, tdev, total;
};

Layout layout_for(const StepParams& p, size_t elem, int storage) {
    Layout L;
    const size_t fs = (size_t)p.fstride;
    L.state = 0;
    size_t off = align256(tslb::NFIELDS * fs * elem) * 2;
    L.staging = off;
    off += align256(fs * sizeof(float));
    L.partials = off;
    off += align256((size_t)tslb::max_partials(p, storage) * 2 * sizeof(double));
    L.result = off;
    off += 256;
    L.tdev = off;
    off += 256;
    L.total = off;
    return L;
}

size_t elem_size(int storage) { return storage == TSLB_FP32 ? 4 : 2; }

int auto_tile_z(int nz) { return nz < 32 ? nz : 32; }

bool valid_grid(const tslb_grid* g, const int face[6], std::string& why) {
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        const int lo = face[2 * a], hi = face[2 * a + 1];
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) {
            why = "unknown face rule";
            return false;
        }
        if ((lo == TSLB_BC_PERIODIC) != (hi == TSLB_BC_PERIODIC)) {
            why = "a periodic face must be paired with a periodic face";
            return false;
        }
        if (n[a] < 1 || (lo != TSLB_BC_PERIODIC && n[a] < 2)) {
            why = "grid too small for its face rules (>= 1 periodic, >= 2 otherwise)";
            return false;
        }
    }
    for (int k = 0; k < 6; ++k)
        if (face[k] == TSLB_BC_INLET && k != 4) {
            why = "the inlet is only supported on the -z face";
            return false;
        }
    if ((long long)g->nx * g->ny * g->nz > (1ll << 40)) {
        why = "grid too large";
        return false;
    }
    if ((long long)g->nx * g->ny > (1ll << 31)) {
        why = "x-y plane too large";
        return false;
    }
    return true;
}

// Builds the kernel parameters; returns false with a reason on bad input.
bool make_params(const tslb_grid* grid, double omega, double sigma, const tslb_boundary* bc,
                 const tslb_options* opt, StepParams& p, std::string& why) {
    if (!grid) {
        why = "grid is NULL";
        return false;
    }
    tslb_boundary b;
    std::memset(&b, 0, sizeof(b));
    if (bc) b = *bc;
    if (!valid_grid(grid, b.face, why)) return false;
    if (!(omega > 0.0 && omega < 2.0)) {
        why = "omega must lie in (0, 2)";
        return false;
    }
    if (!(sigma >= 0.0) || !std::isfinite(sigma)) {
        why = "sigma must be finite and >= 0";
        return false;
    }
    if (!(opt->interface_width > 0.f) || !std::isfinite(opt->interface_width)) {
        why = "interface_width must be > 0";
        return false;
    }
    if (!(opt->normal_eps >= 0.f) || !std::isfinite(opt->normal_eps)) {
        why = "normal_eps must be >= 0";
        return false;
    }
    if (opt->storage < 0 || opt->storage > 2) {
        why = "unknown storage type";
        return false;
    }
    if (opt->tile_z < 0) {
        why = "tile_z must be >= 0";
        return false;
    }
    if (b.face[4] == TSLB_BC_INLET && !(b.inlet_diameter >= 0.f)) {
        why = "inlet_diameter must be >= 0";
        return false;
    }
    std::memset(&p, 0, sizeof(p));
    p.nx = grid->nx;
    p.ny = grid->ny;
    p.nz = grid->nz;
    for (int k = 0; k < 6; ++k) p.face[k] = b.face[k];
    p.tile_z = opt->tile_z > 0 ? (opt->tile_z < grid->nz ? opt->tile_z : grid->nz) : auto_tile_z(grid->nz);
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    p.fstride = (N + 63) / 64 * 64;
    p.omega = (float)omega;
    p.sigma = (float)sigma;
    p.gamma = 1.f / opt->interface_width;
    p.normal_eps2 = opt->normal_eps * opt->normal_eps;
    float umag = 0.f;
    for (int a = 0; a < 3; ++a) {
        p.inlet_u[a] = b.inlet_u[a];
        umag += b.inlet_u[a] * b.inlet_u[a];
    }
    p.inlet_umag = std::sqrt(umag);
    p.inlet_half_d = 0.5f * b.inlet_diameter;
    p.inlet_cx = b.inlet_cx;
    p.inlet_cy = b.inlet_cy;
    p.inlet_two_over_w = 2.f / opt->interface_width;
    p.noise_amp = b.noise_amp;
    p.seed_lo = (unsigned)(b.seed & 0xffffffffull);
    p.seed_hi = (unsigned)(b.seed >> 32);
    // 16-bit storage scales: rho - 1, u, P, phi
    const float U = p.inlet_umag > 0.f ? p.inlet_umag : 0.05f;
    const float def[4] = {1.f / (3.f * U * U), 1.f / (2.f * U), 1e3f, 1.f};
    float sc[4];
    for (int g = 0; g < 4; ++g) sc[g] = opt->field_scale[g] > 0.f ? opt->field_scale[g] : def[g];
    for (int f = 0; f < tslb::NFIELDS; ++f) {
        const int g = f == tslb::F_DRHO ? 0 : f <= tslb::F_UZ ? 1 : f <= tslb::F_PYZ ? 2 : 3;
        p.scale[f] = opt->storage == TSLB_FP32 ? 1.f : sc[g];
        p.inv_scale[f] = 1.f / p.scale[f];
    }
    return true;
}

tslb_status cuda_fail(tslb_ctx* c, cudaError_t e, const char* what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return TSLB_ERR_CUDA;
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

tslb_status bad(tslb_ctx* c, const char* why, tslb_status s = TSLB_ERR_INVALID_ARG) {
    c->err = why;
    return s;
}

// Device pointer kind check: on_device pointers must be device-accessible.
bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

tslb_status put_field(tslb_ctx* c, const float* src, int field, int on_device) {
    const float* dsrc = src;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->staging, src, (size_t)c->N * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "host-to-device copy");
        dsrc = c->staging;
    }
    CK(tslb::launch_put_field(c->p, c->storage, dsrc, field, c->buf[c->cur], c->stream), "field conversion");
    return TSLB_OK;
}

tslb_status get_field(tslb_ctx* c, float* dst, int field, int on_device) {
    float* ddst = on_device ? dst : c->staging;
    CK(tslb::launch_get_field(c->p, c->storage, c->buf[c->cur], field, ddst, c->stream), "field conversion");
    if (!on_device)
        CK(cudaMemcpyAsync(dst, c->staging, (size_t)c->N * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "device-to-host copy");
    return TSLB_OK;
}

tslb_status capture_graph(tslb_ctx* c, int parity) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    int q = parity;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < c->graph_steps && le == cudaSuccess; ++k) {
        le = tslb::launch_step(c->p, c->storage, c->buf[q], c->buf[q ^ 1], c->tdev + q, c->tdev + (q ^ 1),
                               c->partials, c->stream);
        q ^= 1;
    }
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(c, le != cudaSuccess ? le : ee, "graph capture");
    }
    cudaError_t ie = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph[parity] = nullptr;
        return cuda_fail(c, ie, "graph instantiate");
    }
    return TSLB_OK;
}

tslb_status finish_sums(tslb_ctx* c, double* mass, double* phi_total) {
    if (!c->parts_valid) {
        CK(tslb::launch_state_sums(c->p, c->storage, c->buf[c->cur], c->partials, &c->nparts, c->stream),
           "state sums");
        c->parts_valid = true;
    }
    CK(tslb::launch_finish_sums(c->partials, c->nparts, c->result, c->stream), "sum reduction");
    double r[2];
    CK(cudaMemcpyAsync(r, c->result, sizeof(r), cudaMemcpyDeviceToHost, c->stream), "sums copy");
    CK(cudaStreamSynchronize(c->stream), "sums synchronise");
    *mass = (double)c->N + r[0];
    *phi_total = r[1];
    if (!std::isfinite(*mass) || !std::isfinite(*phi_total))
        return bad(c, "total mass or phase field is not finite", TSLB_ERR_UNSTABLE);
    return TSLB_OK;
}

}  // namespace

namespace tslb {
void set_global_error(const char* msg) { g_init_err = msg ? msg : ""; }
}  // namespace tslb

extern "C" {

void tslb_default_options(tslb_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->storage = TSLB_FP32;
    opt->interface_width = 3.f;
    opt->normal_eps = 1e-2f;
    opt->check_every = 0;
    opt->tile_z = 0;
    opt->graph_steps = 0;
    opt->cuda_stream = nullptr;
}

size_t tslb_workspace_bytes(const tslb_grid* grid, const tslb_options* opt) {
    tslb_options o;
    tslb_default_options(&o);
    if (opt) o = *opt;
    tslb_boundary b;
    std::memset(&b, 0, sizeof(b));
    StepParams p;
    std::string why;
    // the face rules only affect validity, not the size: check with periodic faces
    if (!make_params(grid, 1.0, 0.0, &b, &o, p, why)) return 0;
    return layout_for(p, elem_size(o.storage), o.storage).total;
}

tslb_status tslb_init(tslb_ctx** out, const tslb_grid* grid, tslb_lattice lattice, double omega, double sigma,
                      const tslb_boundary* bc, const tslb_options* opt, void* workspace, size_t workspace_bytes) {
    if (!out) {
        g_init_err = "out is NULL";
        return TSLB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (lattice != TSLB_LATTICE_D3Q27_D3Q7) {
        g_init_err = "unknown lattice";
        return TSLB_ERR_INVALID_ARG;
    }
    tslb_options o;
    tslb_default_options(&o);
    if (opt) o = *opt;
    StepParams p;
    std::string why;
    if (!make_params(grid, omega, sigma, bc, &o, p, why)) {
        g_init_err = why;
        return TSLB_ERR_INVALID_ARG;
    }
    tslb_ctx* c = new (std::nothrow) tslb_ctx();
    if (!c) {
        g_init_err = "host allocation failed";
        return TSLB_ERR_OOM;
    }
    c->p = p;
    c->storage = o.storage;
    c->elem = elem_size(o.storage);
    c->N = (long long)grid->nx * grid->ny * grid->nz;
    c->check_every = o.check_every > 0 ? o.check_every : 0;
    int gs = o.graph_steps > 0 ? o.graph_steps : 16;
    c->graph_steps = gs >= 2 ? gs & ~1 : 1;
    tslb_status st = TSLB_OK;
    auto fail = [&](tslb_status s) {
        g_init_err = c->err;
        tslb_destroy(c);
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        c->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return fail(TSLB_ERR_CUDA);
    }
    e = tslb::prepare_kernels(c->storage);
    if (e != cudaSuccess) {
        c->err = std::string("kernel set-up: ") + cudaGetErrorString(e);
        return fail(TSLB_ERR_CUDA);
    }
    if (o.cuda_stream) {
        c->stream = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        e = cudaStreamCreate(&c->stream);  // blocking: ordered with the legacy default stream
        if (e != cudaSuccess) {
            c->err = std::string("stream create: ") + cudaGetErrorString(e);
            return fail(TSLB_ERR_CUDA);
        }
        c->own_stream = true;
    }
    const Layout L = layout_for(p, c->elem, c->storage);
    if (workspace) {
        if (workspace_bytes < L.total) {
            c->err = "workspace smaller than tslb_workspace_bytes()";
            return fail(TSLB_ERR_OOM);
        }
        if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
            c->err = "workspace must be 256-byte aligned";
            return fail(TSLB_ERR_INVALID_ARG);
        }
        c->ws = workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        e = cudaMalloc(&c->ws, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->ws = nullptr;
            c->err = std::string("device allocation of the workspace: ") + cudaGetErrorString(e);
            return fail(TSLB_ERR_OOM);
        }
        c->own_ws = true;
        c->ws_bytes = L.total;
    }
    char* base = static_cast<char*>(c->ws);
    c->buf[0] = base + L.state;
    c->buf[1] = base + L.state + align256(tslb::NFIELDS * (size_t)p.fstride * c->elem);
    c->staging = reinterpret_cast<float*>(base + L.staging);
    c->partials = reinterpret_cast<double*>(base + L.partials);
    c->result = reinterpret_cast<double*>(base + L.result);
    c->tdev = reinterpret_cast<long long*>(base + L.tdev);
    (void)st;
    *out = c;
    return TSLB_OK;
}

tslb_status tslb_set_state(tslb_ctx* c, const float* rho, const float* u, const float* pi, const float* phi,
                           int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!rho || !u || !phi) return bad(c, "rho, u and phi are required");
    if (on_device && (!is_device_ptr(rho) || !is_device_ptr(u) || !is_device_ptr(phi) ||
                      (pi && !is_device_ptr(pi))))
        return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    c->cur = 0;
    const long long N = c->N;
    tslb_status s;
    if ((s = put_field(c, rho, tslb::F_DRHO, on_device)) != TSLB_OK) return s;
    for (int a = 0; a < 3; ++a)
        if ((s = put_field(c, u + a * N, tslb::F_UX + a, on_device)) != TSLB_OK) return s;
    if (pi) {
        for (int k = 0; k < 6; ++k)
            if ((s = put_field(c, pi + k * N, tslb::F_PXX + k, on_device)) != TSLB_OK) return s;
    } else {
        char* b0 = static_cast<char*>(c->buf[0]);
        CK(cudaMemsetAsync(b0 + (size_t)tslb::F_PXX * c->p.fstride * c->elem, 0, 6 * (size_t)c->p.fstride * c->elem,
                           c->stream),
           "zero P");
    }
    if ((s = put_field(c, phi, tslb::F_PHI, on_device)) != TSLB_OK) return s;
    CK(cudaMemsetAsync(c->tdev, 0, 2 * sizeof(long long), c->stream), "step counter");
    c->t = 0;
    c->have_state = true;
    c->parts_valid = false;
    c->since_check = 0;
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "set_state synchronise");  // staging reuse
    return TSLB_OK;
}

tslb_status tslb_step(tslb_ctx* c, int64_t n) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (n < 0) return bad(c, "n must be >= 0");
    if (!c->have_state) return bad(c, "tslb_step before tslb_set_state", TSLB_ERR_STATE);
    CK(cudaSetDevice(c->device), "set device");
    while (n > 0) {
        int64_t chunk = n;
        if (c->check_every > 0) {
            const int64_t left = c->check_every - c->since_check;
            if (chunk > left) chunk = left;
        }
        int64_t done = 0;
        while (chunk - done >= c->graph_steps && c->graph_steps > 1) {
            if (!c->graph[c->cur]) {
                tslb_status s = capture_graph(c, c->cur);
                if (s != TSLB_OK) {
                    c->graph_steps = 1;  // fall back to plain launches
                    cudaGetLastError();
                    c->err.clear();
                    break;
                }
            }
            CK(cudaGraphLaunch(c->graph[c->cur], c->stream), "graph launch");
            done += c->graph_steps;
            c->launches += c->graph_steps;
        }
        for (; done < chunk; ++done) {
            const int q = c->cur;
            CK(tslb::launch_step(c->p, c->storage, c->buf[q], c->buf[q ^ 1], c->tdev + q, c->tdev + (q ^ 1),
                                 c->partials, c->stream),
               "step launch");
            c->cur ^= 1;
            c->launches += 1;
        }
        // graphs hold an even number of steps, so only plain launches flip cur
        c->t += chunk;
        n -= chunk;
        const tslb::LaunchShape sh = tslb::step_shape(c->p, c->storage);
        c->nparts = (int)(sh.grid.x * sh.grid.y * sh.grid.z);
        c->parts_valid = true;
        if (c->check_every > 0) {
            c->since_check += chunk;
            if (c->since_check >= c->check_every) {
                c->since_check = 0;
                double m, ph;
                tslb_status s = finish_sums(c, &m, &ph);
                if (s != TSLB_OK) return s;
            }
        }
    }
    return TSLB_OK;
}

tslb_status tslb_get_moments(tslb_ctx* c, float* rho, float* u, float* pi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!c->have_state) return bad(c, "no state", TSLB_ERR_STATE);
    if (on_device && ((rho && !is_device_ptr(rho)) || (u && !is_device_ptr(u)) || (pi && !is_device_ptr(pi))))
        return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const long long N = c->N;
    tslb_status s;
    if (rho && (s = get_field(c, rho, tslb::F_DRHO, on_device)) != TSLB_OK) return s;
    for (int a = 0; u && a < 3; ++a)
        if ((s = get_field(c, u + a * N, tslb::F_UX + a, on_device)) != TSLB_OK) return s;
    for (int k = 0; pi && k < 6; ++k)
        if ((s = get_field(c, pi + k * N, tslb::F_PXX + k, on_device)) != TSLB_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "get_moments synchronise");
    return TSLB_OK;
}

tslb_status tslb_get_phi(tslb_ctx* c, float* phi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!c->have_state) return bad(c, "no state", TSLB_ERR_STATE);
    if (!phi) return bad(c, "phi is NULL");
    if (on_device && !is_device_ptr(phi)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    tslb_status s = get_field(c, phi, tslb::F_PHI, on_device);
    if (s != TSLB_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "get_phi synchronise");
    return TSLB_OK;
}

tslb_status tslb_sums(tslb_ctx* c, double* mass, double* phi_total) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!mass || !phi_total) return bad(c, "mass and phi_total are required");
    if (!c->have_state) return bad(c, "no state", TSLB_ERR_STATE);
    CK(cudaSetDevice(c->device), "set device");
    return finish_sums(c, mass, phi_total);
}

tslb_status tslb_get_time(const tslb_ctx* c, int64_t* t) {
    if (!c || !t) return TSLB_ERR_INVALID_ARG;
    *t = c->t;
    return TSLB_OK;
}

size_t tslb_state_bytes(const tslb_ctx* c) {
    if (!c) return 0;
    return (size_t)tslb::NFIELDS * (size_t)c->N * c->elem + sizeof(int64_t);
}

tslb_status tslb_get_state(tslb_ctx* c, void* dst, int on_device) {
    if (!c || !dst) return TSLB_ERR_INVALID_ARG;
    if (!c->have_state) return bad(c, "no state", TSLB_ERR_STATE);
    if (on_device && !is_device_ptr(dst)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const size_t fb = (size_t)c->N * c->elem;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int f = 0; f < tslb::NFIELDS; ++f)
        CK(cudaMemcpyAsync(static_cast<char*>(dst) + f * fb,
                           static_cast<const char*>(c->buf[c->cur]) + (size_t)f * c->p.fstride * c->elem, fb, kind,
                           c->stream),
           "state copy");
    int64_t t = c->t;
    if (on_device)
        CK(cudaMemcpyAsync(static_cast<char*>(dst) + tslb::NFIELDS * fb, &t, sizeof(t), cudaMemcpyHostToDevice,
                           c->stream),
           "step copy");
    CK(cudaStreamSynchronize(c->stream), "get_state synchronise");
    if (!on_device) std::memcpy(static_cast<char*>(dst) + tslb::NFIELDS * fb, &t, sizeof(t));
    return TSLB_OK;
}

tslb_status tslb_put_state(tslb_ctx* c, const void* src, int on_device) {
    if (!c || !src) return TSLB_ERR_INVALID_ARG;
    if (on_device && !is_device_ptr(src)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const size_t fb = (size_t)c->N * c->elem;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->cur = 0;
    for (int f = 0; f < tslb::NFIELDS; ++f)
        CK(cudaMemcpyAsync(static_cast<char*>(c->buf[0]) + (size_t)f * c->p.fstride * c->elem,
                           static_cast<const char*>(src) + f * fb, fb, kind, c->stream),
           "state copy");
    int64_t t = 0;
    if (on_device)
        CK(cudaMemcpyAsync(&t, static_cast<const char*>(src) + tslb::NFIELDS * fb, sizeof(t), cudaMemcpyDeviceToHost,
                           c->stream),
           "step copy");
    else
        std::memcpy(&t, static_cast<const char*>(src) + tslb::NFIELDS * fb, sizeof(t));
    CK(cudaStreamSynchronize(c->stream), "put_state synchronise");
    if (t < 0) return bad(c, "negative step index in checkpoint");
    long long tt[2] = {(long long)t, (long long)t};
    CK(cudaMemcpyAsync(c->tdev, tt, sizeof(tt), cudaMemcpyHostToDevice, c->stream), "step counter");
    CK(cudaStreamSynchronize(c->stream), "put_state synchronise");
    c->t = t;
    c->have_state = true;
    c->parts_valid = false;
    c->since_check = 0;
    return TSLB_OK;
}

tslb_status tslb_synchronize(tslb_ctx* c) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    CK(cudaSetDevice(c->device), "set device");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    return TSLB_OK;
}

tslb_status tslb_destroy(tslb_ctx* c) {
    if (!c) return TSLB_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
    return TSLB_OK;
}

const char* tslb_last_error(const tslb_ctx* c) {
    if (!c) return g_init_err.c_str();
    return c->err.c_str();
}

const char* tslb_status_string(tslb_status s) {
    switch (s) {
        case TSLB_OK: return "ok";
        case TSLB_ERR_INVALID_ARG: return "invalid argument";
        case TSLB_ERR_OOM: return "out of memory";
        case TSLB_ERR_CUDA: return "CUDA error";
        case TSLB_ERR_UNSTABLE: return "unstable (non-finite sums)";
        case TSLB_ERR_TIMEOUT: return "timeout";
        case TSLB_ERR_STATE: return "bad call order";
        default: return "unknown status";
    }
}

int64_t tslb_kernel_launches(const tslb_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
