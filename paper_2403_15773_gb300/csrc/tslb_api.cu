// Host side of the C ABI declared in include/tslb.h: contexts (one grid or a
// batch of independent grids), argument checking, workspace layout, state
// I/O, graph-captured time stepping, FP64 sums, checkpoints and the tile-shape
// autotuner.  All compute runs in the kernels of tslb_step.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tslb.h"
#include "tslb_internal.h"

using tslb::StepParams;

namespace {

// A named range on the profiler timeline (NVTX) around an entry point's host
// side (the GPU work it enqueues runs later, on the context's stream);
// without a profiler attached the push and pop do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// One grid of a context: its parameters, node count and its two state buffers.
struct Instance {
    StepParams p;
    long long N = 0;
    void* buf[2] = {nullptr, nullptr};
    double* avg = nullptr;  // time sums of phi and u_z (option `average`)
    int tile_begin = 0, tile_end = 0;  // batch: its tiles in the tile list
    bool set = false;
    tslb::TileMaps maps[2] = {};       // TMA tensor maps of the steps from buf[q] (made on first use)
};

}  // namespace

struct tslb_ctx {
    int storage = 0;
    size_t elem = 4;
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    std::vector<Instance> inst;
    bool batch = false;
    int batch_nw = 8;
    bool batch_plain = false;
    bool batch_wrap = false;  // some instance has the side-box maps of periodic faces
    int batch_tma12 = -1;     // every tile of every instance loads by TMA in the 12-warp staged-store
                              // form: 1 / 0, -1 not yet classified
    bool per_tile_loads = false;  // option per_tile_loads: no one-load-path forms
    float* staging = nullptr;
    double* partials = nullptr;   // step partials; state-sum partials after max_tiles
    int max_tiles = 0;
    double* result = nullptr;
    long long* tdev = nullptr;
    int* counters = nullptr;
    tslb::BatchInstance* dinst = nullptr;
    int4* dtiles = nullptr;
    int ntiles = 0;
    int cur = 0;
    int64_t t = 0;
    bool parts_valid = false;  // step partials describe the current state
    int graph_steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int check_every = 0;
    int64_t since_check = 0;
    int64_t launches = 0;
    bool average = false;
    int64_t avg_steps = 0;
    int scheme = 0;          // 0 fused moment-only step, 1 the paper's two-sweep design
    float* pops = nullptr;   // scheme 1: 34 population arrays
    bool tma12[2] = {false, false};  // every tile loads by TMA in the 12-warp form, without / with the
                                     // periodic-face side boxes (tslb::tiles_all_tma at set-up)
    std::string err;
};

namespace {

thread_local std::string g_init_err;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t elem_size(int storage) { return storage == TSLB_FP32 ? 4 : 2; }

// Interior columns of a tile (every step kernel).
int default_tile_width(const tslb_options*) { return 28; }

// SMs of the current device (152 if it cannot be queried).
int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || n <= 0) {
        cudaGetLastError();
        return 152;
    }
    return n;
}

// Default slab depth for blocks of nw warps and tiles tx columns wide: the
// depth (8 .. 128 planes) that minimises (waves of one block per SM) x
// (planes a block marches, its slab plus two halo planes), i.e. the time of
// the last block to finish when every block takes the same time per plane.
int auto_tile_z(const tslb_grid* g, int nw, int tx, int sms) {
    const long long txy = (long long)((g->nx + tx - 1) / tx) * ((g->ny + 2 * nw - 3) / (2 * nw - 2));
    int best = g->nz < 64 ? g->nz : 64;
    long long best_cost = -1;
    for (int tz = 8; tz <= 128; ++tz) {
        const int d = tz < g->nz ? tz : g->nz;
        const long long blocks = txy * ((g->nz + d - 1) / d);
        const long long cost = ((blocks + sms - 1) / sms) * (d + 2);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && d > best)) {
            best_cost = cost;
            best = d;
        }
        if (d == g->nz) break;
    }
    return best;
}

constexpr int kAutotuneTileZ[] = {16, 24, 32, 48, 64};
constexpr int kMinTileZ = 16;  // smallest slab the batch tile list is sized for

bool valid_grid(const tslb_grid* g, const int face[6], std::string& why) {
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        const int lo = face[2 * a], hi = face[2 * a + 1];
        if (lo < 0 || lo > 4 || hi < 0 || hi > 4) {
            why = "unknown face rule";
            return false;
        }
        if (a < 2 && (lo == TSLB_BC_HALO || hi == TSLB_BC_HALO)) {
            why = "the halo rule is only supported on the z faces";
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
    if (opt->block_warps != 0 && opt->block_warps != 8 && opt->block_warps != 12 && opt->block_warps != 14 &&
        opt->block_warps != 16) {
        why = "block_warps must be 0, 8, 12, 14 or 16";
        return false;
    }
    if (opt->closure != TSLB_CLOSURE_PROJECTION && opt->closure != TSLB_CLOSURE_CHAPMAN_ENSKOG) {
        why = "unknown closure";
        return false;
    }
    if (opt->closure == TSLB_CLOSURE_CHAPMAN_ENSKOG && opt->block_warps > 12) {
        why = "the Chapman-Enskog closure runs blocks of 8 or 12 warps";
        return false;
    }
    if (opt->test_tma_stall < 0 || opt->test_tma_stall > 2) {
        why = "test_tma_stall must be 0, 1 or 2";
        return false;
    }
    if (opt->plain_stores != 0 && opt->plain_stores != 1) {
        why = "plain_stores must be 0 or 1";
        return false;
    }
    if (opt->per_tile_loads != 0 && opt->per_tile_loads != 1) {
        why = "per_tile_loads must be 0 or 1";
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
    p.block_warps = opt->block_warps > 0 ? opt->block_warps : 12;
    p.closure = opt->closure;
    p.test_stall = opt->test_tma_stall;
    p.plain_stores = opt->plain_stores;
    p.tile_z = opt->tile_z > 0 ? (opt->tile_z < grid->nz ? opt->tile_z : grid->nz)
                               : auto_tile_z(grid, p.block_warps, default_tile_width(opt), device_sms());
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    const long long halo = tslb::has_halo(p.face) ? (long long)tslb::kHaloPlanes * grid->nx * grid->ny : 0;
    p.fstride = (N + halo + 63) / 64 * 64;
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

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
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

// Tiles of one grid for a block of `nw` warps and slabs of `tile_z` planes
// (the tile width depends on the storage type).
int tiles_of(const StepParams& p, int storage, int nw, int tile_z) {
    StepParams q = p;
    q.block_warps = nw;
    q.tile_z = std::min(tile_z, p.nz);
    const tslb::LaunchShape sh = tslb::step_shape(q, storage);
    return (int)(sh.grid.x * sh.grid.y * sh.grid.z);
}

// Workspace layout.  Per grid: two state buffers.  Shared: one staging field
// for host I/O, FP64 partials (step tiles, then state-sum blocks), the result
// pair, the two-slot step counter, the two batch tile counters, and for a
// batch the device copy of the instances and the tile list.
struct Layout {
    std::vector<size_t> state, avg;
    size_t staging, partials, result, tdev, counters, dinst, dtiles, pops, total;
    int max_tiles, max_conv;
};

Layout layout_for(const std::vector<StepParams>& ps, size_t elem, int storage, bool batch, bool average,
                  int scheme = 0) {
    Layout L;
    size_t off = 0;
    long long maxf = 0;
    int tiles = 0, conv = 0;
    for (const StepParams& p : ps) {
        L.state.push_back(off);
        off += 2 * align256(tslb::stored_fields(p.closure) * (size_t)p.fstride * elem);
        L.avg.push_back(off);
        if (average) off += align256(2 * (size_t)p.fstride * sizeof(double));
        maxf = std::max(maxf, p.fstride);
        if (batch)
            tiles += tiles_of(p, storage, 8, std::min(p.tile_z, kMinTileZ));
        else
            tiles = std::max(tiles, tslb::max_partials(p, storage));
        conv = std::max(conv, tslb::max_partials(p, storage));
        if (scheme == 1) conv = std::max(conv, tslb::twosweep_partials(p));
    }
    L.max_tiles = tiles;
    L.max_conv = conv;
    L.staging = off;
    off += align256((size_t)maxf * sizeof(float));
    L.partials = off;
    off += align256((size_t)(tiles + conv) * 2 * sizeof(double));
    L.result = off;
    off += 256;
    L.tdev = off;
    off += 256;
    L.counters = off;
    off += 256;
    L.dinst = off;
    off += batch ? align256(ps.size() * sizeof(tslb::BatchInstance)) : 0;
    L.dtiles = off;
    off += batch ? align256((size_t)tiles * sizeof(int4)) : 0;
    L.pops = off;
    if (scheme == 1) off += align256(34 * (size_t)ps[0].fstride * sizeof(float));
    L.total = off;
    return L;
}

// Device address through which kernels reach host memory at `p` directly
// (page-locked host memory, mapped into the device's address space), or
// null for pageable memory (which goes through the staging field).
const void* mapped_host_alias(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// One caller field into the state.  Device memory and page-locked host memory
// are read by the conversion kernel itself (the latter over the host link,
// without a staging copy); pageable host memory is copied to the staging
// field first.
tslb_status put_field(tslb_ctx* c, Instance& I, const float* src, int field, int on_device) {
    const float* dsrc = src;
    if (!on_device) {
        dsrc = static_cast<const float*>(mapped_host_alias(src));
        if (!dsrc) {
            CK(cudaMemcpyAsync(c->staging, src, (size_t)I.N * sizeof(float), cudaMemcpyHostToDevice, c->stream),
               "host-to-device copy");
            dsrc = c->staging;
        }
    }
    CK(tslb::launch_put_field(I.p, c->storage, dsrc, field, I.buf[c->cur], c->stream), "field conversion");
    return TSLB_OK;
}

// One state field out to the caller: the conversion kernel writes device
// memory or page-locked host memory directly, pageable host memory through
// the staging field.
tslb_status get_field(tslb_ctx* c, Instance& I, float* dst, int field, int on_device) {
    float* ddst = dst;
    bool staged = false;
    if (!on_device) {
        ddst = static_cast<float*>(const_cast<void*>(mapped_host_alias(dst)));
        if (!ddst) {
            ddst = c->staging;
            staged = true;
        }
    }
    CK(tslb::launch_get_field(I.p, c->storage, I.buf[c->cur], field, ddst, c->stream), "field conversion");
    if (staged)
        CK(cudaMemcpyAsync(dst, c->staging, (size_t)I.N * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "device-to-host copy");
    return TSLB_OK;
}

// Builds the batch tile list for the current block shape and slab depth and
// uploads it with the instances (synchronous: pageable host memory).
tslb_status upload_batch(tslb_ctx* c) {
    std::vector<int4> tiles;
    std::vector<tslb::BatchInstance> di(c->inst.size());
    for (size_t i = 0; i < c->inst.size(); ++i) {
        Instance& I = c->inst[i];
        I.p.block_warps = c->batch_nw;
        I.p.plain_stores = c->batch_plain ? 1 : 0;
        const tslb::LaunchShape sh = tslb::step_shape(I.p, c->storage);
        I.tile_begin = (int)tiles.size();
        for (unsigned bz = 0; bz < sh.grid.z; ++bz)
            for (unsigned by = 0; by < sh.grid.y; ++by)
                for (unsigned bx = 0; bx < sh.grid.x; ++bx) tiles.push_back(make_int4((int)i, bx, by, bz));
        I.tile_end = (int)tiles.size();
        di[i].p = I.p;
        di[i].buf[0] = I.buf[0];
        di[i].buf[1] = I.buf[1];
        for (int q = 0; q < 2; ++q)
            CK(tslb::make_tile_maps(I.p, c->storage, I.buf[q], I.buf[q ^ 1], &di[i].maps[q]), "batch tensor maps");
    }
    c->batch_wrap = false;
    for (const tslb::BatchInstance& b : di) c->batch_wrap = c->batch_wrap || (b.maps[0].wrap && b.maps[1].wrap);
    if (c->batch_tma12 < 0 && c->batch_nw == 12 && !c->batch_plain && !c->per_tile_loads) {
        // which batches the kernel compiled for TMA tile loads alone may run (an
        // instance without side-box maps is classified as the kernel sees it)
        bool all = true;
        for (size_t i = 0; i < di.size() && all; ++i) {
            bool ok = false;
            if (di[i].maps[0].valid && di[i].maps[1].valid)
                CK(tslb::tiles_all_tma(di[i].p, c->storage, c->batch_wrap && di[i].maps[0].wrap && di[i].maps[1].wrap,
                                       c->counters + 3, c->stream, &ok),
                   "tile classification");
            all = ok;
        }
        c->batch_tma12 = all ? 1 : 0;
    }
    if ((int)tiles.size() > c->max_tiles) return bad(c, "batch tile list exceeds its workspace");
    c->ntiles = (int)tiles.size();
    CK(cudaMemcpyAsync(c->dinst, di.data(), di.size() * sizeof(di[0]), cudaMemcpyHostToDevice, c->stream),
       "batch instances upload");
    CK(cudaMemcpyAsync(c->dtiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream),
       "batch tiles upload");
    CK(cudaStreamSynchronize(c->stream), "batch upload synchronise");
    return TSLB_OK;
}

// The tensor maps of a single grid's projection step from parity q, made
// for the current block size if they were made for another one, with
// all_tma set where the 12-warp form may run the kernel compiled for TMA
// tile loads alone (which keeps no time sums).
cudaError_t single_maps(tslb_ctx* c, int q, tslb::TileMaps** out) {
    Instance& I = c->inst[0];
    tslb::TileMaps& m = I.maps[q];
    if (m.block_warps != I.p.block_warps) {  // boxes are shaped for one block size
        cudaError_t e = tslb::make_tile_maps(I.p, c->storage, I.buf[q], I.buf[q ^ 1], &m);
        if (e != cudaSuccess) return e;
        m.block_warps = I.p.block_warps;
    }
    m.all_tma = m.valid && I.p.block_warps == 12 && !c->average && c->tma12[m.wrap ? 1 : 0] ? 1 : 0;
    *out = &m;
    return cudaSuccess;
}

// Whether a batch step launches the kernel compiled for TMA tile loads alone.
bool batch_tma_only(const tslb_ctx* c) {
    return c->batch_tma12 == 1 && c->batch_nw == 12 && !c->batch_plain && !c->average;
}

// One time step from parity q (state buf[q], step counter tdev[q]) to q ^ 1.
cudaError_t launch_one(tslb_ctx* c, int q) {
    if (c->scheme == 1) {
        Instance& I = c->inst[0];
        return tslb::launch_twosweep_step(I.p, static_cast<float*>(I.buf[0]), c->pops, c->tdev + q,
                                          c->tdev + (q ^ 1), c->partials, c->stream);
    }
    if (!c->batch && c->inst[0].p.closure == tslb::CL_CHAPMAN_ENSKOG) {
        Instance& I = c->inst[0];
        tslb::TileMaps& m = I.maps[q];
        if (m.block_warps != I.p.block_warps) {  // the output box is shaped for one block size
            cudaError_t e = tslb::make_tile_maps(I.p, c->storage, I.buf[q], I.buf[q ^ 1], &m);
            if (e != cudaSuccess) return e;
            m.block_warps = I.p.block_warps;
        }
        return tslb::launch_step_ce(I.p, c->storage, I.buf[q], I.buf[q ^ 1], c->tdev + q, c->tdev + (q ^ 1),
                                    c->partials, c->stream, &m);
    }
    if (!c->batch) {
        Instance& I = c->inst[0];
        tslb::TileMaps* m = nullptr;
        cudaError_t e = single_maps(c, q, &m);
        if (e != cudaSuccess) return e;
        return tslb::launch_step(I.p, c->storage, I.buf[q], I.buf[q ^ 1], c->tdev + q, c->tdev + (q ^ 1),
                                 c->partials, c->stream, m);
    }
    return tslb::launch_batch_step(c->batch_nw, c->batch_plain, c->batch_wrap, batch_tma_only(c), c->dinst,
                                   c->dtiles, c->ntiles, q,
                                   c->tdev + q, c->tdev + (q ^ 1), c->counters, c->partials, c->sms, c->stream);
}

// One autotuner trial launch: the step from parity q again.  A batch launch
// takes its tiles from the tile counter of its parity and only rearms the
// other one (for the next step), so a repeated launch of the same parity
// first resets its own.
cudaError_t trial_launch(tslb_ctx* c, int q) {
    if (c->batch) {
        const cudaError_t e = cudaMemsetAsync(c->counters + q, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
    }
    return launch_one(c, q);
}

void drop_graphs(tslb_ctx* c) {
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
}

tslb_status capture_graph(tslb_ctx* c, int parity) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    int q = parity;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < c->graph_steps && le == cudaSuccess; ++k) {
        le = launch_one(c, q);
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

// FP64 totals of one grid: from the step partials when they describe the
// current state, else from a reduction of the stored fields.
tslb_status finish_sums(tslb_ctx* c, int i, double* mass, double* phi_total) {
    Instance& I = c->inst[i];
    const double* parts = c->partials;
    int n = 0;
    if (c->parts_valid) {
        if (c->batch) {
            parts = c->partials + 2 * (size_t)I.tile_begin;
            n = I.tile_end - I.tile_begin;
        } else if (c->scheme == 1) {
            n = tslb::twosweep_partials(I.p);
        } else {
            n = tiles_of(I.p, c->storage, I.p.block_warps, I.p.tile_z);
        }
    } else {
        double* sp = c->partials + 2 * (size_t)c->max_tiles;
        CK(tslb::launch_state_sums(I.p, c->storage, I.buf[c->cur], sp, &n, c->stream), "state sums");
        parts = sp;
    }
    CK(tslb::launch_finish_sums(parts, n, c->result, c->stream), "sum reduction");
    double r[2];
    int err = 0;
    CK(cudaMemcpyAsync(r, c->result, sizeof(r), cudaMemcpyDeviceToHost, c->stream), "sums copy");
    CK(cudaMemcpyAsync(&err, c->counters + 2, sizeof(err), cudaMemcpyDeviceToHost, c->stream), "error word copy");
    CK(cudaStreamSynchronize(c->stream), "sums synchronise");
    if (err == 2)
        return bad(c, "internal: a step kernel compiled for TMA tile loads met a tile that loads element by element",
                   TSLB_ERR_CUDA);
    if (err) return bad(c, "a step kernel gave up waiting for its tile data (bounded wait expired)", TSLB_ERR_TIMEOUT);
    *mass = (double)I.N + r[0];
    *phi_total = r[1];
    if (!std::isfinite(*mass) || !std::isfinite(*phi_total))
        return bad(c, "total mass or phase field is not finite", TSLB_ERR_UNSTABLE);
    return TSLB_OK;
}

tslb_status check_instance(tslb_ctx* c, int i) {
    if (i < 0 || i >= (int)c->inst.size()) return bad(c, "instance index out of range");
    return TSLB_OK;
}

// Creates a context for `count` grids (count == 1: one grid, no batch).
tslb_status create(tslb_ctx** out, int count, const tslb_grid* grids, tslb_lattice lattice, const double* omega,
                   const double* sigma, const tslb_boundary* bcs, const tslb_options* opt, void* workspace,
                   size_t workspace_bytes, bool batch) {
    if (!out) {
        g_init_err = "out is NULL";
        return TSLB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (lattice != TSLB_LATTICE_D3Q27_D3Q7) {
        g_init_err = "unknown lattice";
        return TSLB_ERR_INVALID_ARG;
    }
    if (count < 1 || !grids || !omega || !sigma) {
        g_init_err = "count >= 1 and grids, omega, sigma are required";
        return TSLB_ERR_INVALID_ARG;
    }
    tslb_options o;
    tslb_default_options(&o);
    if (opt) o = *opt;
    if (batch && o.storage != TSLB_FP32) {
        g_init_err = "batches use FP32 storage";
        return TSLB_ERR_INVALID_ARG;
    }
    if (batch && o.block_warps != 0 && o.block_warps != 8 && o.block_warps != 12) {
        g_init_err = "batches use blocks of 8 or 12 warps";
        return TSLB_ERR_INVALID_ARG;
    }
    if (o.scheme != 0 && o.scheme != 1) {
        g_init_err = "scheme must be 0 (fused) or 1 (two sweeps)";
        return TSLB_ERR_INVALID_ARG;
    }
    if (o.scheme == 1 && (batch || o.storage != TSLB_FP32 || o.average)) {
        g_init_err = "the two-sweep scheme runs single grids in FP32 without averages";
        return TSLB_ERR_INVALID_ARG;
    }
    if (o.closure == TSLB_CLOSURE_CHAPMAN_ENSKOG && (batch || o.scheme != 0)) {
        g_init_err = "the Chapman-Enskog closure runs single grids with the fused scheme";
        return TSLB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < count && bcs; ++i)
        if ((bcs[i].face[4] == TSLB_BC_HALO || bcs[i].face[5] == TSLB_BC_HALO) &&
            (batch || o.scheme != 0 || o.closure != TSLB_CLOSURE_PROJECTION)) {
            g_init_err = "halo faces (slabs of a z-split domain) run single grids, fused scheme, projection closure";
            return TSLB_ERR_INVALID_ARG;
        }
    std::vector<StepParams> ps(count);
    for (int i = 0; i < count; ++i) {
        std::string why;
        if (!make_params(&grids[i], omega[i], sigma[i], bcs ? &bcs[i] : nullptr, &o, ps[i], why)) {
            g_init_err = count > 1 ? "grid " + std::to_string(i) + ": " + why : why;
            return TSLB_ERR_INVALID_ARG;
        }
        if (batch) ps[i].tile_z = o.tile_z > 0 ? std::min(o.tile_z, grids[i].nz) : std::min(64, grids[i].nz);
    }
    tslb_ctx* c = new (std::nothrow) tslb_ctx();
    if (!c) {
        g_init_err = "host allocation failed";
        return TSLB_ERR_OOM;
    }
    c->storage = o.storage;
    c->elem = elem_size(o.storage);
    c->batch = batch;
    c->batch_nw = o.block_warps > 0 ? o.block_warps : 8;
    c->batch_plain = o.plain_stores != 0;
    c->per_tile_loads = o.per_tile_loads != 0;
    c->check_every = o.check_every > 0 ? o.check_every : 0;
    int gs = o.graph_steps > 0 ? o.graph_steps : 16;
    c->graph_steps = gs >= 2 ? gs & ~1 : 1;
    auto fail = [&](tslb_status s) {
        g_init_err = c->err;
        tslb_destroy(c);
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        c->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return fail(TSLB_ERR_CUDA);
    }
    e = tslb::prepare_kernels(c->storage);
    if (e == cudaSuccess && o.closure == TSLB_CLOSURE_CHAPMAN_ENSKOG) e = tslb::prepare_kernels_ce(c->storage);
    if (e == cudaSuccess && batch) e = tslb::prepare_batch_kernels();
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
    c->average = o.average != 0;
    c->scheme = o.scheme;
    const Layout L = layout_for(ps, c->elem, c->storage, batch, c->average, c->scheme);
    if (workspace) {
        if (workspace_bytes < L.total) {
            c->err = "workspace smaller than the workspace-bytes query";
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
    c->inst.resize(count);
    for (int i = 0; i < count; ++i) {
        Instance& I = c->inst[i];
        I.p = ps[i];
        I.N = (long long)grids[i].nx * grids[i].ny * grids[i].nz;
        I.buf[0] = base + L.state[i];
        I.buf[1] = base + L.state[i] + align256(tslb::stored_fields(ps[i].closure) * (size_t)ps[i].fstride * c->elem);
        if (c->average) {
            I.avg = reinterpret_cast<double*>(base + L.avg[i]);
            I.p.avg = I.avg;
        }
    }
    c->staging = reinterpret_cast<float*>(base + L.staging);
    c->partials = reinterpret_cast<double*>(base + L.partials);
    c->max_tiles = L.max_tiles;
    c->result = reinterpret_cast<double*>(base + L.result);
    c->tdev = reinterpret_cast<long long*>(base + L.tdev);
    c->counters = reinterpret_cast<int*>(base + L.counters);  // [0..1] batch tile counters, [2] error word,
                                                               // [3] tile classification flag
    for (Instance& I : c->inst) I.p.err = c->counters + 2;
    c->dinst = reinterpret_cast<tslb::BatchInstance*>(base + L.dinst);
    c->dtiles = reinterpret_cast<int4*>(base + L.dtiles);
    if (c->scheme == 1) {
        c->pops = reinterpret_cast<float*>(base + L.pops);
        c->inst[0].buf[1] = c->inst[0].buf[0];  // the moments are updated in place
    }
    e = cudaMemsetAsync(c->counters, 0, 256, c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("counter reset: ") + cudaGetErrorString(e);
        return fail(TSLB_ERR_CUDA);
    }
    if (batch) {
        tslb_status s = upload_batch(c);
        if (s != TSLB_OK) return fail(s);
    } else if (c->scheme == 0 && !c->per_tile_loads) {
        // which grids the step kernel compiled for TMA tile loads alone may run
        const StepParams& p = c->inst[0].p;
        const bool periodic = p.face[0] == tslb::BC_PERIODIC || p.face[2] == tslb::BC_PERIODIC;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            if (w == 0 || (periodic && c->storage == TSLB_FP32))
                e = tslb::tiles_all_tma(p, c->storage, w == 1, c->counters + 3, c->stream, &c->tma12[w]);
        if (e != cudaSuccess) {
            c->err = std::string("tile classification: ") + cudaGetErrorString(e);
            return fail(TSLB_ERR_CUDA);
        }
    }
    *out = c;
    return TSLB_OK;
}

tslb_status set_state_of(tslb_ctx* c, int i, const float* rho, const float* u, const float* pi, const float* phi,
                         int on_device) {
    if (!rho || !u || !phi) return bad(c, "rho, u and phi are required");
    if (on_device && (!is_device_ptr(rho) || !is_device_ptr(u) || !is_device_ptr(phi) ||
                      (pi && !is_device_ptr(pi))))
        return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    Instance& I = c->inst[i];
    const long long N = I.N;
    tslb_status s;
    if ((s = put_field(c, I, rho, tslb::F_DRHO, on_device)) != TSLB_OK) return s;
    for (int a = 0; a < 3; ++a)
        if ((s = put_field(c, I, u + a * N, tslb::F_UX + a, on_device)) != TSLB_OK) return s;
    if (I.p.closure == tslb::CL_CHAPMAN_ENSKOG) {
        // P is not part of the state
    } else if (pi) {
        for (int k = 0; k < 6; ++k)
            if ((s = put_field(c, I, pi + k * N, tslb::F_PXX + k, on_device)) != TSLB_OK) return s;
    } else {
        char* b0 = static_cast<char*>(I.buf[c->cur]);
        CK(cudaMemsetAsync(b0 + (size_t)tslb::F_PXX * I.p.fstride * c->elem, 0,
                           6 * (size_t)I.p.fstride * c->elem, c->stream),
           "zero P");
    }
    if ((s = put_field(c, I, phi, tslb::F_PHI, on_device)) != TSLB_OK) return s;
    if (tslb::has_halo(I.p.face)) {  // ghost planes of halo faces: zero until the first tslb_halo_unpack
        const size_t nxy = (size_t)I.p.nx * I.p.ny;
        char* b0 = static_cast<char*>(I.buf[c->cur]);
        for (int f = 0; f < tslb::stored_fields(I.p.closure); ++f)
            CK(cudaMemsetAsync(b0 + ((size_t)f * I.p.fstride + (size_t)N) * c->elem, 0,
                               tslb::kHaloPlanes * nxy * c->elem, c->stream),
               "zero ghost planes");
    }
    if (I.avg) {
        CK(cudaMemsetAsync(I.avg, 0, 2 * (size_t)I.p.fstride * sizeof(double), c->stream), "clear averages");
        c->avg_steps = 0;
    }
    // the step index restarts with every state that is set
    long long tt[2] = {0, 0};
    CK(cudaMemcpyAsync(c->tdev, tt, sizeof(tt), cudaMemcpyHostToDevice, c->stream), "step counter");
    c->t = 0;
    I.set = true;
    c->parts_valid = false;
    c->since_check = 0;
    CK(cudaStreamSynchronize(c->stream), "set_state synchronise");  // staging and tt reuse
    return TSLB_OK;
}

tslb_status get_moments_of(tslb_ctx* c, int i, float* rho, float* u, float* pi, int on_device) {
    Instance& I = c->inst[i];
    if (!I.set) return bad(c, "no state", TSLB_ERR_STATE);
    if (on_device && ((rho && !is_device_ptr(rho)) || (u && !is_device_ptr(u)) || (pi && !is_device_ptr(pi))))
        return bad(c, "on_device pointers must be device memory");
    if (pi && I.p.closure == tslb::CL_CHAPMAN_ENSKOG)
        return bad(c, "the Chapman-Enskog closure stores no P: pi must be NULL");
    CK(cudaSetDevice(c->device), "set device");
    const long long N = I.N;
    tslb_status s;
    if (rho && (s = get_field(c, I, rho, tslb::F_DRHO, on_device)) != TSLB_OK) return s;
    for (int a = 0; u && a < 3; ++a)
        if ((s = get_field(c, I, u + a * N, tslb::F_UX + a, on_device)) != TSLB_OK) return s;
    for (int k = 0; pi && k < 6; ++k)
        if ((s = get_field(c, I, pi + k * N, tslb::F_PXX + k, on_device)) != TSLB_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "get_moments synchronise");
    return TSLB_OK;
}

tslb_status get_phi_of(tslb_ctx* c, int i, float* phi, int on_device) {
    Instance& I = c->inst[i];
    if (!I.set) return bad(c, "no state", TSLB_ERR_STATE);
    if (!phi) return bad(c, "phi is NULL");
    if (on_device && !is_device_ptr(phi)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    tslb_status s = get_field(c, I, phi, tslb::F_PHI, on_device);
    if (s != TSLB_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "get_phi synchronise");
    return TSLB_OK;
}

bool all_set(const tslb_ctx* c) {
    for (const Instance& I : c->inst)
        if (!I.set) return false;
    return true;
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
    opt->block_warps = 0;
    opt->cuda_stream = nullptr;
}

size_t tslb_workspace_bytes(const tslb_grid* grid, const tslb_options* opt) {
    return tslb_batch_workspace_bytes(1, grid, opt);
}

size_t tslb_batch_workspace_bytes(int32_t count, const tslb_grid* grids, const tslb_options* opt) {
    if (count < 1 || !grids) return 0;
    tslb_options o;
    tslb_default_options(&o);
    if (opt) o = *opt;
    tslb_boundary b;
    std::memset(&b, 0, sizeof(b));
    std::vector<StepParams> ps(count);
    for (int i = 0; i < count; ++i) {
        std::string why;
        // The face rules affect the size only through halo z faces (four ghost
        // planes per field): a single grid is sized for them (where its z axis
        // allows them), a batch, which has none, with periodic faces.
        tslb_boundary bi = b;
        if (count == 1 && grids[i].nz >= 2) bi.face[4] = bi.face[5] = TSLB_BC_HALO;
        if (!make_params(&grids[i], 1.0, 0.0, &bi, &o, ps[i], why)) return 0;
    }
    return layout_for(ps, elem_size(o.storage), o.storage, count > 1, o.average != 0, o.scheme).total;
}

tslb_status tslb_init(tslb_ctx** out, const tslb_grid* grid, tslb_lattice lattice, double omega, double sigma,
                      const tslb_boundary* bc, const tslb_options* opt, void* workspace, size_t workspace_bytes) {
    const NvtxRange r("tslb_init");
    return create(out, 1, grid, lattice, &omega, &sigma, bc, opt, workspace, workspace_bytes, false);
}

tslb_status tslb_init_batch(tslb_ctx** out, int32_t count, const tslb_grid* grids, tslb_lattice lattice,
                            const double* omega, const double* sigma, const tslb_boundary* bcs,
                            const tslb_options* opt, void* workspace, size_t workspace_bytes) {
    const NvtxRange r("tslb_init_batch");
    return create(out, count, grids, lattice, omega, sigma, bcs, opt, workspace, workspace_bytes, count > 1);
}

tslb_status tslb_set_state(tslb_ctx* c, const float* rho, const float* u, const float* pi, const float* phi,
                           int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    c->cur = 0;
    return set_state_of(c, 0, rho, u, pi, phi, on_device);
}

tslb_status tslb_batch_set_state(tslb_ctx* c, int32_t instance, const float* rho, const float* u, const float* pi,
                                 const float* phi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    tslb_status s = check_instance(c, instance);
    if (s != TSLB_OK) return s;
    return set_state_of(c, instance, rho, u, pi, phi, on_device);
}

tslb_status tslb_step(tslb_ctx* c, int64_t n) {
    const NvtxRange r("tslb_step");
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (n < 0) return bad(c, "n must be >= 0");
    if (!all_set(c)) return bad(c, "tslb_step before the state of every grid is set", TSLB_ERR_STATE);
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
            CK(launch_one(c, c->cur), "step launch");
            c->cur ^= 1;
            c->launches += 1;
        }
        // graphs hold an even number of steps, so only plain launches flip cur
        c->t += chunk;
        if (c->average) c->avg_steps += chunk;
        n -= chunk;
        c->parts_valid = true;
        if (c->check_every > 0) {
            c->since_check += chunk;
            if (c->since_check >= c->check_every) {
                c->since_check = 0;
                for (int i = 0; i < (int)c->inst.size(); ++i) {
                    double m, ph;
                    tslb_status s = finish_sums(c, i, &m, &ph);
                    if (s != TSLB_OK) return s;
                }
            }
        }
    }
    return TSLB_OK;
}

tslb_status tslb_get_moments(tslb_ctx* c, float* rho, float* u, float* pi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    return get_moments_of(c, 0, rho, u, pi, on_device);
}

tslb_status tslb_batch_get_moments(tslb_ctx* c, int32_t instance, float* rho, float* u, float* pi,
                                   int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    tslb_status s = check_instance(c, instance);
    if (s != TSLB_OK) return s;
    return get_moments_of(c, instance, rho, u, pi, on_device);
}

tslb_status tslb_get_phi(tslb_ctx* c, float* phi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    return get_phi_of(c, 0, phi, on_device);
}

tslb_status tslb_batch_get_phi(tslb_ctx* c, int32_t instance, float* phi, int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    tslb_status s = check_instance(c, instance);
    if (s != TSLB_OK) return s;
    return get_phi_of(c, instance, phi, on_device);
}

tslb_status tslb_sums(tslb_ctx* c, double* mass, double* phi_total) {
    return tslb_batch_sums(c, 0, mass, phi_total);
}

tslb_status tslb_batch_sums(tslb_ctx* c, int32_t instance, double* mass, double* phi_total) {
    const NvtxRange r("tslb_sums");
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!mass || !phi_total) return bad(c, "mass and phi_total are required");
    tslb_status s = check_instance(c, instance);
    if (s != TSLB_OK) return s;
    if (!c->inst[instance].set) return bad(c, "no state", TSLB_ERR_STATE);
    CK(cudaSetDevice(c->device), "set device");
    return finish_sums(c, instance, mass, phi_total);
}

tslb_status tslb_get_time(const tslb_ctx* c, int64_t* t) {
    if (!c || !t) return TSLB_ERR_INVALID_ARG;
    *t = c->t;
    return TSLB_OK;
}

// Slab depths tried for blocks of nw warps: the fixed list, plus (one grid)
// the depths that fill k = 2 .. 8 waves of one block per SM to at least 90 %
// (a last, partly empty wave costs as much as a full one).
std::vector<int> slab_candidates(const tslb_ctx* c, int nw) {
    std::vector<int> tz(std::begin(kAutotuneTileZ), std::end(kAutotuneTileZ));
    if (c->batch) tz.push_back(128);  // fewer re-staged planes; a batch's grids still give many tiles
    if (!c->batch) {
        const StepParams& p = c->inst[0].p;
        const long long txy = tiles_of(p, c->storage, nw, p.nz);  // tiles of one full-depth slab
        for (int k = 2; k <= 8; ++k) {
            const long long slabs = (long long)k * c->sms / txy;
            if (slabs < 1) continue;
            const int d = (int)((p.nz + slabs - 1) / slabs);
            const long long blocks = txy * ((p.nz + d - 1) / d);
            if (d >= 8 && d <= p.nz && blocks * 10 >= (long long)k * c->sms * 9 && blocks <= (long long)k * c->sms)
                tz.push_back(d);
        }
    }
    std::sort(tz.begin(), tz.end());
    tz.erase(std::unique(tz.begin(), tz.end()), tz.end());
    return tz;
}

tslb_status tslb_autotune(tslb_ctx* c, int32_t steps_per_trial, int32_t* block_warps, int32_t* tile_z,
                          int32_t* plain_stores) {
    const NvtxRange r("tslb_autotune");
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (steps_per_trial < 1) return bad(c, "steps_per_trial must be >= 1");
    if (!all_set(c)) return bad(c, "tslb_autotune before the state of every grid is set", TSLB_ERR_STATE);
    if (c->scheme == 1) return bad(c, "the two-sweep scheme has no tile shape to tune");
    CK(cudaSetDevice(c->device), "set device");
    const int q = c->cur;
    // kernel forms tried: blocks of 8 and 12 warps (14 and 16 for one grid
    // under the projection closure), and for FP32 storage the 8-, 12- (and for
    // one grid under the projection closure 16-) warp forms with plain stores
    const bool ce = !c->batch && c->inst[0].p.closure == tslb::CL_CHAPMAN_ENSKOG;
    struct Form {
        int nw;
        bool plain;
    };
    std::vector<Form> forms = {{8, false}, {12, false}};
    if (!ce && !c->batch) {
        forms.push_back({14, false});
        forms.push_back({16, false});
    }
    if (c->storage == TSLB_FP32) {
        forms.push_back({8, true});
        forms.push_back({12, true});
        if (!ce && !c->batch) forms.push_back({16, true});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event create");
    CK(cudaEventCreate(&e1), "event create");
    std::vector<int> keep_tz(c->inst.size());
    for (size_t i = 0; i < c->inst.size(); ++i) keep_tz[i] = c->inst[i].p.tile_z;
    // the trial steps must not add to the time sums
    for (Instance& I : c->inst) I.p.avg = nullptr;
    float best = 1e30f;
    int best_nw = c->batch ? c->batch_nw : c->inst[0].p.block_warps;
    bool best_plain = c->batch ? c->batch_plain : c->inst[0].p.plain_stores != 0;
    int best_tz = keep_tz[0];
    tslb_status st = TSLB_OK;
    for (size_t si = 0; si < forms.size() && st == TSLB_OK; ++si)
        for (int tz : slab_candidates(c, forms[si].nw)) {
            // each trial re-runs the step from the current state into the other
            // buffer, so the state itself does not advance
            for (Instance& I : c->inst) {
                I.p.block_warps = forms[si].nw;
                I.p.plain_stores = forms[si].plain ? 1 : 0;
                I.p.tile_z = std::min(tz, I.p.nz);
            }
            if (c->batch) {
                c->batch_nw = forms[si].nw;
                c->batch_plain = forms[si].plain;
                if ((st = upload_batch(c)) != TSLB_OK) break;
            }
            cudaError_t e = trial_launch(c, q);
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int k = 0; k < steps_per_trial && e == cudaSuccess; ++k) e = trial_launch(c, q);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = cuda_fail(c, e, "autotune trial");
                break;
            }
            if (ms < best) {
                best = ms;
                best_nw = forms[si].nw;
                best_plain = forms[si].plain;
                best_tz = tz;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // apply the winner (or restore on failure)
    for (size_t i = 0; i < c->inst.size(); ++i) {
        Instance& I = c->inst[i];
        I.p.avg = I.avg;
        I.p.block_warps = best_nw;
        I.p.plain_stores = best_plain ? 1 : 0;
        I.p.tile_z = st == TSLB_OK ? std::min(best_tz, I.p.nz) : keep_tz[i];
    }
    if (c->batch) {
        c->batch_nw = best_nw;
        c->batch_plain = best_plain;
        tslb_status s2 = upload_batch(c);
        if (st == TSLB_OK) st = s2;
    }
    // the trials wrote the other buffer and the other step-counter slot: restore it
    // (and rearm the tile counter of the next batch step)
    long long tt = (long long)c->t;
    CK(cudaMemcpyAsync(c->tdev + (q ^ 1), &tt, sizeof(tt), cudaMemcpyHostToDevice, c->stream), "step counter");
    if (c->batch) CK(cudaMemsetAsync(c->counters + q, 0, sizeof(int), c->stream), "tile counter");
    CK(cudaStreamSynchronize(c->stream), "autotune synchronise");
    drop_graphs(c);
    c->parts_valid = false;
    if (block_warps) *block_warps = best_nw;
    if (tile_z) *tile_z = best_tz;
    if (plain_stores) *plain_stores = best_plain ? 1 : 0;
    return st;
}

tslb_status tslb_step_form(tslb_ctx* c, int32_t* block_warps, int32_t* tile_z, int32_t* plain_stores,
                           int32_t* tma_only) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    const Instance& I = c->inst[0];
    if (c->batch) {
        if (block_warps) *block_warps = c->batch_nw;
        if (tile_z) *tile_z = I.p.tile_z;
        if (plain_stores) *plain_stores = c->batch_plain ? 1 : 0;
        if (tma_only) *tma_only = batch_tma_only(c) ? 1 : 0;
        return TSLB_OK;
    }
    bool to = false;
    if (c->scheme == 0 && I.p.closure == tslb::CL_PROJECTION) {
        CK(cudaSetDevice(c->device), "set device");
        tslb::TileMaps* m = nullptr;
        CK(single_maps(c, c->cur, &m), "tensor maps");
        to = m->all_tma && I.p.plain_stores == 0;
    }
    if (block_warps) *block_warps = I.p.block_warps;
    if (tile_z) *tile_z = I.p.tile_z;
    if (plain_stores) *plain_stores = I.p.plain_stores;
    if (tma_only) *tma_only = to ? 1 : 0;
    return TSLB_OK;
}

size_t tslb_state_bytes(const tslb_ctx* c) {
    if (!c) return 0;
    return (size_t)tslb::stored_fields(c->inst[0].p.closure) * (size_t)c->inst[0].N * c->elem + sizeof(int64_t);
}

tslb_status tslb_get_state(tslb_ctx* c, void* dst, int on_device) {
    if (!c || !dst) return TSLB_ERR_INVALID_ARG;
    if (c->batch) return bad(c, "checkpoints are per single-grid context");
    Instance& I = c->inst[0];
    if (!I.set) return bad(c, "no state", TSLB_ERR_STATE);
    if (on_device && !is_device_ptr(dst)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const size_t fb = (size_t)I.N * c->elem;
    const int nf = tslb::stored_fields(I.p.closure);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int f = 0; f < nf; ++f)
        CK(cudaMemcpyAsync(static_cast<char*>(dst) + f * fb,
                           static_cast<const char*>(I.buf[c->cur]) + (size_t)f * I.p.fstride * c->elem, fb, kind,
                           c->stream),
           "state copy");
    int64_t t = c->t;
    if (on_device)
        CK(cudaMemcpyAsync(static_cast<char*>(dst) + nf * fb, &t, sizeof(t), cudaMemcpyHostToDevice,
                           c->stream),
           "step copy");
    CK(cudaStreamSynchronize(c->stream), "get_state synchronise");
    if (!on_device) std::memcpy(static_cast<char*>(dst) + nf * fb, &t, sizeof(t));
    return TSLB_OK;
}

tslb_status tslb_put_state(tslb_ctx* c, const void* src, int on_device) {
    if (!c || !src) return TSLB_ERR_INVALID_ARG;
    if (c->batch) return bad(c, "checkpoints are per single-grid context");
    if (on_device && !is_device_ptr(src)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    Instance& I = c->inst[0];
    const size_t fb = (size_t)I.N * c->elem;
    const int nf = tslb::stored_fields(I.p.closure);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->cur = 0;
    for (int f = 0; f < nf; ++f)
        CK(cudaMemcpyAsync(static_cast<char*>(I.buf[0]) + (size_t)f * I.p.fstride * c->elem,
                           static_cast<const char*>(src) + f * fb, fb, kind, c->stream),
           "state copy");
    int64_t t = 0;
    if (on_device)
        CK(cudaMemcpyAsync(&t, static_cast<const char*>(src) + nf * fb, sizeof(t), cudaMemcpyDeviceToHost,
                           c->stream),
           "step copy");
    else
        std::memcpy(&t, static_cast<const char*>(src) + nf * fb, sizeof(t));
    CK(cudaStreamSynchronize(c->stream), "put_state synchronise");
    if (t < 0) return bad(c, "negative step index in checkpoint");
    long long tt[2] = {(long long)t, (long long)t};
    CK(cudaMemcpyAsync(c->tdev, tt, sizeof(tt), cudaMemcpyHostToDevice, c->stream), "step counter");
    CK(cudaStreamSynchronize(c->stream), "put_state synchronise");
    c->t = t;
    I.set = true;
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
    drop_graphs(c);
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

int32_t tslb_batch_count(const tslb_ctx* c) { return c ? (int32_t)c->inst.size() : 0; }

tslb_status tslb_get_averages(tslb_ctx* c, int32_t instance, double* phi_sum, double* uz_sum, int64_t* steps,
                              int on_device) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    tslb_status s = check_instance(c, instance);
    if (s != TSLB_OK) return s;
    if (!c->average) return bad(c, "the context was created without the average option", TSLB_ERR_STATE);
    if (on_device && ((phi_sum && !is_device_ptr(phi_sum)) || (uz_sum && !is_device_ptr(uz_sum))))
        return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    Instance& I = c->inst[instance];
    const size_t bytes = (size_t)I.N * sizeof(double);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (phi_sum) CK(cudaMemcpyAsync(phi_sum, I.avg, bytes, kind, c->stream), "averages copy");
    if (uz_sum) CK(cudaMemcpyAsync(uz_sum, I.avg + I.p.fstride, bytes, kind, c->stream), "averages copy");
    CK(cudaStreamSynchronize(c->stream), "averages synchronise");
    if (steps) *steps = c->avg_steps;
    return TSLB_OK;
}

tslb_status tslb_reset_averages(tslb_ctx* c) {
    if (!c) return TSLB_ERR_INVALID_ARG;
    if (!c->average) return bad(c, "the context was created without the average option", TSLB_ERR_STATE);
    CK(cudaSetDevice(c->device), "set device");
    for (Instance& I : c->inst)
        CK(cudaMemsetAsync(I.avg, 0, 2 * (size_t)I.p.fstride * sizeof(double), c->stream), "clear averages");
    CK(cudaStreamSynchronize(c->stream), "averages synchronise");
    c->avg_steps = 0;
    return TSLB_OK;
}

size_t tslb_halo_values(const tslb_ctx* c) {
    if (!c || c->batch) return 0;
    return (size_t)(tslb::F_PHI + 2) * c->inst[0].p.nx * c->inst[0].p.ny;
}

tslb_status tslb_halo_pack(tslb_ctx* c, int32_t side, void* dst, int on_device) {
    if (!c || !dst || (side != 0 && side != 1)) return TSLB_ERR_INVALID_ARG;
    if (c->batch) return bad(c, "halo messages are per single-grid context");
    Instance& I = c->inst[0];
    if (!I.set) return bad(c, "no state", TSLB_ERR_STATE);
    if (on_device && !is_device_ptr(dst)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const size_t nxy = (size_t)I.p.nx * I.p.ny, e = c->elem;
    // side 0: what the neighbour below needs (moments of plane 0, phi of planes 0, 1);
    // side 1: what the neighbour above needs (plane nz - 1; planes nz - 2, nz - 1)
    const size_t zm = side == 0 ? 0 : (size_t)I.p.nz - 1, zp = side == 0 ? 0 : (size_t)I.p.nz - 2;
    const char* b = static_cast<const char*>(I.buf[c->cur]);
    char* d = static_cast<char*>(dst);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpy2DAsync(d, nxy * e, b + zm * nxy * e, (size_t)I.p.fstride * e, nxy * e, tslb::F_PHI, kind,
                         c->stream),
       "halo pack (moments)");
    CK(cudaMemcpyAsync(d + (size_t)tslb::F_PHI * nxy * e, b + ((size_t)tslb::F_PHI * I.p.fstride + zp * nxy) * e,
                       2 * nxy * e, kind, c->stream),
       "halo pack (phase field)");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "halo pack synchronise");
    return TSLB_OK;
}

tslb_status tslb_halo_unpack(tslb_ctx* c, int32_t side, const void* src, int on_device) {
    if (!c || !src || (side != 0 && side != 1)) return TSLB_ERR_INVALID_ARG;
    if (c->batch) return bad(c, "halo messages are per single-grid context");
    Instance& I = c->inst[0];
    if (!I.set) return bad(c, "no state", TSLB_ERR_STATE);
    if (I.p.face[4 + side] != tslb::BC_HALO) return bad(c, "that z face does not have the halo rule");
    if (on_device && !is_device_ptr(src)) return bad(c, "on_device pointers must be device memory");
    CK(cudaSetDevice(c->device), "set device");
    const size_t nxy = (size_t)I.p.nx * I.p.ny, e = c->elem, nz = (size_t)I.p.nz;
    // side 0 (from the neighbour below): moments -> plane -1 (stored as nz + 3),
    // phi -> planes -2, -1 (nz + 2, nz + 3); side 1 (from above): moments ->
    // plane nz, phi -> planes nz, nz + 1
    const size_t zm = side == 0 ? nz + 3 : nz, zp = side == 0 ? nz + 2 : nz;
    char* b = static_cast<char*>(I.buf[c->cur]);
    const char* sp = static_cast<const char*>(src);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpy2DAsync(b + zm * nxy * e, (size_t)I.p.fstride * e, sp, nxy * e, nxy * e, tslb::F_PHI, kind,
                         c->stream),
       "halo unpack (moments)");
    CK(cudaMemcpyAsync(b + ((size_t)tslb::F_PHI * I.p.fstride + zp * nxy) * e, sp + (size_t)tslb::F_PHI * nxy * e,
                       2 * nxy * e, kind, c->stream),
       "halo unpack (phase field)");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "halo unpack synchronise");
    return TSLB_OK;
}

}  // extern "C"
