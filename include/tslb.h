/*
 * tslb.h - C ABI of the GB300 (sm_103a) multicomponent thread-safe lattice
 * Boltzmann library (arXiv 2403.15773, Montessori, Hegele, Lauricella).
 *
 * The library advances the fused per-time-step update of the paper: a D3Q27
 * flow solver with third-order Hermite equilibria and recursive third-order
 * regularisation (Sec. 2, Eq. fullstrcoll, eqts, noneqts), coupled to a D3Q7
 * conservative phase-field solver with anti-diffusion and continuum-surface
 * surface tension (Sec. 2.2, Eq. intcapturing, antidiff).  As in the paper,
 * the state is stored as moments only (Sec. 2: rho, rho u and the six
 * components of Pi^neq per node, plus the phase field phi), and each step
 * rebuilds every node's post-streamed populations from its neighbours'
 * moments (Sec. 2, Fig. 1).  One CUDA kernel launch performs one time step.
 *
 * Conventions used by every entry point:
 *   - Grid arrays are structure-of-arrays, x fastest: node n = x + nx*(y + ny*z),
 *     N = nx*ny*nz.  Vectors are 3 blocks of N (x, y, z); the second-order
 *     tensor P is 6 blocks of N in the order xx, yy, zz, xy, xz, yz.
 *   - Moments exchanged with the caller: rho; u = j / rho (the velocity of the
 *     stored momentum, before the half-force shift of the forcing scheme);
 *     P = Pi - rho cs2 I - rho u u (the non-equilibrium momentum flux of
 *     Sec. 2 relative to u); phi in [-1, 1], +1 = component A.
 *   - on_device != 0: the pointer is CUDA device memory of the context's
 *     device; 0: host memory (pageable or pinned).  The moment and phi calls
 *     (set_state, get_moments, get_phi and their batch forms) read and write
 *     page-locked host memory directly from their conversion kernels, over
 *     the host link; pageable host memory goes through a staging copy.
 *   - All work is issued on the context's stream; calls that return data to
 *     the host synchronise that stream.  A context must not be used from two
 *     host threads at once.
 *   - Errors are returned as tslb_status; no call aborts or throws.
 *     tslb_last_error() gives a message for the last failing call.
 */
#ifndef TSLB_H
#define TSLB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSLB_API __attribute__((visibility("default")))
#else
#define TSLB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tslb_ctx tslb_ctx;

typedef enum {
    TSLB_OK = 0,
    TSLB_ERR_INVALID_ARG = 1, /* bad size, pointer, parameter or boundary spec */
    TSLB_ERR_OOM = 2,         /* device or host allocation failed / workspace too small */
    TSLB_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    TSLB_ERR_UNSTABLE = 4,    /* the total mass or phase field became non-finite */
    TSLB_ERR_TIMEOUT = 5,     /* a step kernel's bounded wait for its tile data gave up (reported by
                                 tslb_sums and the check_every checks) */
    TSLB_ERR_STATE = 6        /* call out of order (e.g. tslb_step before tslb_set_state) */
} tslb_status;

typedef enum { TSLB_LATTICE_D3Q27_D3Q7 = 0 } tslb_lattice;

/* Storage of the per-node fields in HBM (11, or 5 under the Chapman-Enskog
 * closure).  All arithmetic is FP32. */
typedef enum { TSLB_FP32 = 0, TSLB_FP16 = 1, TSLB_BF16 = 2 } tslb_storage;

/* Face rules.  INLET is allowed on the -z face only. */
typedef enum {
    TSLB_BC_PERIODIC = 0,  /* wrap; both faces of an axis must be periodic */
    TSLB_BC_INLET = 1,     /* jet inlet: ghost with rho and P of the adjacent fluid node and
                              imposed u, phi (non-equilibrium extrapolation, Eq. original_neq) */
    TSLB_BC_OUTFLOW = 2,   /* zero-gradient copy of the adjacent fluid node */
    TSLB_BC_FREE_SLIP = 3, /* specular mirror about the half-way plane */
    TSLB_BC_HALO = 4       /* z faces only: the face borders a neighbouring slab of a domain split
                              along z; the ghost planes beyond it (moments of one plane, phi of
                              two) are written by tslb_halo_unpack before each step */
} tslb_bc;

typedef struct {
    int32_t nx, ny, nz; /* nodes per axis; >= 1 on periodic axes, >= 2 otherwise */
} tslb_grid;

/* Closure of the non-equilibrium second moment a2_neq of the collision
 * (Sec. 2.1).
 * PROJECTION: a2_neq = Pi - Pi^eq of the stored moments; the state holds
 *   rho - 1, u, P, phi (11 fields).
 * CHAPMAN_ENSKOG: a2_neq = -(cs2/omega)(d_a j_b + d_b j_a), the strain rate of
 *   j = rho u by the isotropic D3Q27 gradient stencil, evaluated at every node
 *   and ghost over the ghost-resolved momentum field; the state holds rho - 1,
 *   u, phi (5 fields) and P does not exist (tslb_get_moments refuses pi,
 *   tslb_set_state ignores it).  Single grids, scheme 0, block_warps 8 or 12. */
typedef enum { TSLB_CLOSURE_PROJECTION = 0, TSLB_CLOSURE_CHAPMAN_ENSKOG = 1 } tslb_closure;

/* Boundary specification.  The inlet imposes on the -z face a smoothed top
 * hat of diameter inlet_diameter centred at (inlet_cx, inlet_cy):
 *   phi_B = -tanh(2 (r - D/2) / W), u_B = s (inlet_u + xi), s = (1 + phi_B)/2,
 *   xi_c = noise_amp |inlet_u| (2 r_c - 1), r_c = (philox4x32_10_c >> 8) 2^-24,
 * with Philox4x32-10 (Salmon et al., SC'11) on counter (x + nx y, t_lo, t_hi, 0)
 * and key (seed_lo, seed_hi), t the step index. */
typedef struct {
    int32_t face[6]; /* tslb_bc for -x, +x, -y, +y, -z, +z */
    float inlet_u[3];
    float inlet_diameter;
    float inlet_cx, inlet_cy;
    float noise_amp;
    uint64_t seed;
} tslb_boundary;

typedef struct {
    int32_t storage;        /* tslb_storage; default TSLB_FP32 */
    float interface_width;  /* W: anti-diffusion Gamma = 1/W gives a tanh(2x/W) interface; default 3 */
    float normal_eps;       /* the interface normal is grad phi / sqrt(|grad phi|^2 + eps^2); default 1e-2 */
    float field_scale[4];   /* 16-bit storage: stored value = scale * (rho - 1), scale * u,
                               scale * P, scale * d with d = phi -+ (1 + 1/16) the deviation of
                               phi from the nearer of +-(1 + 1/16) (its sign tells which; |phi|
                               saturates at 1 + 1/16); 0 = default (1/(3 U^2), 1/(2 U), 1e3, 1) */
    int32_t check_every;    /* tslb_step checks the FP64 sums for non-finite values every this
                               many steps (synchronises); 0 = never (default) */
    int32_t tile_z;         /* z extent of one thread block's slab; 0 = automatic (single grids: the
                               depth in 8..128 minimising waves of one block per SM times the planes
                               a block marches; batches: 64) */
    int32_t graph_steps;    /* steps per captured CUDA graph replayed by tslb_step; 0 = automatic,
                               1 = plain launches */
    int32_t block_warps;    /* warps per block of the step kernel: 8, 12, 14 or 16 (tiles of 14,
                               22, 26 or 30 interior rows; 28 interior columns; 14 and 16 keep
                               part of each thread's state in tensor memory); 0 = 12 for a
                               single grid, 8 for a batch.  14 and 16: single grids under the
                               projection closure */
    int32_t scheme;         /* 0: the fused moment-only step (default, 88 B per update in FP32);
                               1: the paper's two-sweep design kept as an ablation: collide+push
                               into 34 population arrays in HBM, then their moments (360 B per
                               update; single grid, FP32, no averages, no autotune) */
    int32_t average;        /* 1: every step also adds the new phi and u_z of each node to FP64
                               time sums (the time-averaged fields of Sec. 3: centre-line and
                               radial profiles of <phi> and <u_z>); 0 = off (default) */
    int32_t closure;        /* tslb_closure of the non-equilibrium second moment; default
                               TSLB_CLOSURE_PROJECTION */
    int32_t test_tma_stall; /* testing only: 1 makes the step kernel's TMA tiles wait for bytes no copy
                               delivers in their first loads, so the bounded wait expires (about
                               1 s per block) and tslb_sums returns TSLB_ERR_TIMEOUT; 2 does the
                               same to the first loads of the plane march, so the tile gives up
                               with later loads still in flight (it lets them land before it
                               releases its barriers); 0 = off (default) */
    int32_t plain_stores;   /* FP32 storage, blocks of 8, 12 or 16 warps (8 or 12 under the
                               Chapman-Enskog closure): 1 = the step kernel writes each
                               finished plane with plain stores instead of staging it in shared
                               memory for one TMA store; the smaller shared-memory footprint leaves
                               the L1 cache more room for tiles that load element by element
                               (rows not a multiple of 16 bytes, grids narrower than a tile with
                               periodic x or y faces); 0 = staged TMA stores (default).  Results
                               are the same either way; tslb_autotune tries both. */
    int32_t per_tile_loads; /* 1 = the step kernel chooses its load path tile by tile (TMA box
                               copies, or element-wise loads where a tile's ghost sources lie
                               outside its boxes) in every block size; 0 = automatic (default):
                               the library runs the 12-warp kernel's own tile set-up once per tile
                               (single grids at tslb_init, batches when they first take 12-warp
                               blocks), and where every tile (of every grid) loads by TMA and the
                               option average is off, blocks of 12 warps with staged stores run a
                               kernel compiled for that load path alone (fewer registers and
                               instructions in the plane march).
                               Results are the same either way (for comparison and testing). */
    void* cuda_stream;      /* cudaStream_t to issue work on; NULL = a stream the library creates
                               (blocking, so ordered with the legacy default stream) */
} tslb_options;

/* Fills *opt with the defaults above. */
TSLB_API void tslb_default_options(tslb_options* opt);

/* Bytes of device workspace tslb_init needs for this grid and options (the two
 * state buffers, the per-block FP64 partial sums and a few counters), or 0 if
 * the arguments are invalid.  The size holds the ghost planes of halo z faces,
 * so it serves every boundary specification. */
TSLB_API size_t tslb_workspace_bytes(const tslb_grid* grid, const tslb_options* opt);

/* Creates a context on the current CUDA device.
 *   omega: BGK relaxation frequency in (0, 2); nu = (1/3)(1/omega - 1/2) (Sec. 2).
 *   sigma: surface tension >= 0 (Sec. 2.2: F = -(sigma/2) kappa grad phi for phi in [-1, 1]).
 *   bc:    face rules and inlet; NULL = fully periodic.
 *   opt:   NULL = defaults.
 *   workspace: device memory of at least tslb_workspace_bytes() bytes, 256-byte
 *          aligned, owned by the caller and kept alive until tslb_destroy; NULL =
 *          the library allocates (cudaMalloc) and frees it.
 * The state is undefined until tslb_set_state. */
TSLB_API tslb_status tslb_init(tslb_ctx** out, const tslb_grid* grid, tslb_lattice lattice, double omega,
                      double sigma, const tslb_boundary* bc, const tslb_options* opt,
                      void* workspace, size_t workspace_bytes);

/* Sets the state from rho[N], u[3N] and phi[N]; pi[6N] sets P (NULL = 0, i.e.
 * the populations start at the third-order equilibrium; ignored under the
 * Chapman-Enskog closure).  Step index := 0. */
TSLB_API tslb_status tslb_set_state(tslb_ctx* ctx, const float* rho, const float* u, const float* pi,
                           const float* phi, int on_device);

/* Advances n >= 0 time steps (asynchronous on the context stream unless
 * check_every > 0).  Each step: one fused kernel (Sec. 2, Eq. fullstrcoll with
 * the third-order terms of Eq. eqts/noneqts, and the D3Q7 update of Eq.
 * intcapturing/antidiff) plus, inside it, the FP64 per-block partial sums of
 * rho and phi of the new state. */
TSLB_API tslb_status tslb_step(tslb_ctx* ctx, int64_t n);

/* Copies the current moments out (rho[N], u[3N], pi[6N]; any may be NULL;
 * pi must be NULL under the Chapman-Enskog closure, else TSLB_ERR_INVALID_ARG). */
TSLB_API tslb_status tslb_get_moments(tslb_ctx* ctx, float* rho, float* u, float* pi, int on_device);

/* Copies the current phase field out (phi[N]). */
TSLB_API tslb_status tslb_get_phi(tslb_ctx* ctx, float* phi, int on_device);

/* Total mass sum(rho) and total phase field sum(phi) of the current state in
 * FP64, reduced in a fixed order (bitwise reproducible).  Returns
 * TSLB_ERR_UNSTABLE (and still the values) if either is not finite. */
TSLB_API tslb_status tslb_sums(tslb_ctx* ctx, double* mass, double* phi_total);

/* Number of steps taken since tslb_set_state / tslb_put_state. */
TSLB_API tslb_status tslb_get_time(const tslb_ctx* ctx, int64_t* t);

/* Checkpoint: the raw stored fields (11 N values of the storage type, 5 N
 * under the Chapman-Enskog closure) plus the step index, tslb_state_bytes()
 * bytes in total.  put_state restores a buffer written by get_state of a
 * context with the same grid, storage and closure. */
TSLB_API size_t tslb_state_bytes(const tslb_ctx* ctx);
TSLB_API tslb_status tslb_get_state(tslb_ctx* ctx, void* dst, int on_device);
TSLB_API tslb_status tslb_put_state(tslb_ctx* ctx, const void* src, int on_device);

/* Blocks until all work of the context has finished. */
TSLB_API tslb_status tslb_synchronize(tslb_ctx* ctx);

/* Frees the context (and the workspace if the library allocated it). */
TSLB_API tslb_status tslb_destroy(tslb_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing tslb_init
 * when ctx is NULL).  Never NULL. */
TSLB_API const char* tslb_last_error(const tslb_ctx* ctx);
TSLB_API const char* tslb_status_string(tslb_status s);

/* Number of step-kernel launches issued by this context so far (each launch
 * is one time step over the whole grid). */
TSLB_API int64_t tslb_kernel_launches(const tslb_ctx* ctx);

/* ---- Batches of independent grids (one launch per time step for all). ----
 *
 * A batch context advances `count` independent grids (each with its own size,
 * omega, sigma and faces; same options, FP32 storage) together: each time
 * step is one persistent kernel launch whose blocks take the tiles of all
 * grids from a device work counter, and tslb_step replays those launches
 * from a captured CUDA graph.  tslb_step, tslb_get_time, tslb_autotune,
 * tslb_synchronize and tslb_destroy take batch contexts; the single-grid
 * tslb_set_state / tslb_get_moments / tslb_get_phi / tslb_sums act on grid 0.
 * Setting any grid's state restarts the step index of the batch at 0.
 * Checkpoints (tslb_get_state / tslb_put_state) are single-grid only. */
TSLB_API size_t tslb_batch_workspace_bytes(int32_t count, const tslb_grid* grids, const tslb_options* opt);
TSLB_API tslb_status tslb_init_batch(tslb_ctx** out, int32_t count, const tslb_grid* grids,
                                     tslb_lattice lattice, const double* omega, const double* sigma,
                                     const tslb_boundary* bcs /* count entries, NULL = all periodic */,
                                     const tslb_options* opt, void* workspace, size_t workspace_bytes);
TSLB_API tslb_status tslb_batch_set_state(tslb_ctx* ctx, int32_t instance, const float* rho, const float* u,
                                          const float* pi, const float* phi, int on_device);
TSLB_API tslb_status tslb_batch_get_moments(tslb_ctx* ctx, int32_t instance, float* rho, float* u, float* pi,
                                            int on_device);
TSLB_API tslb_status tslb_batch_get_phi(tslb_ctx* ctx, int32_t instance, float* phi, int on_device);
TSLB_API tslb_status tslb_batch_sums(tslb_ctx* ctx, int32_t instance, double* mass, double* phi_total);
TSLB_API int32_t tslb_batch_count(const tslb_ctx* ctx);

/* Time sums of phi and u_z (option `average`), N doubles each (either may be
 * NULL), accumulated over the *steps steps taken since the state was set or
 * the sums were reset; the time averages are sum / steps.  Autotuner trials
 * are not counted. */
TSLB_API tslb_status tslb_get_averages(tslb_ctx* ctx, int32_t instance, double* phi_sum, double* uz_sum,
                                       int64_t* steps, int on_device);
TSLB_API tslb_status tslb_reset_averages(tslb_ctx* ctx);

/* Tile-shape autotuner: times the step kernel for blocks of 8 and 12 warps
 * (and 14 and 16 for one grid under the projection closure; with FP32 storage under
 * the projection closure also the 8-, 12- and 16-warp forms with plain_stores) and
 * z slabs of 16, 24, 32, 48 and 64 planes (a batch also 128), plus, for one grid, the slab
 * depths whose block count fills 2 to 8 waves of one block per SM to at least
 * 90 % (steps_per_trial launches each, CUDA events on the context stream), and
 * keeps the fastest for all later steps.  Every trial recomputes the step from
 * the current state into the spare buffer, so the state and the step index do
 * not change.  Drops captured graphs; synchronises.  Reports the choice in
 * *block_warps, *tile_z and *plain_stores (any may be NULL). */
TSLB_API tslb_status tslb_autotune(tslb_ctx* ctx, int32_t steps_per_trial, int32_t* block_warps, int32_t* tile_z,
                                   int32_t* plain_stores);

/* The step kernel form the next tslb_step launches: *block_warps,
 * *tile_z (a batch: its first grid's), *plain_stores, and *tma_only = 1 if
 * it is the kernel compiled for TMA tile loads alone (option per_tile_loads),
 * 0 otherwise (any pointer may be NULL).  A single grid's tensor maps of the
 * current block size are encoded here if no step has yet. */
TSLB_API tslb_status tslb_step_form(tslb_ctx* ctx, int32_t* block_warps, int32_t* tile_z, int32_t* plain_stores,
                                    int32_t* tma_only);

/* The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory when they ask for the totals.  cudaMalloc
 * and cudaFree synchronise the whole device, which an asynchronous pipeline
 * cannot afford, and a process whose device memory is held by another
 * allocator's pool may have none left to allocate; tslb_sums needs a context
 * whose workspace had to be allocated first.
 *
 * Writes out[0] = sum(rho) and out[1] = sum(phi) in FP64 for the caller's FP32
 * device arrays rho[n] and phi[n] (out: 2 doubles of device memory), reduced in
 * a fixed order, asynchronously on cuda_stream (NULL = legacy default stream).
 * Allocates nothing: its scratch is a fixed array of 16384 FP64 partial pairs
 * (256 KiB) in the library's own device memory, held by every GPU that loads
 * the library until the process exits.  n must lie in [1, 268435456] (16384
 * partials of 16384 values; 512 x 512 x 1024 nodes); larger n returns
 * TSLB_ERR_INVALID_ARG without launching anything.  The first call on a device
 * is its set-up: it looks up the scratch's device address, which the library
 * keeps until the process exits, and with CUDA's lazy module loading it is
 * also the call that loads the library's kernels onto the device (which may
 * allocate and synchronise once).  So make a first call on each device before
 * any stream capture and before any section that must not allocate, and do not
 * reset the device (cudaDeviceReset) while the process still uses this entry
 * point.  All calls share the scratch: calls whose work overlaps on the GPU
 * race on it and must be ordered by the caller (same stream, or events).
 * Returns TSLB_ERR_CUDA if a launch fails; messages via tslb_last_error(NULL). */
TSLB_API tslb_status tslb_field_sums_noalloc(const float* rho, const float* phi, int64_t n,
                                             double* out, void* cuda_stream);

/* ---- Slabs of a domain split along z (multi-GPU decomposition). ----
 *
 * The paper runs one GPU and names multi-GPU runs as future work (Sec. 4
 * and 5); the update reaches one node (moments) and two nodes (phi, for its
 * stencils) beyond a plane, so a domain split into z slabs needs, before
 * every step, one plane of the ten moment fields and two planes of phi from
 * each neighbouring slab.  A slab is a single-grid context (projection
 * closure, fused scheme) whose z faces toward its neighbours have the
 * TSLB_BC_HALO rule; its other faces keep the global rules (the inlet on the
 * first slab, the outflow on the last).  Per step: tslb_halo_pack on each
 * slab, exchange the messages, tslb_halo_unpack, tslb_step(ctx, 1).
 *
 * A message is tslb_halo_values() values of the storage type: the ten
 * moment fields (rho - 1, u, P, in the stored form) of one plane, nx*ny each,
 * then phi of two planes in increasing z.  Side 0 is the -z side, 1 the +z
 * side.  tslb_halo_pack(side) writes what the neighbour on that side needs
 * (side 0: moments of plane 0, phi of planes 0, 1; side 1: plane nz - 1,
 * planes nz - 2, nz - 1); tslb_halo_unpack(side) stores a message from the
 * neighbour on that side into the ghost planes (the face must have the halo
 * rule).  Both are asynchronous on the context stream for device buffers and
 * synchronise for host buffers; the ghost planes are zero after
 * tslb_set_state.  0 for a batch context. */
TSLB_API size_t tslb_halo_values(const tslb_ctx* ctx);
TSLB_API tslb_status tslb_halo_pack(tslb_ctx* ctx, int32_t side, void* dst, int on_device);
TSLB_API tslb_status tslb_halo_unpack(tslb_ctx* ctx, int32_t side, const void* src, int on_device);

/* Measurement helper (the paper has no counterpart): the FP32 fused
 * multiply-add rate of the current device, the arithmetic roofline of the
 * step kernel (whose collision and streaming sweeps are FP32 work).  Runs a
 * kernel of independent FMA chains in registers on 4 blocks of 512 threads
 * per SM, scalar FFMA (packed = 0) or packed fma.rn.f32x2 (packed = 1), on
 * cuda_stream (NULL = legacy default stream), times its second launch with
 * CUDA events and synchronises.  *lane_ops_per_s = fused multiply-adds per
 * second summed over all lanes (a packed instruction counts two).  Returns
 * TSLB_ERR_INVALID_ARG for packed outside {0, 1} or a NULL result pointer,
 * TSLB_ERR_CUDA if a CUDA call fails; messages via tslb_last_error(NULL). */
TSLB_API tslb_status tslb_fp32_lane_rate(int32_t packed, void* cuda_stream, double* lane_ops_per_s);

#ifdef __cplusplus
}
#endif
#endif
