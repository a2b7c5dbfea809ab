// Internal interface between the C-ABI host code (tslb_api.cu) and the CUDA
// kernels (tslb_step.cu) of the TSLB library.  Not installed, not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tslb {

enum { BC_PERIODIC = 0, BC_INLET = 1, BC_OUTFLOW = 2, BC_FREE_SLIP = 3, BC_HALO = 4 };
// A z face with the HALO rule borders a neighbouring slab of a domain split
// along z: the ghost planes beyond it hold the neighbour's stored fields,
// written by the caller before each step.  A grid with a HALO face stores
// four ghost planes after the interior of every field: planes nz, nz + 1
// (above) and, at plane indices nz + 2, nz + 3, the planes -2, -1 (below).
constexpr int kHaloPlanes = 4;
inline __host__ __device__ bool has_halo(const int face[6]) { return face[4] == BC_HALO || face[5] == BC_HALO; }
enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2 };

// Stored fields of one state buffer, each a block of `fstride` elements:
// rho - 1, u (3), P (xx, yy, zz, xy, xz, yz), phi.
enum {
    F_DRHO = 0, F_UX, F_UY, F_UZ, F_PXX, F_PYY, F_PZZ, F_PXY, F_PXZ, F_PYZ, F_PHI, NFIELDS
};

// Closure of the non-equilibrium second moment: the projection Pi - Pi^eq of
// the stored P (all 11 fields stored), or the Chapman-Enskog estimate from the
// strain rate of the momentum field (P not stored: rho - 1, u, phi in slots
// 0..4).
enum { CL_PROJECTION = 0, CL_CHAPMAN_ENSKOG = 1 };
inline __host__ __device__ int stored_fields(int closure) { return closure == CL_CHAPMAN_ENSKOG ? 5 : NFIELDS; }
// Buffer slot of field f (f must be stored under the closure).
inline __host__ __device__ int field_slot(int closure, int f) {
    return closure == CL_CHAPMAN_ENSKOG && f == F_PHI ? 4 : f;
}

// Everything the step kernel needs, passed by value (__grid_constant__).
struct StepParams {
    int nx, ny, nz;
    int face[6];
    int tile_z;
    int block_warps;         // warps per block of the step kernel (8, 12 or 16)
    int closure;             // CL_PROJECTION or CL_CHAPMAN_ENSKOG
    long long fstride;       // elements between consecutive fields of a buffer
    float omega, sigma, gamma, normal_eps2;
    float inlet_u[3], inlet_umag, inlet_half_d, inlet_cx, inlet_cy, inlet_two_over_w, noise_amp;
    unsigned seed_lo, seed_hi;
    float scale[NFIELDS];    // 16-bit storage: stored = scale * value
    float inv_scale[NFIELDS];
    double* avg;             // time sums of phi and u_z (2 blocks of fstride doubles) or null
    int* err;                // set to 1 by a kernel whose bounded wait for its tile data gave up
    int test_stall;          // testing: TMA tiles expect bytes no copy delivers, in their first
                             // loads (1) or in the first loads of the march (2): the wait expires
    int plain_stores;        // FP32, 8, 12 or 16 warps: plain stores instead of the staging box + TMA store
};

// Tensor maps of one step for the TMA tile copies of the step kernel: the 10
// moment fields of the input buffer as a 4D tensor {nx, ny, nz, field}, its
// phase field as a 3D tensor {nx, ny, nz}, and (FP32) the 11 fields of the
// output buffer, with the box shapes of the block size they were made for.
// valid = 0: every tile loads element by element; store = 0: plain stores.
// FP32 grids with periodic x or y faces also get the side boxes that bring a
// tile the sources of its ghosts across those faces (wrap = 1): a 4-column
// strip of the moments (x wrap), one moment row (y wrap) and their 4-column
// corner, and the phase-field equivalents (two rows).
struct TileMaps {
    CUtensorMap mom;
    CUtensorMap phi;
    CUtensorMap out;
    CUtensorMap momx, momy, momc;
    CUtensorMap phix, phiy, phic;
    int valid;
    int store;
    int wrap;
    int block_warps;
    int all_tma;  // every tile of the grid loads by TMA (tiles_all_tma) and no time sums are
                  // kept: 12-warp blocks with staged stores run the step kernel compiled for
                  // that load path alone
};



// One grid of a batch: its parameters, its two state buffers and the tensor
// maps of the steps from buf[q] to buf[q ^ 1] (device memory, 64-byte aligned).
struct BatchInstance {
    StepParams p;
    const void* buf[2];
    TileMaps maps[2];
};

struct LaunchShape {
    dim3 grid, block;
    size_t smem;
    int nw;                  // warps per block (rows of a tile incl. 2 halo rows)
};

// Geometry of the step kernel launch for this grid (tile_z = z slab per block).
LaunchShape step_shape(const StepParams& p, int storage);

// One time step: state `in` (step index *t_in) -> state `out` (*t_out = *t_in + 1),
// per-block FP64 partial sums (sum rho, sum phi) into partials[2 * block].
// maps: tensor maps of `in` (TMA tile loads when maps->valid and made for
// p.block_warps), or null.
cudaError_t launch_step(const StepParams& p, int storage, const void* in, void* out,
                        const long long* t_in, long long* t_out, double* partials,
                        cudaStream_t s, const TileMaps* maps = nullptr);

// Encodes the tensor maps of a step from state buffer `in` to `out` for
// blocks of p.block_warps warps (maps->valid = 0 where TMA cannot address the
// layout: rows not a multiple of 16 bytes).  Host only; needs no device work.
cudaError_t make_tile_maps(const StepParams& p, int storage, const void* in, const void* out, TileMaps* maps);

// Whether every tile of grid p loads by TMA in the 12-warp staged-store form
// of the step kernel (with the periodic-face side boxes if wrap; FP32 only):
// the kernel's own tile set-up, run once per x-y tile, ORs a refusal into
// *flag (one device int, scratch).  Synchronises stream s; not for use while
// it is being captured.  *all = false for other closures.
cudaError_t tiles_all_tma(const StepParams& p, int storage, bool wrap, int* flag, cudaStream_t s, bool* all);

// Kernel attributes (dynamic shared memory) of the step kernel; once per device.
cudaError_t prepare_kernels(int storage);

// Step kernel of the Chapman-Enskog closure (tslb_step_ce.cu; FP32 or 16-bit
// storage, blocks of 8 or 12 warps), same contract as launch_step.
// maps: the output map of the 5 stored fields (staged TMA stores, FP32) or null.
cudaError_t launch_step_ce(const StepParams& p, int storage, const void* in, void* out,
                           const long long* t_in, long long* t_out, double* partials, cudaStream_t s,
                           const TileMaps* maps = nullptr);
cudaError_t prepare_kernels_ce(int storage);

// One caller field (float, device) -> one stored field (rho - 1 for F_DRHO).
cudaError_t launch_put_field(const StepParams& p, int storage, const float* src, int field,
                             void* state, cudaStream_t s);

// One stored field -> float moment (rho for F_DRHO, the value itself otherwise).
cudaError_t launch_get_field(const StepParams& p, int storage, const void* state, int field,
                             float* dst, cudaStream_t s);

// Partial sums of a stored state (used when no step has produced them).
cudaError_t launch_state_sums(const StepParams& p, int storage, const void* state,
                              double* partials, int* nparts, cudaStream_t s);

// Fixed-order FP64 reduction of n partial pairs into result[0..1].
cudaError_t launch_finish_sums(const double* partials, int n, double* result, cudaStream_t s);

// Largest number of partial pairs any launch above writes for this grid.
int max_partials(const StepParams& p, int storage);

// Batched FP32 step: tiles[k] = (instance, bx, by, bz) over all instances,
// taken from counters[parity] by one persistent block per SM on `sms` SMs,
// blocks of `nw` warps (8 or 12), with plain stores if `plain`, in the form
// for periodic faces if `wrap` (some instance has side-box maps), compiled
// for TMA tile loads alone if `tma_only` (12 warps, staged stores: every tile
// of every instance loads by TMA, tiles_all_tma); tile k writes
// partials[2k..2k+1].
cudaError_t prepare_batch_kernels();
cudaError_t launch_batch_step(int nw, bool plain, bool wrap, bool tma_only, const BatchInstance* insts,
                              const int4* tiles, int ntiles, int parity, const long long* t_in, long long* t_out,
                              int* counters, double* partials, int sms, cudaStream_t s);

// The paper's two-sweep design (ablation): collide+push of the moments M into
// 34 population arrays `pops` (27 f_i - w_i, then 7 g_k), then the moments of
// the populations back into M (in place) with block partial sums.
int twosweep_partials(const StepParams& p);
cudaError_t launch_twosweep_step(const StepParams& p, float* M, float* pops, const long long* t_in,
                                 long long* t_out, double* partials, cudaStream_t s);

// Message returned by tslb_last_error(NULL) (calls that have no context).
void set_global_error(const char* msg);

}  // namespace tslb
