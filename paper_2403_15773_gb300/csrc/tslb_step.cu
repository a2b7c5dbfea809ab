// Fused time step of the multicomponent thread-safe lattice Boltzmann method
// (arXiv 2403.15773) for sm_103a, and the small kernels around it.
//
// One launch = one time step over the whole grid.  Each thread block owns a
// slab of 28 x TY interior columns and marches through its z range plane by
// plane.  A warp holds two rows of 32 staged columns (interior, one halo
// column each side, two spare lanes); the block holds TY interior rows plus
// one halo row above and below.
//
// Per staged node and plane the kernel
//   1. reads the moments (rho - 1, u, P) and the phase field of the node and of
//      its ghost images: one thread loads each plane's boxes with TMA
//      (cp.async.bulk.tensor, mbarrier completion) one or two planes ahead,
//      and ghosts of mirror / copy faces read their source inside the box;
//      ghosts across periodic faces read theirs from small side boxes loaded
//      with the plane (FP32 kernels of 8 and 12 warps); the remaining tiles
//      whose ghost sources leave the box load element by element (cp.async,
//      or 16-bit loads through registers);
//   2. evaluates grad phi and its Hessian with the isotropic D3Q27 stencils
//      (the phase field of three planes read straight from the ring of
//      loaded planes), the normal n, the curvature kappa = div n and the
//      surface-tension force F = -(sigma/2) kappa grad phi (Sec. 2.2);
//   3. forms the post-collision populations of the node in Hermite form,
//        f_i^post = w_i [A0 + c.A1/cs2 + H2:A2/(2 cs^4) + H3:A3/(6 cs^6)],
//      with A1 = j + F, A2 = rho u u + (1-omega) Pi^neq + (1-omega/2)(uF + Fu),
//      A3 = rho u u u + (1-omega)(u Pi^neq + ...)  (Eq. fullstrcoll, eqts,
//      noneqts; Guo forcing), and the D3Q7 post-collision set
//        g_i^post = w_i [phi + c_i.(phi u / cs7^2 + Gamma (1 - phi^2) n)]
//      (Eq. intcapturing, antidiff);
//   4. streams and takes moments.  Instead of 27 explicit populations per node
//      the rebuild-and-gather of Sec. 2 (Fig. 1) is done axis by axis: D3Q27 is
//      the tensor product of three D1Q3 lattices, so the Hermite coefficients
//      of one axis are turned into the three 1D populations of that axis,
//      shifted by +-1 node (warp shuffles along x, shared memory along y,
//      registers of the z march along z), and turned into raw moments of that
//      axis before the next axis is processed.  The result is exactly
//      rho' = sum_i f_i(x - c_i), j' = sum_i c_i f_i(x - c_i),
//      Pi' = sum_i c_i c_i f_i(x - c_i) up to FP32 rounding;
//   5. stores rho' - 1, u' = j'/rho', P' = Pi' - rho' cs2 I - rho' u' u' and
//      phi' (FP32: into a staging box that leaves by one TMA store per plane,
//      or with plain stores in the kernel form without the box; 16-bit: plain
//      stores), and accumulates the FP64 block partials of sum(rho - 1),
//      sum(phi).
// Steps 1-3 and the x and y populations of a plane (phase (d)) and the y and
// z shifts and the output of the plane before it (phase (e)) run in one
// stretch of code per plane with one block barrier: a software pipeline whose
// y exchange is double-buffered by plane parity.
//
// All arithmetic is FP32 and works with deviations from the rest state
// (rho - 1, Pi - cs2 I) so that no O(1) terms cancel.
#include <cstring>

#include "tslb_device.cuh"

namespace tslb {
namespace {

// ----------------------------------------------------- step kernel (pairs)

// Shared memory of a block of NW warps with storage type S; ST: the staging
// box of finished planes (FP32 blocks of up to 12 warps; without it, plain
// stores and a smaller footprint, which leaves the L1 cache more of the
// storage it shares with shared memory); WR: each slot also holds the side
// boxes of ghosts across periodic faces.  The moment and
// phase-field planes of a tile are held as the boxes a TMA copy writes: a
// moment box is [10 fields][NR rows][MW columns], a phase-field box
// [NR + 2 rows][PW columns], each starting at the staged tile's first column
// rounded down to 16 bytes (offsets offm / offp inside the box).
template <int NW, typename S, bool ST = true, bool WR = false>
struct Step2Smem {
    static constexpr int NT = 32 * NW;                       // threads
    static constexpr int NR = 2 * NW;                        // staged rows (two per warp)
    static constexpr int TY = NR - 2;                        // interior rows
    static constexpr int NPH = PHX * (NR + 2);               // phase-field elements (halo 2)
    static constexpr int AL = 16 / (int)sizeof(S);           // elements per 16 bytes
    // interior columns of a tile: 28, so that the staged columns (interior and
    // one halo column each side) leave lanes 30 and 31 spare for the interface
    // stencil's neighbour columns, and FP32 tiles start on 16-byte boundaries
    // (finished planes leave by TMA store; 16-bit storage uses plain stores)
    static constexpr bool kFp32 = sizeof(S) == 4;
    static constexpr int TXS = TX;
    // blocks of more than 12 warps keep the carries of the z march in tensor
    // memory between planes (registers: 65536 / threads); 12-warp blocks keep
    // them in registers (the 16-bit form spills a little, and is still faster
    // than with the round trips through tensor memory)
    static constexpr bool TC = NW > 12;
    // box columns: staged columns x0-1 .. x0+30 (moments) and x0-2 .. x0+31
    // (phase field) from the 16-byte boundary below them
    static constexpr int MW = kFp32 ? 36 : 40;
    static constexpr int PW = kFp32 ? 36 : 40;
    static constexpr int MAXOFFM = kFp32 ? 3 : 7, MAXOFFP = kFp32 ? 2 : 6;
    static constexpr int FS = NR * MW;                       // elements between fields of a moment box
    static constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t MOM_BOX = sizeof(S) * 10 * FS;           // bytes of one moment box
    static constexpr size_t PHI_BOX = sizeof(S) * (NR + 2) * PW;     // bytes of one phase-field box
    // WR: each slot also holds the side boxes of ghosts across periodic faces,
    // after its box: moments X [10][NR][4], Y [10][MW], C [10][4]; phase field
    // X [NR + 2][4], Y [2][PW], C [2][4] (byte offsets within the slot)
    static constexpr size_t MX_BYTES = sizeof(S) * 10 * NR * 4, MY_BYTES = sizeof(S) * 10 * MW;
    static constexpr size_t MC_BYTES = sizeof(S) * 10 * 4;
    static constexpr size_t PX_BYTES = sizeof(S) * (NR + 2) * 4, PY_BYTES = sizeof(S) * 2 * PW;
    static constexpr size_t PC_BYTES = sizeof(S) * 2 * 4;
    static constexpr size_t MX = r128(MOM_BOX), MY = MX + r128(MX_BYTES), MC = MY + r128(MY_BYTES);
    static constexpr size_t PX = r128(PHI_BOX), PY = PX + r128(PX_BYTES), PC = PY + r128(PY_BYTES);
    static constexpr size_t MOM_SLOT = WR ? MC + r128(MC_BYTES) : r128(MOM_BOX);
    static constexpr size_t PHI_SLOT = WR ? PC + r128(PC_BYTES) : r128(PHI_BOX);
    // planes between the load of a plane's moments and their use (the phase
    // field is loaded one plane further ahead)
    static constexpr int PF = NW <= 8 ? 2 : 1;
    static constexpr int MS = PF + 1, PS = PF + 3, NB = PF + 2;      // moment slots, phase slots, mbarriers
    static constexpr size_t MOM = 0;                                 // [MS] moment boxes
    static constexpr size_t RING = MOM + MS * MOM_SLOT;              // [PS] phase-field boxes
    static constexpr int EPT = (NPH + NT - 1) / NT;                  // phase-field elements per thread
    static constexpr size_t YX_BUF = sizeof(float) * 20 * (size_t)NT;  // one y exchange [20][NT]
    static constexpr size_t YX = RING + PS * PHI_SLOT;               // [2][20][NT] y exchange (plane parity)
    static constexpr size_t OUT_BOX = sizeof(float) * NFIELDS * TY * TXS;  // [11][TY][TXS]
    static constexpr size_t OUT_SLOT = r128(OUT_BOX);
    static constexpr size_t OUT = r128(YX + 2 * YX_BUF);             // [2] output staging boxes
    static constexpr size_t TAIL = NB * sizeof(uint64_t) + 16 + 128;  // mbarriers, TMEM address, base slack
    static constexpr size_t kMax = 227 * 1024;
    // Finished planes leave through two staging boxes by TMA store (one plane's
    // store overlaps the next plane) where shared memory has room for them
    // (FP32, up to 12 warps); otherwise by plain stores.
    static constexpr bool kTmaStore = kFp32 && ST && OUT + 2 * OUT_SLOT + TAIL <= kMax;
    static constexpr int OUTN = kTmaStore ? 2 : 0;
    static constexpr size_t BAR = OUT + OUTN * OUT_SLOT;              // NB mbarriers
    static constexpr size_t TMA_ADDR = BAR + NB * sizeof(uint64_t);   // TMEM column address (TC)
    static constexpr size_t BYTES = TMA_ADDR + 16 + 128;              // + alignment slack of the base
    // TMEM: 128 columns per warp (four warps per lane quarter): the 40 carries
    // of the z march at columns 0 .. 39, the 48 values (d) hands to (e) at 64 .. 111
    static constexpr uint32_t TM_COLS = 512;
    static_assert(MAXOFFM + 32 <= MW && MAXOFFP + PHX <= PW, "box too narrow for the aligned tile");
    static_assert(!kTmaStore || (TXS * sizeof(S)) % 16 == 0, "store box rows must be 16-byte multiples");
    static_assert(BYTES <= kMax, "more shared memory than a block can have");
    static_assert(!TC || NW <= 16, "TMEM: at most four warps share a lane quarter");
};

// The dynamic shared memory base rounded up to 128 bytes (TMA boxes).  The
// offset is added to the shared array itself so that the compiler keeps
// addressing it as shared memory (a round trip through an integer address
// would turn every access into a generic load or store).
__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
    return p + ((0u - smem_u32(p)) & 127u);
}

// One tile of one time step: the 28 x (2 NW - 2) interior columns at tile
// (bx, by), planes [bz * tile_z, (bz + 1) * tile_z), from state `in` (step t)
// to state `out`; writes the tile's FP64 partial sums to part[0..1].  Returns
// false (in every thread) if tile loads were still in flight when the block
// gave up on them: its mbarriers and shared memory must then not be reused.
// maps: tensor maps of `in` for TMA loads, or null (element-wise loads).
// ST: staged TMA stores (FP32); WR: side boxes for ghosts across periodic
// faces (FP32, maps with the side-box tensor maps).  TS: this tile's finished
// planes do leave through the staging boxes (a kernel form with them, and
// maps with the output map: staged_stores()); a compile-time flag, so that
// the march has no branch on it.
// MODE: TILE_ANY chooses the load path per tile at run time; TILE_TMA is
// compiled for TMA loads alone (no element-wise path in the march: fewer
// registers and instructions) and without the time sums of phi and u_z, for
// launches whose tiles all load by TMA and that keep no time sums;
// TILE_CLASSIFY stops after the set-up and returns whether this tile can load
// by TMA (tile_class_kernel).  The last two exist for blocks of at most 12
// warps (no tensor-memory carries).  UR: copies of the march body the plane
// loop is unrolled into (4 for the single-grid kernel compiled for TMA
// loads alone; 2 elsewhere: 4 measured slower with the batch kernel's
// 64-plane slabs).
constexpr int TILE_ANY = 0, TILE_TMA = 1, TILE_CLASSIFY = 2;

template <int NW, typename S, bool ST, bool WR, bool TS, int MODE = TILE_ANY, int UR = 2>
__device__ __forceinline__ bool step_tile(const StepParams& P, const TileMaps* maps, const S* __restrict__ in,
                                          S* __restrict__ out, const long long t, const int bx, const int by,
                                          const int bz, double* __restrict__ part) {
    using L = Step2Smem<NW, S, ST, WR>;
    constexpr int NT = L::NT, NR = L::NR, NPH = L::NPH, MW = L::MW, PW = L::PW, FS = L::FS, AL = L::AL;
    constexpr int TY = L::TY;
    constexpr int OSL = (int)(L::OUT_SLOT / sizeof(float));
    constexpr int EPT = L::EPT;
    constexpr int MSL = (int)(L::MOM_SLOT / sizeof(S)), PSL = (int)(L::PHI_SLOT / sizeof(S));
    constexpr int PF = L::PF, MS = L::MS, PS = L::PS, NB = L::NB;
    // slots of plane q (q >= z0 - 2) and the mbarrier of the loads issued at
    // iteration i (>= z0 - 1), counted from the tile's first plane so that the
    // two copies of the unrolled march see fixed parities
    auto mslot = [z0 = bz * P.tile_z](int q) { return (q - z0 + 12) % MS; };
    auto pslot = [z0 = bz * P.tile_z](int q) { return (q - z0 + 20) % PS; };
    auto bslot = [z0 = bz * P.tile_z](int i) { return (i - z0 + 12) % (PF + 1); };
    // output staging box and y-exchange buffer of plane q (parity from z0)
    auto obuf = [z0 = bz * P.tile_z](int q) { return (q - z0 + 8) & 1; };
    constexpr int BPRO = PF + 1;  // mbarrier of the prologue loads
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* const sm = align128(smem_raw);
    S* const momb = reinterpret_cast<S*>(sm + L::MOM);
    S* const ring = reinterpret_cast<S*>(sm + L::RING);
    float* const yx = reinterpret_cast<float*>(sm + L::YX);
    float* const outb = reinterpret_cast<float*>(sm + L::OUT);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(sm + L::BAR);

    const int lane = threadIdx.x, w = threadIdx.y, tid = lane + 32 * w;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const long long fs = P.fstride;
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * P.tile_z;
    const int z1 = min(z0 + P.tile_z, nz);
    const bool use_maps = maps != nullptr && maps->valid && maps->block_warps == NW;
    // finished planes leave through the staging box by TMA store (FP32)
    static_assert(!TS || L::kTmaStore, "staged stores need the staging boxes");
    static_assert(MODE == TILE_ANY || !L::TC, "TMA-only and classification forms: blocks of at most 12 warps");
    constexpr bool tst = TS;
    if (MODE != TILE_CLASSIFY && use_maps && tid == 0) {
        for (int k = 0; k < NB; ++k) mbar_init(bar + k, 1);
        fence_mbar_init();
    }

    // box origins (x aligned down to 16 bytes; floor for negative x)
    const int xm = (x0 - 1) & ~(AL - 1), xp = (x0 - 2) & ~(AL - 1);
    const int ym = y0 - 1, yp = y0 - 2;
    const int offm = x0 - 1 - xm, offp = x0 - 2 - xp;

    // the two staged nodes of this thread (constant along the march)
    int unused = 0;
    float sgx, sgyA, sgyB;
    const int gx = x0 - 1 + lane, gyA = y0 - 1 + 2 * w, gyB = gyA + 1;
    const int sx = resolve_axis(gx, nx, P.face[0], P.face[1], sgx, unused);
    const int syA = resolve_axis(gyA, ny, P.face[2], P.face[3], sgyA, unused);
    const int syB = resolve_axis(gyB, ny, P.face[2], P.face[3], sgyB, unused);
    const int sxyA = sx + nx * syA, sxyB = sx + nx * syB;  // < 2^31: the plane size is checked on the host
    const bool col_ok = lane >= 1 && lane <= TX && gx < nx;
    const bool storeA = col_ok && w >= 1 && gyA < ny;       // staged row 2w is interior for w >= 1
    const bool storeB = col_ok && w <= NW - 2 && gyB < ny;  // staged row 2w+1 for w <= NW-2

    // Where each staged value is read in shared memory: at its own box position
    // (element-wise loads fetch the ghost-resolved source into it), or, for TMA
    // tiles, at the box position of its resolved source (ghost images of
    // mirror and copy faces lie inside the box; a tile whose sources do not,
    // e.g. across a periodic wrap, loads element-wise).
    // Staged values beyond the ghost layers a stencil reaches (ragged tiles)
    // feed no stored node: they keep their own position.
    int mrdA = (2 * w) * MW + lane + offm, mrdB = mrdA + MW;
    const bool usex = gx >= -1 && gx <= nx, useA = usex && gyA >= -1 && gyA <= ny, useB = usex && gyB >= -1 && gyB <= ny;
    const int resA = useA ? (syA - ym) * MW + (sx - xm) : mrdA, resB = useB ? (syB - ym) * MW + (sx - xm) : mrdB;
    bool inbox = (!useA || (sx >= xm && sx - xm < MW && syA >= ym && syA - ym < NR)) &&
                 (!useB || (sx >= xm && sx - xm < MW && syB >= ym && syB - ym < NR));
    // WR kernels (FP32 grids with periodic x or y faces): a ghost across such a
    // face reads its source from the side boxes loaded with the plane (a
    // 4-column strip at x = nx - 4 or 0, one moment row / two phase-field rows
    // at y = ny - 1 (ny - 2) or 0, their corner), at its own field stride.  A
    // tile needs at most one x strip and one y strip (else it loads element
    // by element).
    int fsA = FS, fsB = FS;
    bool wrx = false, wry = false;
    int xs0 = 0, ysm = 0, ysp = 0;
    [[maybe_unused]] const bool perx = P.face[0] == BC_PERIODIC, pery = P.face[2] == BC_PERIODIC;
    if constexpr (WR) {
        const bool xl = perx && x0 == 0, xr = perx && x0 + 31 >= nx;
        const bool yt = pery && y0 == 0, yb = pery && y0 + NR - 1 >= ny;
        wrx = xl || xr;
        wry = yt || yb;
        xs0 = xl ? nx - 4 : 0;
        ysm = yt ? ny - 1 : 0;
        ysp = yt ? ny - 2 : 0;
        bool ok = !(xl && xr) && !(yt && yb);
        auto side = [&](bool use, int gy, int sy, int& rd, int& fsd, int res) {
            if (!use) return;
            const bool wx = perx && (gx < 0 || gx >= nx), wy = pery && (gy < 0 || gy >= ny);
            if (!wx && !wy) {
                rd = res;
                ok = ok && sx >= xm && sx - xm < MW && sy >= ym && sy - ym < NR;
            } else if (!wy) {
                rd = (int)(L::MX / sizeof(S)) + (sy - ym) * 4 + (sx - xs0);
                fsd = NR * 4;
                ok = ok && sy >= ym && sy - ym < NR && sx >= xs0 && sx - xs0 < 4;
            } else if (!wx) {
                rd = (int)(L::MY / sizeof(S)) + (sx - xm);
                fsd = MW;
                ok = ok && sx >= xm && sx - xm < MW && sy == ysm;
            } else {
                rd = (int)(L::MC / sizeof(S)) + (sx - xs0);
                fsd = 4;
                ok = ok && sx >= xs0 && sx - xs0 < 4 && sy == ysm;
            }
        };
        int rA = mrdA, rB = mrdB;
        side(useA, gyA, syA, rA, fsA, resA);
        side(useB, gyB, syB, rB, fsB, resB);
        inbox = ok;
        mrdA = rA;
        mrdB = rB;
    }
    // Where the phase field of footprint node (row r, column c) is read in a
    // ring slot: its own box position (element-wise loads fetch the
    // ghost-resolved source into it) or, for TMA tiles, the box position of
    // its resolved source (WR: the side boxes); nodes beyond the ghost layers
    // the stencils reach keep their own position.  ok: the source lies in the
    // boxes a TMA tile loads.
    const bool inlet_face = P.face[4] == BC_INLET;
    const bool inlet_planes = inlet_face && z0 < 2;
    auto phi_source = [&](int r, int c, int& own, int& res, int& src_xy, float& phib_v, bool& ok) {
        float sg;
        const int psx = resolve_axis(x0 - 2 + c, nx, P.face[0], P.face[1], sg, unused);
        const int psy = resolve_axis(y0 - 2 + r, ny, P.face[2], P.face[3], sg, unused);
        const int gxe = x0 - 2 + c, gye = y0 - 2 + r;
        const bool used = gxe >= -2 && gxe <= nx + 1 && gye >= -2 && gye <= ny + 1;
        src_xy = psx + nx * psy;
        own = r * PW + c + offp;
        res = used ? (psy - yp) * PW + (psx - xp) : own;
        const bool wxe = WR && perx && (gxe < 0 || gxe >= nx), wye = WR && pery && (gye < 0 || gye >= ny);
        if (used && (wxe || wye)) {  // WR: phase-field side boxes
            const int px0 = (int)(L::PX / sizeof(S)), py0 = (int)(L::PY / sizeof(S)), pc0 = (int)(L::PC / sizeof(S));
            if (!wye) {
                res = px0 + (psy - yp) * 4 + (psx - xs0);
                ok = ok && psy >= yp && psy - yp < NR + 2 && psx >= xs0 && psx - xs0 < 4;
            } else if (!wxe) {
                res = py0 + (psy - ysp) * PW + (psx - xp);
                ok = ok && psy >= ysp && psy - ysp < 2 && psx >= xp && psx - xp < PW;
            } else {
                res = pc0 + (psy - ysp) * 4 + (psx - xs0);
                ok = ok && psy >= ysp && psy - ysp < 2 && psx >= xs0 && psx - xs0 < 4;
            }
        } else {
            ok = ok && (!used || (psx >= xp && psx - xp < PW && psy >= yp && psy - yp < NR + 2));
        }
        phib_v = inlet_planes ? inlet_phi(P, psx, psy) : 0.f;
    };
    // the footprint nodes this thread loads element by element (idx = tid + e NT)
    int pxy[EPT], prd[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int idx = tid + e * NT;
        pxy[e] = 0;
        prd[e] = 0;
        if (idx < NPH) {
            int res;
            float pb;
            phi_source(idx / PHX, idx % PHX, prd[e], res, pxy[e], pb, inbox);
        }
    }
    // the footprint nodes the interface stencil of this thread's row pair
    // reads: rows 2w .. 2w + 3 of its own column (lane 31: column 0)
    int rd4[4], res4[4];
    float phib4[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int sxy;
        phi_source(2 * w + r, own_column(lane), rd4[r], res4[r], sxy, phib4[r], inbox);
    }
    // TMEM for the z-march carries and the handoffs (blocks of more than 12
    // warps): warp 0 allocates the block's columns; each warp uses 128 columns
    // of its lane quarter
    [[maybe_unused]] uint32_t tm_base = 0, tm_addr = 0;
    [[maybe_unused]] uint32_t* const tm_slot = reinterpret_cast<uint32_t*>(sm + L::TMA_ADDR);
    if constexpr (L::TC) {
        if (w == 0) tmem_alloc(tm_slot, L::TM_COLS);
        tmem_fence_before();
    }
    const bool tma_ok = __syncthreads_and(use_maps && inbox && (!WR || !(wrx || wry) || maps->wrap)) != 0;
    if constexpr (MODE == TILE_CLASSIFY) return tma_ok;
    // TILE_TMA: the host launches this form only where every tile loads by
    // TMA.  A tile that cannot (not met) still loads its boxes, reads at its
    // own box positions (all inside shared memory), and reports error 2.
    if (MODE == TILE_TMA && !tma_ok && tid == 0 && P.err) *P.err = 2;
    const bool tma = MODE == TILE_TMA || tma_ok;  // a constant in the TILE_TMA form
    if constexpr (L::TC) {
        tmem_fence_after();
        tm_base = *tm_slot;
        tm_addr = tm_base + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(w >> 2) * 128u;
    }
    if (tma && tma_ok) {
        if constexpr (!WR) {  // (WR: mrdA / mrdB set above)
            mrdA = resA;
            mrdB = resB;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) rd4[r] = res4[r];
    } else if constexpr (WR) {  // element-wise after all (or TILE_TMA, not met): own positions, box stride
        mrdA = (2 * w) * MW + lane + offm;
        mrdB = mrdA + MW;
        fsA = fsB = FS;
    }

    // Loads of the phase field at plane qp (if do_p) and the moments at plane
    // qm (if do_m) into their ring / moment slots.  TMA: one thread posts the
    // byte count on mbarrier kb and issues the box copies.  Element-wise: FP32
    // cp.async straight into shared memory; 16-bit values wait in registers
    // until commit().  Inlet planes of the phase field are never loaded (the
    // imposed values are used directly).  Returns whether bar[kb] got copies.
    // (16-bit element-wise loads: the raw values wait in registers, the two
    // rows of a moment field packed into one 32-bit register)
    unsigned short rphi[EPT];
    unsigned rmom[10];
    // bytes a plane's phase-field / moment copies deliver (WR: with the side boxes)
    const unsigned pbytes = (unsigned)L::PHI_BOX + (WR ? (wrx ? (unsigned)L::PX_BYTES : 0u) +
                                                             (wry ? (unsigned)L::PY_BYTES : 0u) +
                                                             (wrx && wry ? (unsigned)L::PC_BYTES : 0u)
                                                       : 0u);
    const unsigned mbytes = (unsigned)L::MOM_BOX + (WR ? (wrx ? (unsigned)L::MX_BYTES : 0u) +
                                                             (wry ? (unsigned)L::MY_BYTES : 0u) +
                                                             (wrx && wry ? (unsigned)L::MC_BYTES : 0u)
                                                       : 0u);
    // WR: the side boxes of plane z (resolved) into the slots at dp / dm
    auto side_phi = [&](S* dp, int z, uint64_t* b) {
        if constexpr (WR) {
            if (wrx) tma_load_3d(dp + L::PX / sizeof(S), &maps->phix, xs0, yp, z, b);
            if (wry) tma_load_3d(dp + L::PY / sizeof(S), &maps->phiy, xp, ysp, z, b);
            if (wrx && wry) tma_load_3d(dp + L::PC / sizeof(S), &maps->phic, xs0, ysp, z, b);
        }
    };
    auto side_mom = [&](S* dm, int z, uint64_t* b) {
        if constexpr (WR) {
            if (wrx) tma_load_4d(dm + L::MX / sizeof(S), &maps->momx, xs0, ym, z, 0, b);
            if (wry) tma_load_4d(dm + L::MY / sizeof(S), &maps->momy, xm, ysm, z, 0, b);
            if (wrx && wry) tma_load_4d(dm + L::MC / sizeof(S), &maps->momc, xs0, ysm, z, 0, b);
        }
    };
    auto issue = [&](bool do_p, int qp, bool do_m, int qm, int kb) -> bool {
        // only the inlet face is never loaded (its phase field is imposed)
        const bool lp = do_p && !(inlet_face && qp < 0);
        if (tma) {  // the issuing thread alone resolves the planes and addresses
            if (tid == 0 && (lp || do_m)) {
                float sg;
                int in2 = 0;
                fence_proxy_async();
                // (P.test_stall == 2: the first loads of the march expect 16 bytes more
                // than they deliver, so the march gives up with later loads in flight)
                mbar_expect_tx(bar + kb, (lp ? pbytes : 0u) + (do_m ? mbytes : 0u) +
                                             (P.test_stall == 2 && qm == z0 - 1 + PF ? 16u : 0u));
                if (lp) {
                    const int z = resolve_axis(qp, nz, P.face[4], P.face[5], sg, in2);
                    tma_load_3d(ring + pslot(qp) * PSL, &maps->phi, xp, yp, z, bar + kb);
                    side_phi(ring + pslot(qp) * PSL, z, bar + kb);
                }
                if (do_m) {
                    const int z = resolve_axis(qm, nz, P.face[4], P.face[5], sg, in2);
                    tma_load_4d(momb + mslot(qm) * MSL, &maps->mom, xm, ym, z, 0, bar + kb);
                    side_mom(momb + mslot(qm) * MSL, z, bar + kb);
                }
            }
            return lp || do_m;
        }
        float sg;
        int in2 = 0;
        const int szp = do_p ? resolve_axis(qp, nz, P.face[4], P.face[5], sg, in2) : 0;
        const int szm = do_m ? resolve_axis(qm, nz, P.face[4], P.face[5], sg, in2) : 0;
        S* const pdst = ring + pslot(qp) * PSL;
        S* const mdst = momb + mslot(qm) * MSL;
        if (lp) {
            const S* src = in + F_PHI * fs + nxy * szp;
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (tid + e * NT < NPH) {
                    if constexpr (Io<S>::kAsync)
                        cp_async4(reinterpret_cast<float*>(pdst + prd[e]), reinterpret_cast<const float*>(src + pxy[e]));
                    else
                        rphi[e] = __ldg(reinterpret_cast<const unsigned short*>(src + pxy[e]));
                }
        }
        if (do_m) {
            const S* srcA = in + nxy * szm + sxyA;
            const S* srcB = in + nxy * szm + sxyB;
#pragma unroll
            for (int f = 0; f < 10; ++f) {
                if constexpr (Io<S>::kAsync) {
                    cp_async4(reinterpret_cast<float*>(mdst + mrdA + f * FS), reinterpret_cast<const float*>(srcA + f * fs));
                    cp_async4(reinterpret_cast<float*>(mdst + mrdB + f * FS), reinterpret_cast<const float*>(srcB + f * fs));
                } else {
                    rmom[f] = (unsigned)__ldg(reinterpret_cast<const unsigned short*>(srcA + f * fs)) |
                              ((unsigned)__ldg(reinterpret_cast<const unsigned short*>(srcB + f * fs)) << 16);
                }
            }
        }
        return false;
    };
    // 16-bit element-wise loads: registers -> shared memory (raw values).
    auto commit = [&](bool do_p, int qp, bool do_m, int qm) {
        if constexpr (!Io<S>::kAsync) {
            if (tma) return;
            if (do_p && !(inlet_face && qp < 0)) {
                unsigned short* dst = reinterpret_cast<unsigned short*>(ring + pslot(qp) * PSL);
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (tid + e * NT < NPH) dst[prd[e]] = rphi[e];
            }
            if (do_m) {
                unsigned short* dst = reinterpret_cast<unsigned short*>(momb + mslot(qm) * MSL);
#pragma unroll
                for (int f = 0; f < 10; ++f) {
                    dst[mrdA + f * FS] = (unsigned short)(rmom[f] & 0xffffu);
                    dst[mrdB + f * FS] = (unsigned short)(rmom[f] >> 16);
                }
            }
        }
    };
    unsigned pend = 0, phase = 0;  // mbarriers with copies in flight; their phase parities
    bool dead = false;             // a bounded wait gave up: finish the tile without further waits
    auto wait_bar = [&](int kb) {
        if (!((pend >> kb) & 1u)) return;
        if (!dead && !mbar_wait(bar + kb, (phase >> kb) & 1u)) {
            dead = true;
            if (P.err) *P.err = 1;
        }
        phase ^= 1u << kb;
        pend &= ~(1u << kb);
    };
    // prologue: phase field at planes z0-2 .. z0+PF-1, moments at planes z0-1 .. z0+PF-2
    if (tma) {
        if (tid == 0) {
            float sg;
            int in2 = 0;
            unsigned bytes = PF * mbytes;
            for (int q = z0 - 2; q <= z0 + PF - 1; ++q)
                if (!(inlet_face && q < 0)) bytes += pbytes;
            fence_proxy_async();
            // (P.test_stall == 1: 16 bytes more than the copies deliver, so the wait below expires)
            mbar_expect_tx(bar + BPRO, bytes + (P.test_stall == 1 ? 16u : 0u));
            for (int q = z0 - 2; q <= z0 + PF - 1; ++q)
                if (!(inlet_face && q < 0)) {
                    const int z = resolve_axis(q, nz, P.face[4], P.face[5], sg, in2);
                    tma_load_3d(ring + pslot(q) * PSL, &maps->phi, xp, yp, z, bar + BPRO);
                    side_phi(ring + pslot(q) * PSL, z, bar + BPRO);
                }
            for (int k = 0; k < PF; ++k) {
                const int z = resolve_axis(z0 - 1 + k, nz, P.face[4], P.face[5], sg, in2);
                tma_load_4d(momb + mslot(z0 - 1 + k) * MSL, &maps->mom, xm, ym, z, 0, bar + BPRO);
                side_mom(momb + mslot(z0 - 1 + k) * MSL, z, bar + BPRO);
            }
        }
        pend |= 1u << BPRO;
    } else {
        for (int q = z0 - 2; q <= z0 + PF - 1; ++q) {
            issue(true, q, false, 0, BPRO);
            commit(true, q, false, 0);
        }
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            issue(false, 0, true, z0 - 1 + k, BPRO);
            commit(false, 0, true, z0 - 1 + k);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    wait_bar(BPRO);

    // z march carries: for the groups whose z moments 1, 2 are needed
    // (g < 3) p(i-2), z(i-1) and p(i-1); for the others (and phi) the partial
    // zeroth moment p(i-2) + z(i-1) and p(i-1)
    float2 cPP[3], cZ[3], cP[6], cA[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) cP[k] = cA[k] = bc(0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) cPP[k] = cZ[k] = bc(0.f);
    float2 cAph = bc(0.f), cVP = bc(0.f);
    float sum_rho = 0.f, sum_phi = 0.f;
    // TMEM form: the 34 carry values (40 columns) of each thread live in its
    // TMEM lane between planes; (e) loads them, advances them and stores them
    [[maybe_unused]] auto carries_pack = [&](float (&c)[40]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c[2 * k] = cPP[k].x, c[2 * k + 1] = cPP[k].y;
            c[6 + 2 * k] = cZ[k].x, c[7 + 2 * k] = cZ[k].y;
            c[24 + 2 * k] = cA[3 + k].x, c[25 + 2 * k] = cA[3 + k].y;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) c[12 + 2 * k] = cP[k].x, c[13 + 2 * k] = cP[k].y;
        c[30] = cAph.x, c[31] = cAph.y, c[32] = cVP.x, c[33] = cVP.y;
#pragma unroll
        for (int k = 34; k < 40; ++k) c[k] = 0.f;
    };
    [[maybe_unused]] auto carries_unpack = [&](const float (&c)[40]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cPP[k] = make_float2(c[2 * k], c[2 * k + 1]);
            cZ[k] = make_float2(c[6 + 2 * k], c[7 + 2 * k]);
            cA[3 + k] = make_float2(c[24 + 2 * k], c[25 + 2 * k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) cP[k] = make_float2(c[12 + 2 * k], c[13 + 2 * k]);
        cAph = make_float2(c[30], c[31]);
        cVP = make_float2(c[32], c[33]);
    };
    [[maybe_unused]] auto carries_store = [&]() {
        float c[40];
        carries_pack(c);
#pragma unroll
        for (int k = 0; k < 5; ++k) tmem_st8(tm_addr + 8u * k, c + 8 * k);
        tmem_wait_st(c);
    };
    if constexpr (L::TC) carries_store();

    const unsigned msx = sgx < 0.f ? 0x80000000u : 0u, msyA = sgyA < 0.f ? 0x80000000u : 0u,
                   msyB = sgyB < 0.f ? 0x80000000u : 0u;
    const float om1 = 1.f - P.omega, fo = 1.f - 0.5f * P.omega;
    const float sig_half = -0.5f * P.sigma;

    // Software-pipelined march, one barrier per iteration i = z0 - 1 .. z1 + 1:
    //   barrier: the y exchange and handoffs of plane i - 1 are complete; the
    //      y exchange of plane i - 2 has been read, so plane i reuses its
    //      buffer; the ring and moment slots loaded next are free;
    //   store of plane i - 3 (staged two iterations ago);
    //   loads of phi(i + 1 + PF) and the moments of i + PF; wait for those of
    //      phi(i + 1) and the moments of i (issued PF iterations earlier);
    //   (e) plane i - 1: y shift and moments, z shift and moments, output of
    //      plane i - 2 (into its staging box);
    //   (d) plane i: interface stencils (phase field of planes i - 1 .. i + 1),
    //      collision, x sweep, y populations into the y exchange of plane i.
    // (e) of one plane and (d) of the next share one stretch of code without a
    // barrier between them; the values (d) hands to (e) live in registers
    // across one barrier.  (e) and (d) run in every iteration, so that stretch
    // has no branch: (e) of planes z0 - 2 and z0 - 1 (first two iterations)
    // and (d) of plane z1 + 1 (last) work on values no stored node depends on
    // (their own planes are not stored, and the z carries they leave are
    // overwritten before the first stored plane), and the output stores of an
    // iteration are predicated on its plane being one of the tile's.
    float2 hYZ[9];
    float hPA[9], hMB[9];
    float2 h_hx = bc(0.f), h_vzp = bc(0.f), h_vzm = bc(0.f);
    float h_dyA = 0.f, h_dyB = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        hYZ[k] = bc(0.f);
        hPA[k] = hMB[k] = 0.f;
    }
    // The z mirror sign and inlet flag of the planes the march meets: the
    // ghost plane below the grid (z = -1, tiles with z0 = 0), the one above
    // (z = nz), interior planes in between.  The imposed inlet velocity of the
    // inlet ghost plane is drawn once per tile: FP32 writes it over the
    // velocity of that plane's moment slot (each staged node at the position
    // it reads, the velocity of its resolved source node, so nodes sharing a
    // source write the same value), where (d) reads it like any plane;
    // 16-bit storage keeps it in registers (with the x / y mirror signs) and
    // selects it for that plane.
    float sgz_lo = 1.f, sgz_hi = 1.f;
    int inl_lo = 0, inl_unused = 0;
    resolve_axis(-1, nz, P.face[4], P.face[5], sgz_lo, inl_lo);
    resolve_axis(nz, nz, P.face[4], P.face[5], sgz_hi, inl_unused);
    [[maybe_unused]] float2 iux = bc(0.f), iuy = bc(0.f), iuz = bc(0.f);
    if (inl_lo && z0 == 0) {
        float ua[3], ub[3];
        inlet_velocity(P, sx, syA, t, ua);
        inlet_velocity(P, sx, syB, t, ub);
        if constexpr (L::kFp32) {  // (the barrier that starts the march orders these writes before (d) reads them)
            S* const m = momb + mslot(z0 - 1) * MSL;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                m[mrdA + (1 + f) * (WR ? fsA : FS)] = ua[f];
                m[mrdB + (1 + f) * (WR ? fsB : FS)] = ub[f];
            }
            fence_proxy_async();  // before a later TMA load writes this slot again
        } else {
            iux = make_float2(ua[0] * sgx, ub[0] * sgx);
            iuy = make_float2(ua[1] * sgyA, ub[1] * sgyB);
            iuz = make_float2(ua[2], ub[2]);
        }
    }
    // (unrolled by two: the z carries and handoffs then pass between the two
    // copies of the body by register renaming instead of moves)
#pragma unroll UR
    for (int i = z0 - 1; i <= z1 + 1; ++i) {
        if (__syncthreads_or(dead)) break;
        const bool dd = i <= z1;  // plane i is one the tile needs (d) of
        // plane i - 3 was staged two iterations ago (and fenced): store it
        if (tst && tid == 0 && i >= z0 + 3) {
            tma_store_4d(&maps->out, outb + obuf(i - 3) * OSL, x0, y0, i - 3, 0);
            bulk_commit();
        }
        const bool do_m = dd && i + PF <= z1, do_p = dd && i + 1 + PF <= z1 + 1;
        if (dd) {
            const int kb = bslot(i);
            if ((do_m || do_p) && issue(do_p, i + 1 + PF, do_m, i + PF, kb)) pend |= 1u << kb;
            if (!tma) cp_async_commit();
            wait_bar(bslot(i + 1));  // == bslot(i - PF)
        }
        // z mirror sign and inlet flag of plane i
        const float sgz_cur = i < 0 ? sgz_lo : (i >= nz ? sgz_hi : 1.f);
        const bool inl_cur = inl_lo && i < 0;
        // the output of (e) in this iteration (plane i - 2) is stored
        const bool outA = storeA && i >= z0 + 2, outB = storeB && i >= z0 + 2;

        // (e) plane i - 1: y shift and moments, z shift and moments, output of plane i - 2
        float2 avg_phi, avg_uz;  // the new phi and u_z of plane i - 2 (time averages)
        {
            if constexpr (L::TC) {  // the handoffs of (d) of plane i - 1, parked in TMEM
                float c[48];
#pragma unroll
                for (int k = 0; k < 6; ++k) tmem_ld8(tm_addr + 64u + 8u * k, c + 8 * k);
                tmem_wait_ld48(c);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    hYZ[k] = make_float2(c[2 * k], c[2 * k + 1]);
                    hPA[k] = c[18 + k];
                    hMB[k] = c[27 + k];
                }
                h_hx = make_float2(c[36], c[37]);
                h_vzp = make_float2(c[38], c[39]);
                h_vzm = make_float2(c[40], c[41]);
                h_dyA = c[42];
                h_dyB = c[43];
            }
            const float* yb = yx + obuf(i - 1) * (20 * NT);
            const float* yprev = yb + (w > 0 ? tid - 32 : tid);       // row 2w-1
            const float* ynext = yb + (w < NW - 1 ? tid + 32 : tid);  // row 2w+2
            float2 Y[3][3][3];
#pragma unroll
            for (int qx = 0; qx < 3; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = 3 * qx + c;
                    if (!L::kFp32 && qx == 2) {  // zeroth y moment only (16-bit forms; see (d))
                        Y[qx][0][c] = make_float2(yprev[(2 * k) * NT], ynext[(2 * k + 1) * NT]) + hYZ[k];
                    } else {
                        const float2 qp = make_float2(yprev[(2 * k) * NT], hPA[k]);
                        const float2 qm = make_float2(hMB[k], ynext[(2 * k + 1) * NT]);
                        const float2 s = qp + qm;
                        Y[qx][0][c] = s + hYZ[k];
                        Y[qx][1][c] = qp - qm;
                        Y[qx][2][c] = s;
                    }
                }
            const float2 hxy = mad(0.125f, make_float2(yprev[18 * NT], h_dyB) + make_float2(h_dyA, ynext[19 * NT]), h_hx);

            if constexpr (L::TC) {
                float c[40];
#pragma unroll
                for (int k = 0; k < 5; ++k) tmem_ld8(tm_addr + 8u * k, c + 8 * k);
                tmem_wait_ld(c);
                carries_unpack(c);
            }
            const int gqx[6] = {0, 1, 0, 2, 0, 1}, gqy[6] = {0, 0, 1, 0, 2, 1};
            float2 O0[6], O1[6], O2[6];
#pragma unroll
            for (int g = 0; g < 6; ++g) {
                const Tri2 tr = pops2(Y[gqx[g]][gqy[g]][0], Y[gqx[g]][gqy[g]][1], Y[gqx[g]][gqy[g]][2]);
                if (g < 3) {
                    O0[g] = cPP[g] + cZ[g] + tr.m;
                    O1[g] = cPP[g] - tr.m;
                    O2[g] = cPP[g] + tr.m;
                    cPP[g] = cP[g];
                    cZ[g] = tr.z;
                } else {
                    O0[g] = cA[g] + tr.m;
                    cA[g] = cP[g] + tr.z;
                }
                cP[g] = tr.p;
            }
            const float2 phin = mad(0.125f, h_vzm, cAph);
            cAph = mad(0.125f, cVP, hxy);
            cVP = h_vzp;
            if constexpr (L::TC) carries_store();

            {  // (every lane computes; halo and out-of-grid lanes, and planes before z0, do not write)
                const float2 dr = O0[0], jx = O0[1], jy = O0[2], jz = O1[0];
                const float2 rn = bc(1.f) + dr, irn = rcp2(rn);
                const float2 ux = jx * irn, uy = jy * irn, uz = jz * irn;
                const float2 rux = rn * ux, ruy = rn * uy, ruz = rn * uz;
                const float2 mdr = (-1.f / 3.f) * dr;
                float2 val[NFIELDS];
                val[F_DRHO] = dr;
                val[F_UX] = ux;
                val[F_UY] = uy;
                val[F_UZ] = uz;
                val[F_PXX] = O0[3] + mdr - rux * ux;
                val[F_PYY] = O0[4] + mdr - ruy * uy;
                val[F_PZZ] = O2[0] + mdr - ruz * uz;
                val[F_PXY] = O0[5] - rux * uy;
                val[F_PXZ] = O1[1] - rux * uz;
                val[F_PYZ] = O1[2] - ruy * uz;
                val[F_PHI] = phin;
                const long long zo = nxy * (i - 2);
                if constexpr (tst) {  // into the staging box of plane i - 2: [field][tile row][tile column]
                    float* ob = outb + obuf(i - 2) * OSL + (2 * w - 1) * TX + (lane - 1);
                    if (outA) {
#pragma unroll
                        for (int f = 0; f < NFIELDS; ++f) ob[f * TY * TX] = val[f].x;
                    }
                    if (outB) {
#pragma unroll
                        for (int f = 0; f < NFIELDS; ++f) ob[f * TY * TX + TX] = val[f].y;
                    }
                } else {
                    if (outA) {
                        S* o = out + zo + sxyA;
#pragma unroll
                        for (int f = 0; f < F_PHI; ++f) Io<S>::st(o + f * fs, val[f].x, P.scale[f]);
                        Io<S>::st_phi(o + F_PHI * fs, val[F_PHI].x, P.scale[F_PHI]);
                    }
                    if (outB) {
                        S* o = out + zo + sxyB;
#pragma unroll
                        for (int f = 0; f < F_PHI; ++f) Io<S>::st(o + f * fs, val[f].y, P.scale[f]);
                        Io<S>::st_phi(o + F_PHI * fs, val[F_PHI].y, P.scale[F_PHI]);
                    }
                }
                if (outA) {
                    sum_rho += Io<S>::round_trip(dr.x, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip_phi(phin.x, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                if (outB) {
                    sum_rho += Io<S>::round_trip(dr.y, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip_phi(phin.y, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                avg_phi = phin;
                avg_uz = uz;
            }
        }

        // (d) plane i: stencils, collision, x sweep, y populations -> y exchange of
        // plane i and the handoffs to its (e) in the next iteration
        {
            const S* mA = momb + mslot(i) * MSL + mrdA;
            const S* mB = momb + mslot(i) * MSL + mrdB;
            auto ld2 = [&](int f) {
                return make_float2(Io<S>::cvt(mA[f * (WR ? fsA : FS)], P.inv_scale[f]),
                                   Io<S>::cvt(mB[f * (WR ? fsB : FS)], P.inv_scale[f]));
            };
            // mirror images: the signs of the x, y, z velocity components and of
            // the off-diagonal P components flip the FP32 sign bit (the ALU
            // pipe, not the FMA pipe that the step is short of)
            const unsigned mz = sgz_cur < 0.f ? 0x80000000u : 0u;
            auto flip = [](float2 v, unsigned ma, unsigned mb) {
                return make_float2(__uint_as_float(__float_as_uint(v.x) ^ ma), __uint_as_float(__float_as_uint(v.y) ^ mb));
            };
            const float2 drho = ld2(0);
            float2 ux = flip(ld2(1), msx, msx), uy = flip(ld2(2), msyA, msyB), uz = flip(ld2(3), mz, mz);
            const float2 pxx = ld2(4), pyy = ld2(5), pzz = ld2(6);
            const float2 pxy = flip(ld2(7), msx ^ msyA, msx ^ msyB), pxz = flip(ld2(8), msx ^ mz, msx ^ mz),
                         pyz = flip(ld2(9), msyA ^ mz, msyB ^ mz);
            if constexpr (!L::kFp32) {
                ux = inl_cur ? iux : ux;
                uy = inl_cur ? iuy : uy;
                uz = inl_cur ? iuz : uz;
            }

            // interface terms from the phase field of planes i - 1, i, i + 1 at
            // rows 2w .. 2w + 3 of the lane's own column (its z combinations S,
            // D, L), the neighbour columns by shuffles (interface_nb)
            float2 phi, Fx, Fy, Fz, nxv, nyv, nzv;
            {
                static_assert(TX <= 28, "the interface stencil takes columns from the spare lanes 30, 31");
                const S* pm = ring + pslot(i - 1) * PSL;
                const S* pc = ring + pslot(i) * PSL;
                const S* pp = ring + pslot(i + 1) * PSL;
                const bool im = inlet_face && i - 1 < 0, ic = inlet_face && i < 0;
                const float inv = P.inv_scale[F_PHI];
                float zS[4], zD[4], zL[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float a = im ? phib4[r] : Io<S>::cvt_phi(pm[rd4[r]], inv);
                    const float b = ic ? phib4[r] : Io<S>::cvt_phi(pc[rd4[r]], inv);
                    const float c = Io<S>::cvt_phi(pp[rd4[r]], inv);
                    const float s = c + a;
                    zS[r] = fmaf(4.f, b, s);
                    zD[r] = c - a;
                    zL[r] = fmaf(-2.f, b, s);
                    if (r == 1) phi.x = b;
                    if (r == 2) phi.y = b;
                }
                // (the inlet ghost plane carries no interface terms)
                interface_nb(zS, zD, zL, lane, sig_half, P.normal_eps2, Fx, Fy, Fz, nxv, nyv, nzv,
                             inl_cur ? 0.f : 1.f);
            }

            // Guo forcing: v = u + F / (2 rho)
            const float2 rho = bc(1.f) + drho;
            const float2 irho = rcp2(rho);
            const float2 hf = 0.5f * irho;
            const float2 vx = mad(hf, Fx, ux), vy = mad(hf, Fy, uy), vz = mad(hf, Fz, uz);

            // D3Q7: g_i^post = w_i (B0 + c_i . B1); x terms by shuffles, the
            // y terms of the row pair's edges through shared memory
            float* yb = yx + obuf(i) * (20 * NT) + tid;
            {
                const float2 ga = P.gamma * (bc(1.f) - phi * phi);
                const float2 fphi = 4.f * phi;
                const float2 b1x = mad(fphi, vx, ga * nxv);
                const float2 b1y = mad(fphi, vy, ga * nyv);
                const float2 b1z = mad(fphi, vz, ga * nzv);
                const float2 fromL = shfl_up2(phi + b1x), fromR = shfl_down2(phi - b1x);
                h_hx = mad(0.25f, phi, 0.125f * (fromL + fromR));
                const float2 yp2 = phi + b1y, ym2 = phi - b1y;
                yb[18 * NT] = yp2.y;
                yb[19 * NT] = ym2.x;
                h_dyA = ym2.y;  // row 2w+1 -> row 2w
                h_dyB = yp2.x;  // row 2w -> row 2w+1
                h_vzp = phi + b1z;
                h_vzm = phi - b1z;
            }

            // collision in Hermite form.  Non-equilibrium second moment relative
            // to rho v v: N = P + rho u u - rho v v = P - (u F + F v) / 2
            // (rho (v - u) = F / 2); forcing products F_a v_b shared with
            // the (1 - omega/2)(v F + F v) term.
            const float2 fvxx = Fx * vx, fvyy = Fy * vy, fvzz = Fz * vz;
            const float2 fxvy = Fx * vy, fxvz = Fx * vz, fyvz = Fy * vz;
            const float2 nxx = mad(-0.5f, mad(Fx, ux, fvxx), pxx);
            const float2 nyy = mad(-0.5f, mad(Fy, uy, fvyy), pyy);
            const float2 nzz = mad(-0.5f, mad(Fz, uz, fvzz), pzz);
            const float2 nxy = mad(-0.5f, mad(ux, Fy, fxvy), pxy);
            const float2 nxz = mad(-0.5f, mad(ux, Fz, fxvz), pxz);
            const float2 nyz = mad(-0.5f, mad(uy, Fz, fyvz), pyz);
            float2 X[3][8];
            collide_xsweep2(rho, drho, ux, uy, uz, vx, vy, vz, Fx, Fy, Fz, nxx, nyy, nzz, nxy, nxz, nyz, fvxx, fvyy,
                            fvzz, mad(vx, Fy, fxvy), mad(vx, Fz, fxvz), mad(vy, Fz, fyvz), om1, fo, X);

            // y populations; the row pair exchanges inside the thread, the pair
            // edges go through shared memory: p(+1) of row 2w+1 to the thread
            // below, p(-1) of row 2w to the thread above
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int qx = 0; qx < 3; ++qx) {
                    const float2 b0 = X[qx][3 * c], b1 = X[qx][3 * c + 1];
                    const Tri2 tr = c < 2 ? pops2(b0, b1, X[qx][3 * c + 2]) : pops2_01(b0, b1);
                    const int k = 3 * qx + c;
                    yb[(2 * k) * NT] = tr.p.y;
                    yb[(2 * k + 1) * NT] = tr.m.x;
                    if (!L::kFp32 && qx == 2) {
                        // (16-bit forms, short of registers) x moment 2 needs only the zeroth
                        // y moment: the own rows' part of it is handed over as one sum
                        hYZ[k] = make_float2(tr.z.x + tr.m.y, tr.z.y + tr.p.x);
                        hPA[k] = hMB[k] = 0.f;
                    } else {
                        hYZ[k] = tr.z;
                        hPA[k] = tr.p.x;
                        hMB[k] = tr.m.y;
                    }
                }
        }

        if constexpr (L::TC) {  // park this plane's handoffs in TMEM until its (e) in the next iteration
            float c[48];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                c[2 * k] = hYZ[k].x, c[2 * k + 1] = hYZ[k].y;
                c[18 + k] = hPA[k];
                c[27 + k] = hMB[k];
            }
            c[36] = h_hx.x, c[37] = h_hx.y, c[38] = h_vzp.x, c[39] = h_vzp.y;
            c[40] = h_vzm.x, c[41] = h_vzm.y, c[42] = h_dyA, c[43] = h_dyB;
#pragma unroll
            for (int k = 44; k < 48; ++k) c[k] = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) tmem_st8(tm_addr + 64u + 8u * k, c + 8 * k);
            tmem_wait_st48(c);
        }
        // time sums of the new phi and u_z of plane i - 2 (FP64; TILE_TMA is
        // launched only without them)
        if (MODE != TILE_TMA && P.avg && (outA || outB)) {
            const long long zo = nxy * (i - 2);
            if (outA) {
                double* a = P.avg + zo + sxyA;
                a[0] += (double)avg_phi.x;
                a[fs] += (double)avg_uz.x;
            }
            if (outB) {
                double* a = P.avg + zo + sxyB;
                a[0] += (double)avg_phi.y;
                a[fs] += (double)avg_uz.y;
            }
        }
        // element-wise copies land by the end of the iteration that issued them
        // (the barrier then publishes them to the threads that read them)
        if (!tma) cp_async_wait<0>();
        commit(do_p, i + 1 + PF, do_m, i + PF);
        if (tst) {
            fence_proxy_async();  // the staging box is read by a TMA store after the barrier
            // the store issued this iteration has read its box before the box
            // takes the plane after next
            if (tid == 0) bulk_wait_read<0>();
        }
    }
    // the last plane (z1 - 1) waits in its staging box
    if constexpr (L::TC) tmem_fence_before();
    __syncthreads();
    if constexpr (L::TC) {  // every TMEM access of the block has completed: release the columns
        tmem_fence_after();
        if (w == 0) tmem_dealloc(tm_base, L::TM_COLS);
    }
    if (tst && tid == 0) {
        if (!dead) {
            tma_store_4d(&maps->out, outb + obuf(z1 - 1) * OSL, x0, y0, z1 - 1, 0);
            bulk_commit();
        }
        bulk_wait<0>();
    }
    cp_async_wait<0>();
    // Loads still in flight after a failed wait (the march stopped early):
    // give them a bounded chance to land before the mbarriers are invalidated,
    // since a copy must not complete on an invalidated barrier.  If one does
    // not land, the barriers are left as they are and the tile reports it.
    bool drained = true;
    for (int k = 0; k < NB; ++k)
        if ((pend >> k) & 1u) drained = mbar_wait(bar + k, (phase >> k) & 1u) && drained;
    const bool clean = __syncthreads_and(drained) != 0;
    if (use_maps && tid == 0 && clean)  // the next tile of a persistent block initialises them again
        for (int k = 0; k < NB; ++k) mbar_inval(bar + k);
    if (!clean && tid == 0 && P.err) *P.err = 1;

    double a = sum_rho, b = sum_phi;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(FULL, a, off);
        b += __shfl_xor_sync(FULL, b, off);
    }
    __syncthreads();
    double* red = reinterpret_cast<double*>(yx);
    if (lane == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int k = 0; k < NW; ++k) {
            A += red[2 * k];
            B += red[2 * k + 1];
        }
        part[0] = A;
        part[1] = B;
    }
    __syncthreads();  // shared memory is reused by the block's next tile
    return clean;
}

// Whether a tile's finished planes leave through the staging boxes: the
// kernel form has them and the maps carry an output map for this block size.
template <int NW, typename S, bool ST, bool WR>
__device__ __forceinline__ bool staged_stores(const TileMaps* maps) {
    return Step2Smem<NW, S, ST, WR>::kTmaStore && maps != nullptr && maps->valid && maps->block_warps == NW &&
           maps->store;
}

// One time step of one grid: one block per tile.  TO: every tile of the
// grid loads by TMA (tile_class_kernel said so), the march is compiled for
// that path alone.
template <int NW, typename S, bool ST, bool WR, bool TO = false>
__global__ void __launch_bounds__(32 * NW, 1)
    step2_kernel(const __grid_constant__ StepParams P, const __grid_constant__ TileMaps M, const S* __restrict__ in,
                 S* __restrict__ out, const long long* __restrict__ t_in, long long* __restrict__ t_out,
                 double* __restrict__ partials) {
    constexpr int MODE = TO ? TILE_TMA : TILE_ANY, UR = TO ? 4 : 2;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const long long t = *t_in;
    if constexpr (Step2Smem<NW, S, ST, WR>::kTmaStore) {
        if (staged_stores<NW, S, ST, WR>(&M))
            step_tile<NW, S, ST, WR, true, MODE, UR>(P, &M, in, out, t, blockIdx.x, blockIdx.y, blockIdx.z,
                                                     partials + 2 * blk);
        else
            step_tile<NW, S, ST, WR, false, MODE, UR>(P, &M, in, out, t, blockIdx.x, blockIdx.y, blockIdx.z,
                                                      partials + 2 * blk);
    } else {
        step_tile<NW, S, ST, WR, false, MODE, UR>(P, &M, in, out, t, blockIdx.x, blockIdx.y, blockIdx.z,
                                                  partials + 2 * blk);
    }
    if (blk == 0 && threadIdx.x == 0 && threadIdx.y == 0) *t_out = t + 1;
}

// Tile classification: each block runs the set-up of its tile in the step
// kernel form <NW, S, ST, WR> (x-y tile (blockIdx.x, blockIdx.y); the choice
// does not depend on z) and ORs 1 into *flag if that tile would load element
// by element.  M: maps flags only (valid, block_warps, wrap); the choice
// depends on the grid, its faces and the box shapes, not on the buffers.
template <int NW, typename S, bool ST, bool WR>
__global__ void __launch_bounds__(32 * NW, 1)
    tile_class_kernel(const __grid_constant__ StepParams P, const __grid_constant__ TileMaps M, int* __restrict__ flag) {
    const bool ok =
        step_tile<NW, S, ST, WR, false, TILE_CLASSIFY>(P, &M, nullptr, nullptr, 0, blockIdx.x, blockIdx.y, 0, nullptr);
    if (!ok && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(flag, 1);
}

// One time step of a batch of independent grids in one persistent launch:
// each block takes the next tile of the batch's tile list from a device
// counter (tiles[k] = instance, bx, by, bz) until the list is exhausted.  The
// instance's parameters are staged in shared memory for the tile; its tensor
// maps are read from the instance table in device memory.  counters[q]
// serves the steps of parity q; each launch zeroes the other one for the next.
// TO: every tile of every grid loads by TMA (tile_class_kernel said so).
template <int NW, bool ST, bool WR, bool TO = false>
__global__ void __launch_bounds__(32 * NW, 1)
    step_batch_kernel(const BatchInstance* __restrict__ insts, const int4* __restrict__ tiles, int ntiles,
                      int parity, const long long* __restrict__ t_in, long long* __restrict__ t_out,
                      int* __restrict__ counters, double* __restrict__ partials) {
    __shared__ StepParams sP;
    __shared__ const float* s_io[2];
    __shared__ int s_tile;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const long long t = *t_in;
    if (blockIdx.x == 0 && tid == 0) counters[parity ^ 1] = 0;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&counters[parity], 1);
        __syncthreads();
        const int k = s_tile;
        if (k >= ntiles) break;
        const int4 tl = tiles[k];
        {
            const int* src = reinterpret_cast<const int*>(&insts[tl.x].p);
            int* dst = reinterpret_cast<int*>(&sP);
            for (int i = tid; i < (int)(sizeof(StepParams) / sizeof(int)); i += 32 * NW) dst[i] = src[i];
            if (tid == 0) {
                s_io[0] = static_cast<const float*>(insts[tl.x].buf[parity]);
                s_io[1] = static_cast<const float*>(insts[tl.x].buf[parity ^ 1]);
            }
        }
        __syncthreads();
        // the grid's tensor maps live in device memory, written before the launch
        const TileMaps* maps = &insts[tl.x].maps[parity];
        if (tid == 0) fence_tensormap_acquire(maps);
        constexpr int MODE = TO ? TILE_TMA : TILE_ANY;
        float* const o = const_cast<float*>(s_io[1]);
        bool clean;
        if constexpr (Step2Smem<NW, float, ST, WR>::kTmaStore) {
            clean = staged_stores<NW, float, ST, WR>(maps)
                        ? step_tile<NW, float, ST, WR, true, MODE>(sP, maps, s_io[0], o, t, tl.y, tl.z, tl.w,
                                                                   partials + 2 * k)
                        : step_tile<NW, float, ST, WR, false, MODE>(sP, maps, s_io[0], o, t, tl.y, tl.z, tl.w,
                                                                    partials + 2 * k);
        } else {
            clean = step_tile<NW, float, ST, WR, false, MODE>(sP, maps, s_io[0], o, t, tl.y, tl.z, tl.w,
                                                              partials + 2 * k);
        }
        if (!clean) break;  // loads that never landed: take no further tile into this shared memory
    }
    if (blockIdx.x == 0 && tid == 0) *t_out = t + 1;
}

// ------------------------------------------------------ state conversion

constexpr int CONV_THREADS = 256;

template <typename S>
__device__ void block_partials(float a, float b, double* partials) {
    __shared__ double ra[CONV_THREADS / 32], rb[CONV_THREADS / 32];
    double da = a, db = b;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        da += __shfl_xor_sync(FULL, da, off);
        db += __shfl_xor_sync(FULL, db, off);
    }
    if ((threadIdx.x & 31) == 0) {
        ra[threadIdx.x >> 5] = da;
        rb[threadIdx.x >> 5] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < CONV_THREADS / 32; ++w) {
            A += ra[w];
            B += rb[w];
        }
        partials[2 * blockIdx.x] = A;
        partials[2 * blockIdx.x + 1] = B;
    }
}

template <typename S>
__global__ void __launch_bounds__(CONV_THREADS) put_field_kernel(const __grid_constant__ StepParams P,
                                                                 const float* __restrict__ src, int field,
                                                                 S* __restrict__ st) {
    const long long N = (long long)P.nx * P.ny * P.nz;
    S* dst = st + field_slot(P.closure, field) * P.fstride;
    const float sc = P.scale[field];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = src[i];
        if (field == F_PHI)
            Io<S>::st_phi(dst + i, v, sc);
        else
            Io<S>::st(dst + i, field == F_DRHO ? v - 1.f : v, sc);
    }
}

template <typename S>
__global__ void __launch_bounds__(CONV_THREADS) state_sums_kernel(const __grid_constant__ StepParams P,
                                                                  const S* __restrict__ st,
                                                                  double* partials) {
    const long long N = (long long)P.nx * P.ny * P.nz, fs = P.fstride;
    float sr = 0.f, sp = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        sr += Io<S>::ld(st + F_DRHO * fs + i, P.inv_scale[F_DRHO]);
        sp += Io<S>::ld_phi(st + field_slot(P.closure, F_PHI) * fs + i, P.inv_scale[F_PHI]);
    }
    block_partials<S>(sr, sp, partials);
}

template <typename S>
__global__ void __launch_bounds__(CONV_THREADS) get_field_kernel(const __grid_constant__ StepParams P,
                                                                 const S* __restrict__ st, int field,
                                                                 float* __restrict__ dst) {
    const long long N = (long long)P.nx * P.ny * P.nz;
    const S* src = st + field_slot(P.closure, field) * P.fstride;
    const float inv = P.inv_scale[field];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = field == F_PHI ? Io<S>::ld_phi(src + i, inv) : Io<S>::ld(src + i, inv);
        dst[i] = field == F_DRHO ? 1.f + v : v;
    }
}

constexpr int FIN_THREADS = 256;

__global__ void __launch_bounds__(FIN_THREADS) finish_sums_kernel(const double* __restrict__ partials,
                                                                  int n, double* __restrict__ result) {
    __shared__ double sa[FIN_THREADS], sb[FIN_THREADS];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += FIN_THREADS) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = FIN_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        result[0] = sa[0];
        result[1] = sb[0];
    }
}

int conv_blocks(const StepParams& p) {
    const long long N = (long long)p.nx * p.ny * p.nz;
    long long b = (N + CONV_THREADS - 1) / CONV_THREADS;
    return (int)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

template <int NW, typename S, bool ST, bool WR, bool TO = false>
cudaError_t launch_nw(const StepParams& p, int storage, const void* in, void* out, const long long* t_in,
                      long long* t_out, double* partials, cudaStream_t s, const TileMaps* maps) {
    const LaunchShape sh = step_shape(p, storage);
    TileMaps none;
    if (!maps) {
        memset(&none, 0, sizeof(none));
        maps = &none;
    }
    step2_kernel<NW, S, ST, WR, TO><<<sh.grid, sh.block, Step2Smem<NW, S, ST, WR>::BYTES, s>>>(
        p, *maps, static_cast<const S*>(in), static_cast<S*>(out), t_in, t_out, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step_t(const StepParams& p, int st, const void* in, void* out, const long long* t_in,
                          long long* t_out, double* partials, cudaStream_t s, const TileMaps* m) {
    // 12 warps, staged stores: the TMA-only form where every tile loads by TMA
    const bool to = m && m->valid && m->all_tma && p.block_warps == 12 && p.plain_stores == 0;
    if constexpr (sizeof(S) == 4) {  // FP32 blocks of 8 or 12 warps: plain-store and periodic-face forms
        const bool pl = p.plain_stores != 0, wr = m && m->valid && m->wrap;
        if (p.block_warps == 8) {
            if (wr) return pl ? launch_nw<8, S, false, true>(p, st, in, out, t_in, t_out, partials, s, m)
                              : launch_nw<8, S, true, true>(p, st, in, out, t_in, t_out, partials, s, m);
            if (pl) return launch_nw<8, S, false, false>(p, st, in, out, t_in, t_out, partials, s, m);
        }
        if (p.block_warps == 12) {
            if (wr) return pl   ? launch_nw<12, S, false, true>(p, st, in, out, t_in, t_out, partials, s, m)
                           : to ? launch_nw<12, S, true, true, true>(p, st, in, out, t_in, t_out, partials, s, m)
                                : launch_nw<12, S, true, true>(p, st, in, out, t_in, t_out, partials, s, m);
            if (pl) return launch_nw<12, S, false, false>(p, st, in, out, t_in, t_out, partials, s, m);
        }
        if (p.block_warps == 16 && pl) return launch_nw<16, S, false, false>(p, st, in, out, t_in, t_out, partials, s, m);
    }
    switch (p.block_warps) {
        case 8: return launch_nw<8, S, true, false>(p, st, in, out, t_in, t_out, partials, s, m);
        case 12: return to ? launch_nw<12, S, true, false, true>(p, st, in, out, t_in, t_out, partials, s, m)
                           : launch_nw<12, S, true, false>(p, st, in, out, t_in, t_out, partials, s, m);
        case 14: return launch_nw<14, S, true, false>(p, st, in, out, t_in, t_out, partials, s, m);
        case 16: return launch_nw<16, S, true, false>(p, st, in, out, t_in, t_out, partials, s, m);
        default: return cudaErrorInvalidValue;
    }
}

template <int NW, typename S, bool ST, bool WR, bool TO = false>
cudaError_t prepare_nw() {
    return cudaFuncSetAttribute(step2_kernel<NW, S, ST, WR, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Step2Smem<NW, S, ST, WR>::BYTES);
}

// Whether every tile of the grid loads by TMA in the 12-warp staged-store
// form (with side boxes if WR): one tile_class_kernel launch into *flag.
template <typename S, bool WR>
cudaError_t classify_t(const StepParams& p, int storage, int* flag, cudaStream_t s) {
    StepParams q = p;
    q.block_warps = 12;
    q.plain_stores = 0;
    const LaunchShape sh = step_shape(q, storage);
    TileMaps m;
    memset(&m, 0, sizeof(m));
    m.valid = 1;
    m.block_warps = 12;
    m.wrap = WR ? 1 : 0;
    tile_class_kernel<12, S, true, WR><<<dim3(sh.grid.x, sh.grid.y, 1), dim3(32, 12, 1), 0, s>>>(q, m, flag);
    return cudaGetLastError();
}

template <int NW, bool ST, bool WR, bool TO = false>
cudaError_t launch_batch_nw(const BatchInstance* insts, const int4* tiles, int ntiles, int parity,
                            const long long* t_in, long long* t_out, int* counters, double* partials, int sms,
                            cudaStream_t s) {
    step_batch_kernel<NW, ST, WR, TO><<<sms, dim3(32, NW, 1), Step2Smem<NW, float, ST, WR>::BYTES, s>>>(
        insts, tiles, ntiles, parity, t_in, t_out, counters, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t prepare_t() {
    cudaError_t e = prepare_nw<8, S, true, false>();
    if (e == cudaSuccess) e = prepare_nw<12, S, true, false>();
    if (e == cudaSuccess) e = prepare_nw<12, S, true, false, true>();
    if (e == cudaSuccess) e = prepare_nw<14, S, true, false>();
    if (e == cudaSuccess) e = prepare_nw<16, S, true, false>();
    if constexpr (sizeof(S) == 4) {
        if (e == cudaSuccess) e = prepare_nw<8, S, false, false>();
        if (e == cudaSuccess) e = prepare_nw<12, S, false, false>();
        if (e == cudaSuccess) e = prepare_nw<16, S, false, false>();
        if (e == cudaSuccess) e = prepare_nw<8, S, true, true>();
        if (e == cudaSuccess) e = prepare_nw<12, S, true, true>();
        if (e == cudaSuccess) e = prepare_nw<12, S, true, true, true>();
        if (e == cudaSuccess) e = prepare_nw<8, S, false, true>();
        if (e == cudaSuccess) e = prepare_nw<12, S, false, true>();
    }
    return e;
}

template <int NW, bool ST, bool WR, bool TO = false>
cudaError_t prepare_batch_nw() {
    return cudaFuncSetAttribute(step_batch_kernel<NW, ST, WR, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Step2Smem<NW, float, ST, WR>::BYTES);
}

}  // namespace

static_assert(sizeof(StepParams) % sizeof(int) == 0, "StepParams is copied as ints");

cudaError_t prepare_batch_kernels() {
    cudaError_t e = prepare_batch_nw<8, true, false>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, true, false>();
    if (e == cudaSuccess) e = prepare_batch_nw<8, false, false>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, false, false>();
    if (e == cudaSuccess) e = prepare_batch_nw<8, true, true>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, true, true>();
    if (e == cudaSuccess) e = prepare_batch_nw<8, false, true>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, false, true>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, true, false, true>();
    if (e == cudaSuccess) e = prepare_batch_nw<12, true, true, true>();
    return e;
}

cudaError_t launch_batch_step(int nw, bool plain, bool wrap, bool tma_only, const BatchInstance* insts,
                              const int4* tiles, int ntiles, int parity, const long long* t_in, long long* t_out,
                              int* counters, double* partials, int sms, cudaStream_t s) {
#define TSLB_BATCH(NW_, ST_, WR_) \
    launch_batch_nw<NW_, ST_, WR_>(insts, tiles, ntiles, parity, t_in, t_out, counters, partials, sms, s)
    if (nw == 12 && !plain && tma_only)
        return wrap ? launch_batch_nw<12, true, true, true>(insts, tiles, ntiles, parity, t_in, t_out, counters,
                                                            partials, sms, s)
                    : launch_batch_nw<12, true, false, true>(insts, tiles, ntiles, parity, t_in, t_out, counters,
                                                             partials, sms, s);
    if (nw == 8) return wrap ? (plain ? TSLB_BATCH(8, false, true) : TSLB_BATCH(8, true, true))
                             : (plain ? TSLB_BATCH(8, false, false) : TSLB_BATCH(8, true, false));
    if (nw == 12) return wrap ? (plain ? TSLB_BATCH(12, false, true) : TSLB_BATCH(12, true, true))
                              : (plain ? TSLB_BATCH(12, false, false) : TSLB_BATCH(12, true, false));
#undef TSLB_BATCH
    return cudaErrorInvalidValue;
}

cudaError_t tiles_all_tma(const StepParams& p, int storage, bool wrap, int* flag, cudaStream_t s, bool* all) {
    *all = false;
    if (p.closure != CL_PROJECTION || (wrap && storage != ST_FP32)) return cudaSuccess;
    int h = 1;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        switch (storage) {
            case ST_FP32:
                e = wrap ? classify_t<float, true>(p, storage, flag, s) : classify_t<float, false>(p, storage, flag, s);
                break;
            case ST_FP16: e = classify_t<__half, false>(p, storage, flag, s); break;
            case ST_BF16: e = classify_t<__nv_bfloat16, false>(p, storage, flag, s); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) *all = h == 0;
    return e;
}

cudaError_t prepare_kernels(int storage) {
    switch (storage) {
        case ST_FP32: return prepare_t<float>();
        case ST_FP16: return prepare_t<__half>();
        case ST_BF16: return prepare_t<__nv_bfloat16>();
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
size_t step_smem_bytes_t(int nw, bool plain) {
    if (sizeof(S) == 4 && plain && nw == 8) return Step2Smem<8, S, false>::BYTES;
    if (sizeof(S) == 4 && plain && nw == 12) return Step2Smem<12, S, false>::BYTES;
    if (sizeof(S) == 4 && plain && nw == 16) return Step2Smem<16, S, false>::BYTES;
    switch (nw) {
        case 8: return Step2Smem<8, S>::BYTES;
        case 12: return Step2Smem<12, S>::BYTES;
        case 14: return Step2Smem<14, S>::BYTES;
        default: return Step2Smem<16, S>::BYTES;
    }
}

size_t step_smem_bytes(int nw, int storage, bool plain) {
    return storage == ST_FP32 ? step_smem_bytes_t<float>(nw, plain) : step_smem_bytes_t<__half>(nw, plain);
}

LaunchShape step_shape(const StepParams& p, int storage) {
    LaunchShape sh;
    sh.nw = p.block_warps;
    const int ty = 2 * sh.nw - 2;
    const int tx = TX;  // 28 interior columns for every kernel
    sh.grid = dim3((p.nx + tx - 1) / tx, (p.ny + ty - 1) / ty, (p.nz + p.tile_z - 1) / p.tile_z);
    sh.block = dim3(32, sh.nw, 1);
    sh.smem = step_smem_bytes(sh.nw, storage, p.plain_stores != 0);
    return sh;
}

int max_partials(const StepParams& p, int storage) {
    StepParams q = p;
    q.block_warps = 8;  // the smallest tile gives the most blocks
    q.tile_z = 1;       // ... and so does the thinnest slab
    const LaunchShape sh = step_shape(q, storage);
    const long long steps = (long long)sh.grid.x * sh.grid.y * sh.grid.z;
    const int conv = conv_blocks(p);
    return (int)(steps > conv ? steps : conv);
}

cudaError_t launch_step(const StepParams& p, int storage, const void* in, void* out, const long long* t_in,
                        long long* t_out, double* partials, cudaStream_t s, const TileMaps* maps) {
    switch (storage) {
        case ST_FP32: return launch_step_t<float>(p, storage, in, out, t_in, t_out, partials, s, maps);
        case ST_FP16: return launch_step_t<__half>(p, storage, in, out, t_in, t_out, partials, s, maps);
        case ST_BF16: return launch_step_t<__nv_bfloat16>(p, storage, in, out, t_in, t_out, partials, s, maps);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled of the driver, looked up through the runtime (the
// library does not link libcuda directly); null if unavailable.
EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}

template <typename S>
cudaError_t make_maps_t(const StepParams& p, const void* buf, const void* obuf, TileMaps* m) {
    const int nw = p.block_warps;
    const int nr = 2 * nw;
    const int mw = Step2Smem<8, S>::MW, pw = Step2Smem<8, S>::PW, txs = Step2Smem<8, S>::TXS;
    const cuuint64_t es = sizeof(S);
    const CUtensorMapDataType dt = sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    EncodeTiled enc = encode_tiled();
    if (!enc) return cudaSuccess;  // valid stays 0: element-wise loads
    // (a grid with a HALO face also stores its ghost planes after the interior)
    const cuuint64_t nzs = (cuuint64_t)p.nz + (has_halo(p.face) ? kHaloPlanes : 0);
    const cuuint64_t dm[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, nzs, 10};
    const cuuint64_t sm[3] = {p.nx * es, (cuuint64_t)p.nx * p.ny * es, (cuuint64_t)p.fstride * es};
    const cuuint32_t bm[4] = {(cuuint32_t)mw, (cuuint32_t)nr, 1, 10};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    CUresult r = enc(&m->mom, dt, 4, const_cast<void*>(buf), dm, sm, bm, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaSuccess;
    const cuuint32_t bp[3] = {(cuuint32_t)pw, (cuuint32_t)(nr + 2), 1};
    const void* pbase = static_cast<const char*>(buf) + (size_t)F_PHI * p.fstride * es;
    r = enc(&m->phi, dt, 3, const_cast<void*>(pbase), dm, sm, bp, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaSuccess;
    m->valid = 1;
    m->block_warps = nw;
    if (Step2Smem<8, S>::kFp32 && (p.face[0] == BC_PERIODIC || p.face[2] == BC_PERIODIC)) {
        // side boxes of ghosts across periodic faces (see step_tile)
        const cuuint32_t bmx[4] = {4, (cuuint32_t)nr, 1, 10}, bmy[4] = {(cuuint32_t)mw, 1, 1, 10};
        const cuuint32_t bmc[4] = {4, 1, 1, 10};
        const cuuint32_t bpx[3] = {4, (cuuint32_t)(nr + 2), 1}, bpy[3] = {(cuuint32_t)pw, 2, 1}, bpc[3] = {4, 2, 1};
        bool ok = true;
        auto enc4 = [&](CUtensorMap* t, const cuuint32_t* b) {
            ok = ok && enc(t, dt, 4, const_cast<void*>(buf), dm, sm, b, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        auto enc3 = [&](CUtensorMap* t, const cuuint32_t* b) {
            ok = ok && enc(t, dt, 3, const_cast<void*>(pbase), dm, sm, b, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        enc4(&m->momx, bmx);
        enc4(&m->momy, bmy);
        enc4(&m->momc, bmc);
        enc3(&m->phix, bpx);
        enc3(&m->phiy, bpy);
        enc3(&m->phic, bpc);
        m->wrap = ok ? 1 : 0;
    }
    if (Step2Smem<8, S>::kFp32 && obuf && reinterpret_cast<uintptr_t>(obuf) % 16 == 0) {
        const cuuint64_t dout[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, (cuuint64_t)NFIELDS};
        const cuuint32_t bo[4] = {(cuuint32_t)txs, (cuuint32_t)(nr - 2), 1, (cuuint32_t)NFIELDS};
        r = enc(&m->out, dt, 4, const_cast<void*>(obuf), dout, sm, bo, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) m->store = 1;
    }
    return cudaSuccess;
}
}  // namespace

// Output map of the Chapman-Enskog step (FP32): the 5 stored fields of the
// output buffer as {nx, ny, nz, 5}, boxes of [5][2 nw - 2 rows][28 columns].
static cudaError_t make_ce_out_map(const StepParams& p, const void* obuf, TileMaps* m) {
    EncodeTiled enc = encode_tiled();
    if (!enc || !obuf || reinterpret_cast<uintptr_t>(obuf) % 16 != 0) return cudaSuccess;
    const cuuint64_t es = sizeof(float);
    const cuuint64_t dout[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, 5};
    const cuuint64_t sm[3] = {p.nx * es, (cuuint64_t)p.nx * p.ny * es, (cuuint64_t)p.fstride * es};
    const cuuint32_t bo[4] = {(cuuint32_t)TX, (cuuint32_t)(2 * p.block_warps - 2), 1, 5};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(&m->out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(obuf), dout, sm, bo, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        m->store = 1;
        m->block_warps = p.block_warps;
    }
    return cudaSuccess;
}

cudaError_t make_tile_maps(const StepParams& p, int storage, const void* buf, const void* obuf, TileMaps* maps) {
    memset(maps, 0, sizeof(*maps));
    const size_t es = storage == ST_FP32 ? 4 : 2;
    // the Chapman-Enskog step loads element by element; FP32 grids with
    // 16-byte rows get its output map (staged TMA stores)
    if (p.closure == CL_CHAPMAN_ENSKOG) {
        if (storage != ST_FP32 || ((size_t)p.nx * es) % 16 != 0 || (p.block_warps != 8 && p.block_warps != 12))
            return cudaSuccess;
        return make_ce_out_map(p, obuf, maps);
    }
    // TMA needs 16-byte aligned row pitches and bases; box sizes exist for 8, 12, 14 and 16 warps
    if (p.closure != CL_PROJECTION || ((size_t)p.nx * es) % 16 != 0 ||
        (reinterpret_cast<uintptr_t>(buf) % 16) != 0 ||
        (p.block_warps != 8 && p.block_warps != 12 && p.block_warps != 14 && p.block_warps != 16))
        return cudaSuccess;
    return storage == ST_FP32 ? make_maps_t<float>(p, buf, obuf, maps) : make_maps_t<__half>(p, buf, obuf, maps);
}

cudaError_t launch_put_field(const StepParams& p, int storage, const float* src, int field, void* state,
                             cudaStream_t s) {
    const int b = conv_blocks(p);
    switch (storage) {
        case ST_FP32:
            put_field_kernel<float><<<b, CONV_THREADS, 0, s>>>(p, src, field, static_cast<float*>(state));
            break;
        case ST_FP16:
            put_field_kernel<__half><<<b, CONV_THREADS, 0, s>>>(p, src, field, static_cast<__half*>(state));
            break;
        case ST_BF16:
            put_field_kernel<__nv_bfloat16><<<b, CONV_THREADS, 0, s>>>(p, src, field,
                                                                      static_cast<__nv_bfloat16*>(state));
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_get_field(const StepParams& p, int storage, const void* state, int field, float* dst,
                             cudaStream_t s) {
    const int b = conv_blocks(p);
    switch (storage) {
        case ST_FP32:
            get_field_kernel<float><<<b, CONV_THREADS, 0, s>>>(p, static_cast<const float*>(state), field, dst);
            break;
        case ST_FP16:
            get_field_kernel<__half><<<b, CONV_THREADS, 0, s>>>(p, static_cast<const __half*>(state), field, dst);
            break;
        case ST_BF16:
            get_field_kernel<__nv_bfloat16><<<b, CONV_THREADS, 0, s>>>(
                p, static_cast<const __nv_bfloat16*>(state), field, dst);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_state_sums(const StepParams& p, int storage, const void* state, double* partials, int* nparts,
                              cudaStream_t s) {
    const int b = conv_blocks(p);
    *nparts = b;
    switch (storage) {
        case ST_FP32:
            state_sums_kernel<float><<<b, CONV_THREADS, 0, s>>>(p, static_cast<const float*>(state), partials);
            break;
        case ST_FP16:
            state_sums_kernel<__half><<<b, CONV_THREADS, 0, s>>>(p, static_cast<const __half*>(state), partials);
            break;
        case ST_BF16:
            state_sums_kernel<__nv_bfloat16><<<b, CONV_THREADS, 0, s>>>(
                p, static_cast<const __nv_bfloat16*>(state), partials);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_finish_sums(const double* partials, int n, double* result, cudaStream_t s) {
    finish_sums_kernel<<<1, FIN_THREADS, 0, s>>>(partials, n, result);
    return cudaGetLastError();
}

}  // namespace tslb
