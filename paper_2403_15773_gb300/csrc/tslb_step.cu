// Fused time step of the multicomponent thread-safe lattice Boltzmann method
// (arXiv 2403.15773) for sm_103a, and the small kernels around it.
//
// One launch = one time step over the whole grid.  Each thread block owns a
// slab of 30 x TY interior columns and marches through its z range plane by
// plane.  A warp holds one row of 32 staged columns (30 interior + 2 halo);
// the block holds TY interior rows plus one halo row above and below.
//
// Per staged node and plane the kernel
//   1. reads the moments (rho - 1, u, P) and the phase field of the node and of
//      its ghost images (cp.async prefetch one plane ahead; ghosts follow the
//      face rules: wrap, mirror, zero-gradient copy, jet inlet);
//   2. evaluates grad phi and its Hessian with the isotropic D3Q27 stencils,
//      the normal n, the curvature kappa = div n and the surface-tension force
//      F = -(sigma/2) kappa grad phi (Sec. 2.2);
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
//      phi', and accumulates the FP64 block partials of sum(rho - 1), sum(phi).
//
// All arithmetic is FP32 and works with deviations from the rest state
// (rho - 1, Pi - cs2 I) so that no O(1) terms cancel.
#include "tslb_device.cuh"

namespace tslb {
namespace {

// ----------------------------------------------------- step kernel (pairs)

template <int NW>
struct Step2Smem {
    static constexpr int NT = 32 * NW;              // threads
    static constexpr int NR = 2 * NW;               // staged rows (two per warp)
    static constexpr int NS = 32 * NR;              // staged nodes
    static constexpr int NPH = PHX * (NR + 2);      // phase-field elements (halo 2)
    static constexpr int RING = 0;                  // [4][NPH] phase-field planes
    static constexpr int ZC = RING + 4 * NPH;       // [2][3][NPH] z combinations of phi
    static constexpr int MOM = ZC + 6 * NPH;        // [2][10][NS] staged moments
    static constexpr int YX = MOM + 20 * NS;        // [2][20][NT] y exchange
    static constexpr int FLOATS = YX + 40 * NT;
    static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

// One tile of one time step: the 30 x (2 NW - 2) interior columns at tile
// (bx, by), planes [bz * tile_z, (bz + 1) * tile_z), from state `in` (step t)
// to state `out`; writes the tile's FP64 partial sums to part[0..1].
template <int NW, typename S>
__device__ __forceinline__ void step_tile(const StepParams& P, const S* __restrict__ in, S* __restrict__ out,
                                          const long long t, const int bx, const int by, const int bz,
                                          double* __restrict__ part) {
    using L = Step2Smem<NW>;
    constexpr int NT = L::NT, NR = L::NR, NS = L::NS, NPH = L::NPH;
    constexpr int TY = NR - 2;
    constexpr int EPT = (NPH + NT - 1) / NT;
    extern __shared__ __align__(16) float smem[];
    float* const ring = smem + L::RING;
    float* const zc = smem + L::ZC;
    float* const mom = smem + L::MOM;
    float* const yx = smem + L::YX;

    const int lane = threadIdx.x, w = threadIdx.y, tid = lane + 32 * w;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const long long fs = P.fstride;
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * P.tile_z;
    const int z1 = min(z0 + P.tile_z, nz);

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
    const int sA = lane + 64 * w;                           // staged-node slot of row 2w (row 2w+1: +32)

    int pxy[EPT];
    float phib[EPT];
    const bool inlet_planes = P.face[4] == BC_INLET && z0 < 2;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int idx = tid + e * NT;
        pxy[e] = 0;
        phib[e] = 0.f;
        if (idx < NPH) {
            float sg;
            const int psx = resolve_axis(x0 - 2 + idx % PHX, nx, P.face[0], P.face[1], sg, unused);
            const int psy = resolve_axis(y0 - 2 + idx / PHX, ny, P.face[2], P.face[3], sg, unused);
            pxy[e] = psx + nx * psy;
            if (inlet_planes) phib[e] = inlet_phi(P, psx, psy);
        }
    }

    // FP32: cp.async straight into shared memory, one plane ahead.  16-bit
    // storage: the next plane's raw values wait in registers while the
    // current plane is computed and are widened into the same shared-memory
    // slots afterwards (each slot is read only by the thread that fills it).
    unsigned short rphi[EPT], rmom[2][10];
    int rphi_inl = 0;
    auto issue_phi = [&](int q) {
        float sg;
        int inl = 0;
        const int sz = resolve_axis(q, nz, P.face[4], P.face[5], sg, inl);
        float* dst = ring + ((q + 8) & 3) * NPH;
        const S* src = in + F_PHI * fs + nxy * sz;
        rphi_inl = inl;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int idx = tid + e * NT;
            if (idx < NPH) {
                if (inl) {
                    dst[idx] = phib[e];
                } else if constexpr (Io<S>::kAsync) {
                    cp_async4(dst + idx, reinterpret_cast<const float*>(src + pxy[e]));
                } else {
                    rphi[e] = __ldg(reinterpret_cast<const unsigned short*>(src + pxy[e]));
                }
            }
        }
    };
    auto commit_phi = [&](int q) {
        if constexpr (!Io<S>::kAsync) {
            if (!rphi_inl) {
                float* dst = ring + ((q + 8) & 3) * NPH;
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    const int idx = tid + e * NT;
                    if (idx < NPH) dst[idx] = Io<S>::from_raw(rphi[e], P.inv_scale[F_PHI]);
                }
            }
        }
    };
    auto issue_mom = [&](int q, float& sgz, int& inl) {
        inl = 0;
        const int sz = resolve_axis(q, nz, P.face[4], P.face[5], sgz, inl);
        float* dst = mom + ((q + 8) & 1) * 10 * NS + sA;
        const S* srcA = in + nxy * sz + sxyA;
        const S* srcB = in + nxy * sz + sxyB;
#pragma unroll
        for (int f = 0; f < 10; ++f) {
            if constexpr (Io<S>::kAsync) {
                cp_async4(dst + f * NS, reinterpret_cast<const float*>(srcA + f * fs));
                cp_async4(dst + f * NS + 32, reinterpret_cast<const float*>(srcB + f * fs));
            } else {
                rmom[0][f] = __ldg(reinterpret_cast<const unsigned short*>(srcA + f * fs));
                rmom[1][f] = __ldg(reinterpret_cast<const unsigned short*>(srcB + f * fs));
            }
        }
    };
    auto commit_mom = [&](int q) {
        if constexpr (!Io<S>::kAsync) {
            float* dst = mom + ((q + 8) & 1) * 10 * NS + sA;
#pragma unroll
            for (int f = 0; f < 10; ++f) {
                dst[f * NS] = Io<S>::from_raw(rmom[0][f], P.inv_scale[f]);
                dst[f * NS + 32] = Io<S>::from_raw(rmom[1][f], P.inv_scale[f]);
            }
        }
    };

    float sgz_cur, sgz_nxt;
    int inl_cur, inl_nxt;
    for (int q = z0 - 2; q <= z0 + 1; ++q) {
        issue_phi(q);
        commit_phi(q);
    }
    issue_mom(z0 - 1, sgz_cur, inl_cur);
    commit_mom(z0 - 1);
    cp_async_commit();

    float2 cPP[6], cP[6], cZ[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) cPP[k] = cP[k] = cZ[k] = bc(0.f);
    float2 cH = bc(0.f), cVPP = bc(0.f), cVP = bc(0.f);
    float sum_rho = 0.f, sum_phi = 0.f;

    // S: what stage (d) of a plane hands to stage (e) of the same plane one
    // iteration later (y populations kept in the thread, D3Q7 x/z terms)
    float2 sYZ[9];
    float sPA[9], sMB[9];
    float2 s_hx = bc(0.f), s_vzp = bc(0.f), s_vzm = bc(0.f);
    float s_dyA = 0.f, s_dyB = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        sYZ[k] = bc(0.f);
        sPA[k] = sMB[k] = 0.f;
    }
    // the first iteration's stage (e) reads a y-exchange buffer no stage (d)
    // has written: clear both buffers
    for (int k = tid; k < 40 * NT; k += NT) yx[k] = 0.f;

    const float om1 = 1.f - P.omega, fo = 1.f - 0.5f * P.omega;
    const float sig_half = -0.5f * P.sigma;

    // prologue: z combinations of plane z0 - 1
    cp_async_wait<0>();
    {
        const int i = z0 - 2;
        {  // z combinations of phi at plane i + 1
            const float* pm = ring + ((i + 8) & 3) * NPH;
            const float* pc = ring + ((i + 1 + 8) & 3) * NPH;
            const float* pp = ring + ((i + 2 + 8) & 3) * NPH;
            float* z = zc + ((i + 1 + 8) & 1) * 3 * NPH;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int idx = tid + e * NT;
                if (idx < NPH) {
                    const float a = pm[idx], b = pc[idx], c = pp[idx];
                    z[idx] = b;
                    z[NPH + idx] = c + a;
                    z[2 * NPH + idx] = c - a;
                }
            }
        }

    }
    __syncthreads();

    // Software-pipelined march, one barrier per iteration i:
    //   (c) z combinations of plane i + 1,
    //   (e) y / z stages of plane i - 1 (output of plane i - 2),
    //   (d) stencils, collision and x sweep of plane i.
    // Each shared buffer (zc, yx: two each by plane parity; the phase-field
    // ring; the moment slots) is last read one barrier before it is rewritten.
    for (int i = z0 - 1; i <= z1 + 1; ++i) {
        issue_phi(i + 3);
        issue_mom(i + 1, sgz_nxt, inl_nxt);
        cp_async_commit();
        cp_async_wait<1>();

        {  // z combinations of phi at plane i + 1
            const float* pm = ring + ((i + 8) & 3) * NPH;
            const float* pc = ring + ((i + 1 + 8) & 3) * NPH;
            const float* pp = ring + ((i + 2 + 8) & 3) * NPH;
            float* z = zc + ((i + 1 + 8) & 1) * 3 * NPH;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int idx = tid + e * NT;
                if (idx < NPH) {
                    const float a = pm[idx], b = pc[idx], c = pp[idx];
                    z[idx] = b;
                    z[NPH + idx] = c + a;
                    z[2 * NPH + idx] = c - a;
                }
            }
        }

        // (e) plane i - 1: y shift and moments, z shift and moments, output of plane i - 2
        {
            const float* yprev = yx + ((i - 1 + 8) & 1) * 20 * NT + (w > 0 ? tid - 32 : tid);       // row 2w-1
            const float* ynext = yx + ((i - 1 + 8) & 1) * 20 * NT + (w < NW - 1 ? tid + 32 : tid);  // row 2w+2
            float2 Y[3][3][3];
#pragma unroll
            for (int qx = 0; qx < 3; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = 3 * qx + c;
                    const float2 qp = make_float2(yprev[(2 * k) * NT], sPA[k]);
                    const float2 qm = make_float2(sMB[k], ynext[(2 * k + 1) * NT]);
                    const float2 s = qp + qm;
                    Y[qx][0][c] = s + sYZ[k];
                    Y[qx][1][c] = qp - qm;
                    Y[qx][2][c] = s;
                }
            const float2 hxy = mad(0.125f, make_float2(yprev[18 * NT], s_dyB) + make_float2(s_dyA, ynext[19 * NT]), s_hx);

            const int gqx[6] = {0, 1, 0, 2, 0, 1}, gqy[6] = {0, 0, 1, 0, 2, 1};
            float2 O0[6], O1[6], O2[6];
#pragma unroll
            for (int g = 0; g < 6; ++g) {
                const Tri2 tr = pops2(Y[gqx[g]][gqy[g]][0], Y[gqx[g]][gqy[g]][1], Y[gqx[g]][gqy[g]][2]);
                O0[g] = cPP[g] + cZ[g] + tr.m;
                O1[g] = cPP[g] - tr.m;
                O2[g] = cPP[g] + tr.m;
                cPP[g] = cP[g];
                cP[g] = tr.p;
                cZ[g] = tr.z;
            }
            const float2 phin = mad(0.125f, cVPP + s_vzm, cH);
            cH = hxy;
            cVPP = cVP;
            cVP = s_vzp;

            if (i >= z0 + 2 && i <= z1 + 1 && (storeA || storeB)) {
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
                if (storeA) {
                    S* o = out + zo + sxyA;
#pragma unroll
                    for (int f = 0; f < NFIELDS; ++f) Io<S>::st(o + f * fs, val[f].x, P.scale[f]);
                    sum_rho += Io<S>::round_trip(dr.x, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip(phin.x, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                if (storeB) {
                    S* o = out + zo + sxyB;
#pragma unroll
                    for (int f = 0; f < NFIELDS; ++f) Io<S>::st(o + f * fs, val[f].y, P.scale[f]);
                    sum_rho += Io<S>::round_trip(dr.y, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip(phin.y, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                if (P.avg) {  // time sums of the new phi and u_z (FP64)
                    if (storeA) {
                        double* a = P.avg + zo + sxyA;
                        a[0] += (double)phin.x;
                        a[fs] += (double)uz.x;
                    }
                    if (storeB) {
                        double* a = P.avg + zo + sxyB;
                        a[0] += (double)phin.y;
                        a[fs] += (double)uz.y;
                    }
                }
            }
        }

        float2 nYZ[9];
        float nPA[9], nMB[9];
        float2 n_hx, n_vzp, n_vzm;
        float n_dyA, n_dyB;
        // (d) plane i: stencils, collision, x sweep, y populations -> yx[i], S
        {
            const float* m = mom + ((i + 8) & 1) * 10 * NS + sA;
            auto ld2 = [&](int f) { return make_float2(m[f * NS], m[f * NS + 32]); };
            const float2 sgy = make_float2(sgyA, sgyB);
            const float2 drho = ld2(0);
            float2 ux = sgx * ld2(1), uy = sgy * ld2(2), uz = sgz_cur * ld2(3);
            const float2 pxx = ld2(4), pyy = ld2(5), pzz = ld2(6);
            const float2 pxy = (sgx * sgy) * ld2(7), pxz = (sgx * sgz_cur) * ld2(8), pyz = (sgz_cur * sgy) * ld2(9);
            if (inl_cur) {
                float ua[3], ub[3];
                inlet_velocity(P, sx, syA, t, ua);
                inlet_velocity(P, sx, syB, t, ub);
                ux = make_float2(ua[0] * sgx, ub[0] * sgx);
                uy = make_float2(ua[1] * sgyA, ub[1] * sgyB);
                uz = make_float2(ua[2], ub[2]);
            }

            // interface terms from the z combinations of phi at plane i
            float2 phi, Fx, Fy, Fz, nxv, nyv, nzv;
            interface2<NPH>(zc + ((i + 8) & 1) * 3 * NPH, lane, w, sig_half, P.normal_eps2, phi, Fx, Fy, Fz,
                            nxv, nyv, nzv);
            if (inl_cur) {
                Fx = Fy = Fz = bc(0.f);
                nxv = nyv = nzv = bc(0.f);
            }

            // collision in Hermite form (Guo forcing: v = u + F / (2 rho))
            const float2 rho = bc(1.f) + drho;
            const float2 irho = rcp2(rho);
            const float2 hf = 0.5f * irho;
            const float2 hfx = hf * Fx, hfy = hf * Fy, hfz = hf * Fz;
            const float2 vx = ux + hfx, vy = uy + hfy, vz = uz + hfz;
            const float2 nxx = pxx - rho * mad(ux, hfx, hfx * vx);
            const float2 nyy = pyy - rho * mad(uy, hfy, hfy * vy);
            const float2 nzz = pzz - rho * mad(uz, hfz, hfz * vz);
            const float2 nxy = pxy - rho * mad(ux, hfy, hfx * vy);
            const float2 nxz = pxz - rho * mad(ux, hfz, hfx * vz);
            const float2 nyz = pyz - rho * mad(uy, hfz, hfy * vz);
            float2 X[3][8];
            const float2 zero = bc(0.f);
            collide_xsweep2(rho, drho, ux, uy, uz, vx, vy, vz, Fx, Fy, Fz, nxx, nyy, nzz, nxy, nxz, nyz, om1, fo, X);

            // y populations; the row pair exchanges inside the thread, the pair
            // edges go through shared memory: p(+1) of row 2w+1 to the thread
            // below, p(-1) of row 2w to the thread above
            float* yb = yx + ((i + 8) & 1) * 20 * NT + tid;
#pragma unroll
            for (int qx = 0; qx < 3; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 b0 = X[qx][3 * c], b1 = X[qx][3 * c + 1];
                    const float2 b2 = c < 2 ? X[qx][3 * c + 2] : zero;
                    const Tri2 tr = pops2(b0, b1, b2);
                    const int k = 3 * qx + c;
                    yb[(2 * k) * NT] = tr.p.y;
                    yb[(2 * k + 1) * NT] = tr.m.x;
                    nYZ[k] = tr.z;
                    nPA[k] = tr.p.x;
                    nMB[k] = tr.m.y;
                }

            // D3Q7: g_i^post = w_i (B0 + c_i . B1)
            const float2 ga = P.gamma * (bc(1.f) - phi * phi);
            const float2 fphi = 4.f * phi;
            const float2 b1x = mad(fphi, vx, ga * nxv);
            const float2 b1y = mad(fphi, vy, ga * nyv);
            const float2 b1z = mad(fphi, vz, ga * nzv);
            const float2 fromL = shfl_up2(phi + b1x), fromR = shfl_down2(phi - b1x);
            n_hx = mad(0.25f, phi, 0.125f * (fromL + fromR));
            const float2 yp = phi + b1y, ym = phi - b1y;
            yb[18 * NT] = yp.y;
            yb[19 * NT] = ym.x;
            n_dyA = ym.y;  // row 2w+1 -> row 2w
            n_dyB = yp.x;  // row 2w -> row 2w+1
            n_vzp = phi + b1z;
            n_vzm = phi - b1z;
        }
        __syncthreads();
        commit_phi(i + 3);
        commit_mom(i + 1);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            sYZ[k] = nYZ[k];
            sPA[k] = nPA[k];
            sMB[k] = nMB[k];
        }
        s_hx = n_hx;
        s_vzp = n_vzp;
        s_vzm = n_vzm;
        s_dyA = n_dyA;
        s_dyB = n_dyB;
        sgz_cur = sgz_nxt;
        inl_cur = inl_nxt;
    }
    cp_async_wait<0>();

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
}

// One time step of one grid: one block per tile.
template <int NW, typename S>
__global__ void __launch_bounds__(32 * NW, 1)
    step2_kernel(const __grid_constant__ StepParams P, const S* __restrict__ in, S* __restrict__ out,
                 const long long* __restrict__ t_in, long long* __restrict__ t_out,
                 double* __restrict__ partials) {
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const long long t = *t_in;
    step_tile<NW, S>(P, in, out, t, blockIdx.x, blockIdx.y, blockIdx.z, partials + 2 * blk);
    if (blk == 0 && threadIdx.x == 0 && threadIdx.y == 0) *t_out = t + 1;
}

// One time step of a batch of independent grids in one persistent launch:
// each block takes the next tile of the batch's tile list from a device
// counter (tiles[k] = instance, bx, by, bz) until the list is exhausted.  The
// instance's parameters are staged in shared memory for the tile.  counters[q]
// serves the steps of parity q; each launch zeroes the other one for the next.
template <int NW>
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
        step_tile<NW, float>(sP, s_io[0], const_cast<float*>(s_io[1]), t, tl.y, tl.z, tl.w, partials + 2 * k);
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
        sp += Io<S>::ld(st + field_slot(P.closure, F_PHI) * fs + i, P.inv_scale[F_PHI]);
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
        const float v = Io<S>::ld(src + i, inv);
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

template <int NW, typename S>
cudaError_t launch_nw(const StepParams& p, const void* in, void* out, const long long* t_in, long long* t_out,
                      double* partials, cudaStream_t s) {
    const LaunchShape sh = step_shape(p, ST_FP32);
    step2_kernel<NW, S><<<sh.grid, sh.block, sh.smem, s>>>(p, static_cast<const S*>(in), static_cast<S*>(out),
                                                           t_in, t_out, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step_t(const StepParams& p, const void* in, void* out, const long long* t_in,
                          long long* t_out, double* partials, cudaStream_t s) {
    switch (p.block_warps) {
        case 8: return launch_nw<8, S>(p, in, out, t_in, t_out, partials, s);
        case 12: return launch_nw<12, S>(p, in, out, t_in, t_out, partials, s);
        case 16: return launch_nw<16, S>(p, in, out, t_in, t_out, partials, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int NW, typename S>
cudaError_t prepare_nw() {
    return cudaFuncSetAttribute(step2_kernel<NW, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Step2Smem<NW>::BYTES);
}

template <int NW>
cudaError_t launch_batch_nw(const BatchInstance* insts, const int4* tiles, int ntiles, int parity,
                            const long long* t_in, long long* t_out, int* counters, double* partials, int nblocks,
                            cudaStream_t s) {
    step_batch_kernel<NW><<<nblocks, dim3(32, NW, 1), Step2Smem<NW>::BYTES, s>>>(insts, tiles, ntiles, parity, t_in,
                                                                                  t_out, counters, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t prepare_t() {
    cudaError_t e = prepare_nw<8, S>();
    if (e == cudaSuccess) e = prepare_nw<12, S>();
    if (e == cudaSuccess) e = prepare_nw<16, S>();
    return e;
}

}  // namespace

static_assert(sizeof(StepParams) % sizeof(int) == 0, "StepParams is copied as ints");

cudaError_t prepare_batch_kernels() {
    cudaError_t e = cudaFuncSetAttribute(step_batch_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Step2Smem<8>::BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Step2Smem<12>::BYTES);
    return e;
}

cudaError_t launch_batch_step(int nw, const BatchInstance* insts, const int4* tiles, int ntiles, int parity,
                              const long long* t_in, long long* t_out, int* counters, double* partials,
                              int nblocks, cudaStream_t s) {
    switch (nw) {
        case 8: return launch_batch_nw<8>(insts, tiles, ntiles, parity, t_in, t_out, counters, partials, nblocks, s);
        case 12: return launch_batch_nw<12>(insts, tiles, ntiles, parity, t_in, t_out, counters, partials, nblocks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_kernels(int storage) {
    switch (storage) {
        case ST_FP32: return prepare_t<float>();
        case ST_FP16: return prepare_t<__half>();
        case ST_BF16: return prepare_t<__nv_bfloat16>();
        default: return cudaErrorInvalidValue;
    }
}

size_t step_smem_bytes(int nw) {
    switch (nw) {
        case 8: return Step2Smem<8>::BYTES;
        case 12: return Step2Smem<12>::BYTES;
        default: return Step2Smem<16>::BYTES;
    }
}

LaunchShape step_shape(const StepParams& p, int /*storage*/) {
    LaunchShape sh;
    sh.nw = p.block_warps;
    const int ty = 2 * sh.nw - 2;
    sh.grid = dim3((p.nx + TX - 1) / TX, (p.ny + ty - 1) / ty, (p.nz + p.tile_z - 1) / p.tile_z);
    sh.block = dim3(32, sh.nw, 1);
    sh.smem = step_smem_bytes(sh.nw);
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
                        long long* t_out, double* partials, cudaStream_t s) {
    switch (storage) {
        case ST_FP32: return launch_step_t<float>(p, in, out, t_in, t_out, partials, s);
        case ST_FP16: return launch_step_t<__half>(p, in, out, t_in, t_out, partials, s);
        case ST_BF16: return launch_step_t<__nv_bfloat16>(p, in, out, t_in, t_out, partials, s);
        default: return cudaErrorInvalidValue;
    }
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
