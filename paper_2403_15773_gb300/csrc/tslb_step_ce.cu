// Fused time step with the Chapman-Enskog closure of the non-equilibrium
// second moment (Sec. 2.1, recursive regularisation):
//   a2_neq = -(cs2 / omega) (d_a j_b + d_b j_a),
// the gradient of the momentum j = rho u taken by the isotropic D3Q27 stencil
// (1/cs2) sum_i w_i c_i j(x + c_i).  The state then holds only rho - 1, u and
// phi (5 fields, 40 bytes per node and step in FP32 instead of 88): P is
// neither read nor written.
//
// The tile, the z march and the streaming sweeps are those of the projection
// kernel (tslb_step.cu).  What changes:
//   * rho - 1 and u are staged like phi, on the 34 x (rows + 2) footprint of
//     the tile (halo 2), in a ring of four planes, and turned into j (with the
//     mirror signs of ghost images and the imposed inlet velocity) once per
//     plane;
//   * the z combinations S'j = j(z-1) + 4 j(z) + j(z+1) and Dj = j(z+1) -
//     j(z-1) of each plane are formed once per footprint node; the nine
//     derivatives d_a j_b of the staged row pair then follow from y and x
//     combinations (d_x = D_x S'_y S'_z / 72 and its permutations);
//   * only the moments rho, j are gathered after streaming: the sweeps carry
//     the x moments 0 and 1 and the (x, y) moment pairs (0,0), (1,0), (0,1).
#include <cstring>

#include "tslb_device.cuh"

namespace tslb {
namespace {

template <int NW>
struct StepCeSmem {
    static constexpr int NT = 32 * NW;              // threads
    static constexpr int NR = 2 * NW;               // staged rows (two per warp)
    static constexpr int NPH = PHX * (NR + 2);      // footprint nodes of a plane (halo 2)
    static constexpr int RING = 0;                  // [4][NPH] phase-field planes
    static constexpr int ZC = RING + 4 * NPH;       // [2][3][NPH] z combinations of phi
    static constexpr int JR = ZC + 6 * NPH;         // [4][4][NPH] planes of rho - 1, j
    static constexpr int JZ4 = JR + 16 * NPH;       // [2][NPH] (S'jx, S'jy, S'jz, Djx)
    static constexpr int JZ2 = JZ4 + 8 * NPH;       // [2][NPH] (Djy, Djz)
    static constexpr int YX = JZ2 + 4 * NPH;        // [2][14][NT] y exchange
    static constexpr int FLOATS = YX + 28 * NT;
    static constexpr size_t BYTES = sizeof(float) * FLOATS;
    // FP32 form with staged stores: two output staging boxes [5][TY][TX] of
    // finished planes that leave by TMA store (+ slack to align them to 128 B)
    static constexpr int TY = NR - 2;
    static constexpr int OUT_BOX = (5 * TY * TX + 31) / 32 * 32;  // box stride, a multiple of 128 bytes
    static constexpr int OUT = FLOATS;
    static constexpr size_t BYTES_ST = sizeof(float) * (OUT + 2 * OUT_BOX + 32);
    static_assert(JZ4 % 4 == 0 && JZ2 % 2 == 0, "vector slots must be aligned");
    static_assert((TX * sizeof(float)) % 16 == 0, "store box rows must be 16-byte multiples");
    static_assert(BYTES_ST <= 227 * 1024, "more shared memory than a block can have");
};

constexpr int PHI_SLOT = 4;  // buffer slot of phi under this closure

// ST: finished planes (FP32) are staged in shared memory and leave by one TMA
// store per plane (maps->out, 5 fields), instead of plain stores.
template <int NW, typename S, bool ST>
__device__ __forceinline__ void step_tile_ce(const StepParams& P, const TileMaps* maps, const S* __restrict__ in,
                                             S* __restrict__ out, const long long t, const int bx, const int by,
                                             const int bz, double* __restrict__ part) {
    using L = StepCeSmem<NW>;
    constexpr int NT = L::NT, NR = L::NR, NPH = L::NPH;
    constexpr int TY = NR - 2;
    constexpr int EPT = (NPH + NT - 1) / NT;
    extern __shared__ __align__(16) float smem[];
    float* const ring = smem + L::RING;
    float* const zc = smem + L::ZC;
    float* const jr = smem + L::JR;
    float4* const jz4 = reinterpret_cast<float4*>(smem + L::JZ4);
    float2* const jz2 = reinterpret_cast<float2*>(smem + L::JZ2);
    float* const yx = smem + L::YX;
    // (ST) the staging boxes, 128-byte aligned within the dynamic shared memory
    [[maybe_unused]] float* const outb =
        smem + L::OUT + ((0u - (unsigned)__cvta_generic_to_shared(smem + L::OUT)) & 127u) / sizeof(float);

    const int lane = threadIdx.x, w = threadIdx.y, tid = lane + 32 * w;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const long long fs = P.fstride;
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * P.tile_z;
    const int z1 = min(z0 + P.tile_z, nz);

    // the staged pair of this thread: rows 2w, 2w+1 of the tile, column lane
    const int gx = x0 - 1 + lane, gyA = y0 - 1 + 2 * w, gyB = gyA + 1;
    const bool col_ok = lane >= 1 && lane <= TX && gx < nx;
    const bool storeA = col_ok && w >= 1 && gyA < ny;       // staged row 2w is interior for w >= 1
    const bool storeB = col_ok && w <= NW - 2 && gyB < ny;  // staged row 2w+1 for w <= NW-2
    const long long oB = gx + (long long)nx * gyB;           // interior offsets when stored
    const long long oA = oB - nx;

    // footprint nodes of this thread: source offset in the plane, mirror signs
    int pxy[EPT];
    unsigned mirror = 0;  // bit 2e: x mirror image, bit 2e+1: y mirror image
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int idx = tid + e * NT;
        pxy[e] = 0;
        if (idx < NPH) {
            float sgx, sgy;
            int unused = 0;
            const int psx = resolve_axis(x0 - 2 + idx % PHX, nx, P.face[0], P.face[1], sgx, unused);
            const int psy = resolve_axis(y0 - 2 + idx / PHX, ny, P.face[2], P.face[3], sgy, unused);
            pxy[e] = psx + nx * psy;
            mirror |= (sgx < 0.f ? 1u : 0u) << (2 * e);
            mirror |= (sgy < 0.f ? 1u : 0u) << (2 * e + 1);
        }
    }

    // rho - 1 and u of a footprint node -> rho - 1 and j of its image in the
    // slots of plane q (inlet ghosts: rho of the fluid node, imposed u)
    auto to_j = [&](float* dst, int idx, int e, float dr, float ux, float uy, float uz, float sgz, int inl) {
        if (inl) {
            float ui[3];
            inlet_velocity(P, pxy[e] % nx, pxy[e] / nx, t, ui);
            ux = ui[0];
            uy = ui[1];
            uz = ui[2];
        }
        const float rho = 1.f + dr;
        const float sx = (mirror >> (2 * e)) & 1u ? -rho : rho;
        const float sy = (mirror >> (2 * e + 1)) & 1u ? -rho : rho;
        dst[idx] = dr;
        dst[NPH + idx] = sx * ux;
        dst[2 * NPH + idx] = sy * uy;
        dst[3 * NPH + idx] = (sgz * rho) * uz;
    };

    // FP32: cp.async straight into shared memory, three planes ahead, turned
    // into j in place when the plane is first used.  16-bit storage: the raw
    // values wait in registers and are widened and turned into j after the
    // iteration's barrier.  Every footprint slot is filled, converted and
    // combined along z by one thread.
    unsigned short rphi[EPT], rj[4][EPT];
    int r_inl = 0;
    float r_sgz = 1.f;
    auto issue = [&](int q) {
        float sgz;
        int inl = 0;
        const int sz = resolve_axis(q, nz, P.face[4], P.face[5], sgz, inl);
        float* dphi = ring + ((q + 8) & 3) * NPH;
        float* dj = jr + ((q + 8) & 3) * 4 * NPH;
        const S* src = in + nxy * sz;
        r_inl = inl;
        r_sgz = sgz;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int idx = tid + e * NT;
            if (idx < NPH) {
                if (inl) {
                    dphi[idx] = inlet_phi(P, pxy[e] % nx, pxy[e] / nx);
                } else if constexpr (Io<S>::kAsync) {
                    cp_async4(dphi + idx, reinterpret_cast<const float*>(src + PHI_SLOT * fs + pxy[e]));
                } else {
                    rphi[e] = __ldg(reinterpret_cast<const unsigned short*>(src + PHI_SLOT * fs + pxy[e]));
                }
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    if constexpr (Io<S>::kAsync)
                        cp_async4(dj + f * NPH + idx, reinterpret_cast<const float*>(src + f * fs + pxy[e]));
                    else
                        rj[f][e] = __ldg(reinterpret_cast<const unsigned short*>(src + f * fs + pxy[e]));
                }
            }
        }
    };
    auto commit = [&](int q) {
        if constexpr (!Io<S>::kAsync) {
            float* dphi = ring + ((q + 8) & 3) * NPH;
            float* dj = jr + ((q + 8) & 3) * 4 * NPH;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int idx = tid + e * NT;
                if (idx < NPH) {
                    if (!r_inl) dphi[idx] = Io<S>::from_raw_phi(rphi[e], P.inv_scale[F_PHI]);
                    to_j(dj, idx, e, Io<S>::from_raw(rj[0][e], P.inv_scale[F_DRHO]),
                         Io<S>::from_raw(rj[1][e], P.inv_scale[F_UX]), Io<S>::from_raw(rj[2][e], P.inv_scale[F_UY]),
                         Io<S>::from_raw(rj[3][e], P.inv_scale[F_UZ]), r_sgz, r_inl);
                }
            }
        }
    };
    // FP32: the plane q has landed; rho - 1, u -> rho - 1, j in place
    auto convert = [&](int q) {
        if constexpr (Io<S>::kAsync) {
            float sgz;
            int inl = 0;
            resolve_axis(q, nz, P.face[4], P.face[5], sgz, inl);
            float* dj = jr + ((q + 8) & 3) * 4 * NPH;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int idx = tid + e * NT;
                if (idx < NPH)
                    to_j(dj, idx, e, dj[idx], dj[NPH + idx], dj[2 * NPH + idx], dj[3 * NPH + idx], sgz, inl);
            }
        }
    };
    // z combinations of plane q from planes q - 1, q, q + 1: phi (value, sum,
    // difference) and j (S' = sum + 4 value, D = difference)
    auto zcombine = [&](int q) {
        const float* pm = ring + ((q - 1 + 8) & 3) * NPH;
        const float* pc = ring + ((q + 8) & 3) * NPH;
        const float* pp = ring + ((q + 1 + 8) & 3) * NPH;
        float* z = zc + ((q + 8) & 1) * 3 * NPH;
        const float* jm = jr + ((q - 1 + 8) & 3) * 4 * NPH;
        const float* jc = jr + ((q + 8) & 3) * 4 * NPH;
        const float* jp = jr + ((q + 1 + 8) & 3) * 4 * NPH;
        float4* z4 = jz4 + ((q + 8) & 1) * NPH;
        float2* z2 = jz2 + ((q + 8) & 1) * NPH;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int idx = tid + e * NT;
            if (idx < NPH) {
                const float a = pm[idx], b = pc[idx], c = pp[idx];
                z[idx] = b;
                z[NPH + idx] = c + a;
                z[2 * NPH + idx] = c - a;
                float sj[3], dj[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float am = jm[(1 + k) * NPH + idx], ac = jc[(1 + k) * NPH + idx],
                                ap = jp[(1 + k) * NPH + idx];
                    sj[k] = fmaf(4.f, ac, am + ap);
                    dj[k] = ap - am;
                }
                z4[idx] = make_float4(sj[0], sj[1], sj[2], dj[0]);
                z2[idx] = make_float2(dj[1], dj[2]);
            }
        }
    };

    for (int q = z0 - 2; q <= z0 + 1; ++q) {
        issue(q);
        commit(q);
    }
    cp_async_commit();

    float2 cPP[3], cP[3], cZ[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) cPP[k] = cP[k] = cZ[k] = bc(0.f);
    float2 cH = bc(0.f), cVPP = bc(0.f), cVP = bc(0.f);
    float sum_rho = 0.f, sum_phi = 0.f;

    // S: what stage (d) of a plane hands to stage (e) of the same plane one
    // iteration later (y populations kept in the thread, D3Q7 x/z terms)
    float2 sYZ[6];
    float sPA[6], sMB[6];
    float2 s_hx = bc(0.f), s_vzp = bc(0.f), s_vzm = bc(0.f);
    float s_dyA = 0.f, s_dyB = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        sYZ[k] = bc(0.f);
        sPA[k] = sMB[k] = 0.f;
    }
    for (int k = tid; k < 28 * NT; k += NT) yx[k] = 0.f;

    const float om1 = 1.f - P.omega, fo = 1.f - 0.5f * P.omega;
    const float sig_half = -0.5f * P.sigma;
    const float cce = -1.f / (216.f * P.omega);  // -(cs2 / omega) / 72

    // prologue: planes z0 - 2 .. z0 in j form, z combinations of plane z0 - 1
    cp_async_wait<0>();
    convert(z0 - 2);
    convert(z0 - 1);
    convert(z0);
    zcombine(z0 - 1);
    __syncthreads();

    // Software-pipelined march, one barrier per iteration i:
    //   (c) plane i + 2 to j form, z combinations of plane i + 1,
    //   (e) y / z stages of plane i - 1 (output of plane i - 2),
    //   (d) stencils, collision and x sweep of plane i.
    for (int i = z0 - 1; i <= z1 + 1; ++i) {
        // plane i - 3 was staged two iterations ago (and fenced): store it
        if (ST && tid == 0 && i >= z0 + 3) {
            tma_store_4d(&maps->out, outb + ((i - 3 + 8) & 1) * L::OUT_BOX, x0, y0, i - 3, 0);
            bulk_commit();
        }
        issue(i + 3);
        cp_async_commit();
        cp_async_wait<1>();
        convert(i + 2);
        zcombine(i + 1);

        // (e) plane i - 1: y shift and moments, z shift and moments, output of plane i - 2
        {
            const float* yprev = yx + ((i - 1 + 8) & 1) * 14 * NT + (w > 0 ? tid - 32 : tid);       // row 2w-1
            const float* ynext = yx + ((i - 1 + 8) & 1) * 14 * NT + (w < NW - 1 ? tid + 32 : tid);  // row 2w+2
            float2 Y0[2][3], Y1[3];  // Y0[qx][c]: y moment 0 of x moment qx; Y1[c]: y moment 1 of x moment 0
#pragma unroll
            for (int qx = 0; qx < 2; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = 3 * qx + c;
                    const float2 qp = make_float2(yprev[(2 * k) * NT], sPA[k]);
                    const float2 qm = make_float2(sMB[k], ynext[(2 * k + 1) * NT]);
                    Y0[qx][c] = qp + qm + sYZ[k];
                    if (qx == 0) Y1[c] = qp - qm;
                }
            const float2 hxy = mad(0.125f, make_float2(yprev[12 * NT], s_dyB) + make_float2(s_dyA, ynext[13 * NT]), s_hx);

            // groups: (x, y) moments (0,0), (1,0), (0,1)
            float2 O0[3], O1z;
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const float2* yg = g == 0 ? Y0[0] : g == 1 ? Y0[1] : Y1;
                const Tri2 tr = pops2(yg[0], yg[1], yg[2]);
                O0[g] = cPP[g] + cZ[g] + tr.m;
                if (g == 0) O1z = cPP[g] - tr.m;
                cPP[g] = cP[g];
                cP[g] = tr.p;
                cZ[g] = tr.z;
            }
            const float2 phin = mad(0.125f, cVPP + s_vzm, cH);
            cH = hxy;
            cVPP = cVP;
            cVP = s_vzp;

            if (i >= z0 + 2 && i <= z1 + 1 && (storeA || storeB)) {
                const float2 dr = O0[0];
                const float2 irn = rcp2(bc(1.f) + dr);
                const float2 ux = O0[1] * irn, uy = O0[2] * irn, uz = O1z * irn;
                const float2 val[5] = {dr, ux, uy, uz, phin};
                const int fld[5] = {F_DRHO, F_UX, F_UY, F_UZ, F_PHI};
                const long long zo = nxy * (i - 2);
                if constexpr (ST) {  // into the staging box of plane i - 2: [field][tile row][tile column]
                    float* ob = outb + ((i - 2 + 8) & 1) * L::OUT_BOX + (2 * w - 1) * TX + (lane - 1);
                    if (storeA) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) ob[f * TY * TX] = val[f].x;
                    }
                    if (storeB) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) ob[f * TY * TX + TX] = val[f].y;
                    }
                } else {
                    if (storeA) {
                        S* o = out + zo + oA;
#pragma unroll
                        for (int f = 0; f < 4; ++f) Io<S>::st(o + f * fs, val[f].x, P.scale[fld[f]]);
                        Io<S>::st_phi(o + 4 * fs, val[4].x, P.scale[F_PHI]);
                    }
                    if (storeB) {
                        S* o = out + zo + oB;
#pragma unroll
                        for (int f = 0; f < 4; ++f) Io<S>::st(o + f * fs, val[f].y, P.scale[fld[f]]);
                        Io<S>::st_phi(o + 4 * fs, val[4].y, P.scale[F_PHI]);
                    }
                }
                if (storeA) {
                    sum_rho += Io<S>::round_trip(dr.x, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip_phi(phin.x, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                if (storeB) {
                    sum_rho += Io<S>::round_trip(dr.y, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                    sum_phi += Io<S>::round_trip_phi(phin.y, P.scale[F_PHI], P.inv_scale[F_PHI]);
                }
                if (P.avg) {  // time sums of the new phi and u_z (FP64)
                    if (storeA) {
                        double* a = P.avg + zo + oA;
                        a[0] += (double)phin.x;
                        a[fs] += (double)uz.x;
                    }
                    if (storeB) {
                        double* a = P.avg + zo + oB;
                        a[0] += (double)phin.y;
                        a[fs] += (double)uz.y;
                    }
                }
            }
        }

        float2 nYZ[6];
        float nPA[6], nMB[6];
        float2 n_hx, n_vzp, n_vzm;
        float n_dyA, n_dyB;
        // (d) plane i: stencils, collision, x sweep, y populations -> yx[i], S
        {
            float sgz_unused;
            int inl = 0;
            resolve_axis(i, nz, P.face[4], P.face[5], sgz_unused, inl);

            // rho - 1 and j of the pair (footprint rows 2w+1, 2w+2), u = j / rho
            const float* jpl = jr + ((i + 8) & 3) * 4 * NPH;
            const int ec = (lane + 1) + PHX * (2 * w + 1);
            const float2 drho = make_float2(jpl[ec], jpl[ec + PHX]);
            const float2 rho = bc(1.f) + drho;
            const float2 irho = rcp2(rho);
            const float2 ux = make_float2(jpl[NPH + ec], jpl[NPH + ec + PHX]) * irho;
            const float2 uy = make_float2(jpl[2 * NPH + ec], jpl[2 * NPH + ec + PHX]) * irho;
            const float2 uz = make_float2(jpl[3 * NPH + ec], jpl[3 * NPH + ec + PHX]) * irho;

            // strain rate: dA_b = 72 d_a j_b from the z combinations of plane i.
            // Each lane forms the y combinations S'_y S'_z j_b, D_y S'_z j_b and
            // S'_y D_z j_b of its own footprint column (lane 31: column 0) and
            // takes those of the columns x -+ 1 from its neighbour lanes:
            //   dX_b = (S'S')(x+1) - (S'S')(x-1),
            //   dY_b = (DS')(x-1) + 4 (DS')(x) + (DS')(x+1), dZ_b likewise with S'D.
            const float4* z4 = jz4 + ((i + 8) & 1) * NPH;
            const float2* z2 = jz2 + ((i + 8) & 1) * NPH;
            float2 SS[3], DS[3], SD[3];
            {
                const int col = own_column(lane);
                float4 a[4];
                float2 b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int e = col + PHX * (2 * w + r);
                    a[r] = z4[e];
                    b[r] = z2[e];
                }
                // S'_z j_b in a[].x/y/z; D_z j_b in a[].w, b[].x, b[].y
                const float sv[3][4] = {{a[0].x, a[1].x, a[2].x, a[3].x},
                                        {a[0].y, a[1].y, a[2].y, a[3].y},
                                        {a[0].z, a[1].z, a[2].z, a[3].z}};
                const float dv[3][4] = {{a[0].w, a[1].w, a[2].w, a[3].w},
                                        {b[0].x, b[1].x, b[2].x, b[3].x},
                                        {b[0].y, b[1].y, b[2].y, b[3].y}};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float2 sm = make_float2(sv[k][0], sv[k][1]), s0 = make_float2(sv[k][1], sv[k][2]),
                                 sp = make_float2(sv[k][2], sv[k][3]);
                    const float2 dm = make_float2(dv[k][0], dv[k][1]), d0 = make_float2(dv[k][1], dv[k][2]),
                                 dp = make_float2(dv[k][2], dv[k][3]);
                    SS[k] = s0v(sm, s0, sp);
                    DS[k] = sp - sm;
                    SD[k] = s0v(dm, d0, dp);
                }
            }
            const int left = (lane + 31) & 31;
            auto from_left = [&](float2 v) {
                return make_float2(__shfl_sync(FULL, v.x, left), __shfl_sync(FULL, v.y, left));
            };
            float2 dX[3], dY[3], dZ[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dX[k] = shfl_down2(SS[k]) - from_left(SS[k]);
                dY[k] = s0v(from_left(DS[k]), DS[k], shfl_down2(DS[k]));
                dZ[k] = s0v(from_left(SD[k]), SD[k], shfl_down2(SD[k]));
            }
            const float2 c1 = bc(cce), c2 = bc(2.f * cce);
            const float2 nxx = c2 * dX[0], nyy = c2 * dY[1], nzz = c2 * dZ[2];
            const float2 nxy = c1 * (dX[1] + dY[0]), nxz = c1 * (dX[2] + dZ[0]), nyz = c1 * (dY[2] + dZ[1]);

            // interface terms from the z combinations of phi at plane i
            float2 phi, Fx, Fy, Fz, nxv, nyv, nzv;
            interface2<NPH>(zc + ((i + 8) & 1) * 3 * NPH, lane, w, sig_half, P.normal_eps2, phi, Fx, Fy, Fz,
                            nxv, nyv, nzv);
            if (inl) {
                Fx = Fy = Fz = bc(0.f);
                nxv = nyv = nzv = bc(0.f);
            }

            // collision (Guo forcing: v = u + F / (2 rho)) and x sweep
            const float2 hf = 0.5f * irho;
            const float2 vx = mad(hf, Fx, ux), vy = mad(hf, Fy, uy), vz = mad(hf, Fz, uz);
            float2 X[3][8];
            collide_xsweep2(rho, drho, ux, uy, uz, vx, vy, vz, Fx, Fy, Fz, nxx, nyy, nzz, nxy, nxz, nyz, vx * Fx,
                            vy * Fy, vz * Fz, mad(vx, Fy, Fx * vy), mad(vx, Fz, Fx * vz), mad(vy, Fz, Fy * vz), om1,
                            fo, X);

            // y populations of the x moments 0 and 1; the row pair exchanges
            // inside the thread, the pair edges go through shared memory
            const float2 zero = bc(0.f);
            float* yb = yx + ((i + 8) & 1) * 14 * NT + tid;
#pragma unroll
            for (int qx = 0; qx < 2; ++qx)
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
            yb[12 * NT] = yp.y;
            yb[13 * NT] = ym.x;
            n_dyA = ym.y;  // row 2w+1 -> row 2w
            n_dyB = yp.x;  // row 2w -> row 2w+1
            n_vzp = phi + b1z;
            n_vzm = phi - b1z;
        }
        if constexpr (ST) {
            fence_proxy_async();  // the staging box is read by a TMA store after the barrier
            // the store issued this iteration has read its box before that box
            // takes the next iteration's plane
            if (tid == 0) bulk_wait_read<0>();
        }
        __syncthreads();
        commit(i + 3);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            sYZ[k] = nYZ[k];
            sPA[k] = nPA[k];
            sMB[k] = nMB[k];
        }
        s_hx = n_hx;
        s_vzp = n_vzp;
        s_vzm = n_vzm;
        s_dyA = n_dyA;
        s_dyB = n_dyB;
    }
    cp_async_wait<0>();
    if (ST && tid == 0) {  // the last plane waits in its staging box
        if (z1 - 1 >= z0) {
            tma_store_4d(&maps->out, outb + ((z1 - 1 + 8) & 1) * L::OUT_BOX, x0, y0, z1 - 1, 0);
            bulk_commit();
        }
        bulk_wait<0>();
    }

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
}

template <int NW, typename S, bool ST>
__global__ void __launch_bounds__(32 * NW, 1)
    step_ce_kernel(const __grid_constant__ StepParams P, const __grid_constant__ TileMaps M, const S* __restrict__ in,
                   S* __restrict__ out, const long long* __restrict__ t_in, long long* __restrict__ t_out,
                   double* __restrict__ partials) {
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const long long t = *t_in;
    step_tile_ce<NW, S, ST>(P, &M, in, out, t, blockIdx.x, blockIdx.y, blockIdx.z, partials + 2 * blk);
    if (blk == 0 && threadIdx.x == 0 && threadIdx.y == 0) *t_out = t + 1;
}

template <int NW, typename S, bool ST>
cudaError_t launch_ce_nw(const StepParams& p, const TileMaps& m, const void* in, void* out, const long long* t_in,
                         long long* t_out, double* partials, cudaStream_t s) {
    const LaunchShape sh = step_shape(p, ST_FP32);
    step_ce_kernel<NW, S, ST><<<sh.grid, sh.block, ST ? StepCeSmem<NW>::BYTES_ST : StepCeSmem<NW>::BYTES, s>>>(
        p, m, static_cast<const S*>(in), static_cast<S*>(out), t_in, t_out, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_ce_t(const StepParams& p, const TileMaps* maps, const void* in, void* out, const long long* t_in,
                        long long* t_out, double* partials, cudaStream_t s) {
    TileMaps none;
    memset(&none, 0, sizeof(none));
    const TileMaps& m = maps ? *maps : none;
    // staged TMA stores: FP32, an output map made for this block size, not asked off
    const bool st = sizeof(S) == 4 && m.store && m.block_warps == p.block_warps && !p.plain_stores;
    switch (p.block_warps) {
        case 8: return st ? launch_ce_nw<8, S, true>(p, m, in, out, t_in, t_out, partials, s)
                          : launch_ce_nw<8, S, false>(p, m, in, out, t_in, t_out, partials, s);
        case 12: return st ? launch_ce_nw<12, S, true>(p, m, in, out, t_in, t_out, partials, s)
                           : launch_ce_nw<12, S, false>(p, m, in, out, t_in, t_out, partials, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int NW, typename S, bool ST>
cudaError_t prepare_ce_nw() {
    return cudaFuncSetAttribute(step_ce_kernel<NW, S, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(ST ? StepCeSmem<NW>::BYTES_ST : StepCeSmem<NW>::BYTES));
}

template <typename S>
cudaError_t prepare_ce_t() {
    cudaError_t e = prepare_ce_nw<8, S, false>();
    if (e == cudaSuccess) e = prepare_ce_nw<12, S, false>();
    if (e == cudaSuccess) e = prepare_ce_nw<8, S, true>();
    if (e == cudaSuccess) e = prepare_ce_nw<12, S, true>();
    return e;
}

}  // namespace

cudaError_t prepare_kernels_ce(int storage) {
    switch (storage) {
        case ST_FP32: return prepare_ce_t<float>();
        case ST_FP16: return prepare_ce_t<__half>();
        case ST_BF16: return prepare_ce_t<__nv_bfloat16>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_ce(const StepParams& p, int storage, const void* in, void* out, const long long* t_in,
                           long long* t_out, double* partials, cudaStream_t s, const TileMaps* maps) {
    switch (storage) {
        case ST_FP32: return launch_ce_t<float>(p, maps, in, out, t_in, t_out, partials, s);
        case ST_FP16: return launch_ce_t<__half>(p, maps, in, out, t_in, t_out, partials, s);
        case ST_BF16: return launch_ce_t<__nv_bfloat16>(p, maps, in, out, t_in, t_out, partials, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tslb
