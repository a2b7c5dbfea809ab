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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TX = 30;        // interior columns of a tile; a warp stages TX + 2
constexpr int PHX = TX + 4;   // phase-field columns of a tile (halo 2)
constexpr int NW_STEP = 16;   // warps (staged rows) per block of the step kernel

// ------------------------------------------------------------------ helpers

// Source coordinate of grid coordinate g on an axis of n nodes whose lower /
// upper faces follow rule lo / hi.  sign = -1 for a mirror image, inlet = 1
// for the inlet ghost.  Coordinates farther out than any stencil reaches are
// clamped into the grid (their values are never used).
__device__ __forceinline__ int resolve_axis(int g, int n, int lo, int hi, float& sign, int& inlet) {
    sign = 1.f;
    if (g >= 0 && g < n) return g;
    const int kind = g < 0 ? lo : hi;
    int s;
    if (kind == BC_PERIODIC) {
        s = g % n;
        if (s < 0) s += n;
    } else if (kind == BC_FREE_SLIP) {
        sign = -1.f;
        s = g < 0 ? -1 - g : 2 * n - 1 - g;
    } else {
        if (kind == BC_INLET) inlet = 1;
        s = g < 0 ? 0 : n - 1;
    }
    return min(max(s, 0), n - 1);
}

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Imposed phase field of the inlet at lateral node (x, y): smoothed top hat.
__device__ __forceinline__ float inlet_phi(const StepParams& P, int x, int y) {
    const float dx = (float)x - P.inlet_cx, dy = (float)y - P.inlet_cy;
    const float r = sqrtf(dx * dx + dy * dy);
    return -tanhf((r - P.inlet_half_d) * P.inlet_two_over_w);
}

// Imposed inlet velocity at (x, y) and step t: s (U + xi), s = (1 + phi_B)/2,
// xi_c = a |U| (2 r_c - 1), r_c from Philox on counter (x + nx y, t_lo, t_hi, 0).
__device__ void inlet_velocity(const StepParams& P, int x, int y, long long t, float u[3]) {
    const float s = 0.5f * (1.f + inlet_phi(P, x, y));
    uint32_t c[4] = {(uint32_t)(x + P.nx * y), (uint32_t)((unsigned long long)t & 0xffffffffu),
                     (uint32_t)((unsigned long long)t >> 32), 0u};
    philox4x32_10(c, P.seed_lo, P.seed_hi);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float rc = (float)(c[k] >> 8) * (1.f / 16777216.f);
        const float xi = P.noise_amp * P.inlet_umag * (2.f * rc - 1.f);
        u[k] = s * (P.inlet_u[k] + xi);
    }
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stored <-> FP32 conversion of one field value.
template <typename S>
struct Io;
template <>
struct Io<float> {
    static constexpr bool kAsync = true;
    static __device__ __forceinline__ float ld(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v, float) { *p = v; }
    static __device__ __forceinline__ float round_trip(float v, float, float) { return v; }
};
template <>
struct Io<__half> {
    static constexpr bool kAsync = false;
    static __device__ __forceinline__ float ld(const __half* p, float inv) { return __half2float(__ldg(p)) * inv; }
    static __device__ __forceinline__ void st(__half* p, float v, float s) { *p = __float2half_rn(v * s); }
    static __device__ __forceinline__ float round_trip(float v, float s, float inv) {
        return __half2float(__float2half_rn(v * s)) * inv;
    }
};
template <>
struct Io<__nv_bfloat16> {
    static constexpr bool kAsync = false;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, float inv) {
        return __bfloat162float(__ldg(p)) * inv;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v, float s) { *p = __float2bfloat16_rn(v * s); }
    static __device__ __forceinline__ float round_trip(float v, float s, float inv) {
        return __bfloat162float(__float2bfloat16_rn(v * s)) * inv;
    }
};

// One axis of the streaming sweep.  (k0, k1, k2) are the Hermite coefficients
// of the axis (k2 pre-multiplied by h2(+-1) = 2/3); the unnormalised 1D
// populations (x 6) are
//   p(-1) = k0 - k1 + k2,   p(0) = 4 k0 - 2 k2,   p(+1) = k0 + k1 + k2.
struct Tri {
    float m, z, p;
};
__device__ __forceinline__ Tri pops3(float k0, float k1, float k2) {
    return {k0 - k1 + k2, 4.f * k0 - 2.f * k2, k0 + k1 + k2};
}

// x sweep: shift p(+1) one lane up and p(-1) one lane down, then the x raw
// moments (x 6) M0 = q- + q0 + q+, M1 = q+ - q-, M2 = q+ + q-.
__device__ __forceinline__ void xsweep(float k0, float k1, float k2, float& m0, float& m1, float& m2) {
    const Tri t = pops3(k0, k1, k2);
    const float qp = __shfl_up_sync(FULL, t.p, 1);
    const float qm = __shfl_down_sync(FULL, t.m, 1);
    m0 = qm + t.z + qp;
    m1 = qp - qm;
    m2 = qp + qm;
}

__device__ __forceinline__ float s0(const float* v) { return v[0] + 4.f * v[1] + v[2]; }
__device__ __forceinline__ float d1(const float* v) { return v[2] - v[0]; }
__device__ __forceinline__ float l2(const float* v) { return v[0] + v[2] - 2.f * v[1]; }

// ---------------------------------------------------------------- step kernel

template <int NW>
struct StepSmem {
    static constexpr int NT = 32 * NW;
    static constexpr int NPH = PHX * (NW + 2);
    static constexpr int RING = 0;                 // [4][NPH] phase-field planes
    static constexpr int ZC = RING + 4 * NPH;      // [2][3][NPH] z combinations of phi
    static constexpr int MOM = ZC + 6 * NPH;       // [2][10][NT] staged moments
    static constexpr int YX = MOM + 20 * NT;       // [2][20][NT] y exchange
    static constexpr int FLOATS = YX + 40 * NT;
    static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

template <int NW, typename S>
__global__ void __launch_bounds__(32 * NW, 1)
    step_kernel(const __grid_constant__ StepParams P, const S* __restrict__ in, S* __restrict__ out,
                const long long* __restrict__ t_in, long long* __restrict__ t_out,
                double* __restrict__ partials) {
    using L = StepSmem<NW>;
    constexpr int NT = L::NT;
    constexpr int NPH = L::NPH;
    constexpr int TY = NW - 2;
    constexpr int EPT = (NPH + NT - 1) / NT;
    extern __shared__ __align__(16) float smem[];
    float* const ring = smem + L::RING;
    float* const zc = smem + L::ZC;
    float* const mom = smem + L::MOM;
    float* const yx = smem + L::YX;

    const int lane = threadIdx.x, warp = threadIdx.y, tid = lane + 32 * warp;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const long long fs = P.fstride;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * P.tile_z;
    const int z1 = min(z0 + P.tile_z, nz);
    const long long t = *t_in;

    // staged node of this thread (constant along the march)
    int unused = 0;
    float sgx, sgy;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + warp;
    const int sx = resolve_axis(gx, nx, P.face[0], P.face[1], sgx, unused);
    const int sy = resolve_axis(gy, ny, P.face[2], P.face[3], sgy, unused);
    const long long sxy = sx + (long long)nx * sy;
    const bool row_interior = warp >= 1 && warp <= NW - 2;
    const bool store_ok = row_interior && lane >= 1 && lane <= TX && gx < nx && gy < ny;

    // phase-field elements loaded by this thread (columns x0-2.., rows y0-2..)
    long long pxy[EPT];
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
            pxy[e] = psx + (long long)nx * psy;
            if (inlet_planes) phib[e] = inlet_phi(P, psx, psy);
        }
    }

    auto load_phi_plane = [&](int q) {
        float sg;
        int inl = 0;
        const int sz = resolve_axis(q, nz, P.face[4], P.face[5], sg, inl);
        float* dst = ring + ((q + 8) & 3) * NPH;
        const S* src = in + F_PHI * fs + nxy * sz;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int idx = tid + e * NT;
            if (idx < NPH) {
                if (inl) {
                    dst[idx] = phib[e];
                } else if constexpr (Io<S>::kAsync) {
                    cp_async4(dst + idx, reinterpret_cast<const float*>(src + pxy[e]));
                } else {
                    dst[idx] = Io<S>::ld(src + pxy[e], P.inv_scale[F_PHI]);
                }
            }
        }
    };
    auto load_mom_plane = [&](int q, float& sgz, int& inl) {
        inl = 0;
        const int sz = resolve_axis(q, nz, P.face[4], P.face[5], sgz, inl);
        float* dst = mom + ((q + 8) & 1) * 10 * NT + tid;
        const S* src = in + sxy + nxy * sz;
#pragma unroll
        for (int f = 0; f < 10; ++f) {
            if constexpr (Io<S>::kAsync)
                cp_async4(dst + f * NT, reinterpret_cast<const float*>(src + f * fs));
            else
                dst[f * NT] = Io<S>::ld(src + f * fs, P.inv_scale[f]);
        }
    };

    float sgz_cur, sgz_nxt;
    int inl_cur, inl_nxt;
    load_phi_plane(z0 - 2);
    load_phi_plane(z0 - 1);
    load_phi_plane(z0);
    load_mom_plane(z0 - 1, sgz_cur, inl_cur);
    cp_async_commit();

    // z-march carries: for each (qx, qy) group the z populations p(+1) of the
    // two previous planes and p(0) of the previous plane; same for D3Q7.
    float cPP[6], cP[6], cZ[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) cPP[k] = cP[k] = cZ[k] = 0.f;
    float cH = 0.f, cVPP = 0.f, cVP = 0.f;
    float sum_rho = 0.f, sum_phi = 0.f;

    const float om1 = 1.f - P.omega, fo = 1.f - 0.5f * P.omega;
    int buf = 0;
    for (int p = z0 - 1; p <= z1; ++p) {
        load_phi_plane(p + 2);
        load_mom_plane(p + 1, sgz_nxt, inl_nxt);
        cp_async_commit();
        cp_async_wait<1>();

        // (1) z combinations of phi at plane p for the elements of this thread:
        //     phi, phi(z+1) + phi(z-1), phi(z+1) - phi(z-1)
        {
            const float* pm = ring + ((p - 1 + 8) & 3) * NPH;
            const float* pc = ring + ((p + 8) & 3) * NPH;
            const float* pp = ring + ((p + 1 + 8) & 3) * NPH;
            float* z = zc + buf * 3 * NPH;
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
        __syncthreads();

        // (2)-(4a) staged node: interface geometry, post-collision Hermite
        //          coefficients, x sweep, y populations.
        float YZ[9];
        float hx, vzp, vzm;
        {
            const float* m = mom + ((p + 8) & 1) * 10 * NT + tid;
            const float drho = m[0];
            float ux = m[NT] * sgx, uy = m[2 * NT] * sgy, uz = m[3 * NT] * sgz_cur;
            const float pxx = m[4 * NT], pyy = m[5 * NT], pzz = m[6 * NT];
            const float pxy = m[7 * NT] * (sgx * sgy), pxz = m[8 * NT] * (sgx * sgz_cur),
                        pyz = m[9 * NT] * (sgy * sgz_cur);
            if (inl_cur) {
                float ub[3];
                inlet_velocity(P, sx, sy, t, ub);
                ux = ub[0] * sgx;
                uy = ub[1] * sgy;
                uz = ub[2];
            }

            // isotropic stencils of grad phi and its Hessian, separably:
            // z combos from shared memory, then y, then x (all x 216 / weights)
            const float* zb = zc + buf * 3 * NPH;
            const int e0 = (lane + 1) + PHX * (warp + 1);
            float yS[3], yDS[3], yLS[3], ySD[3], yDD[3], ySL[3];
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                float zS[3], zD[3], zL[3];
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const int e = e0 + dx + PHX * dy;
                    const float c0 = zb[e], c1 = zb[NPH + e], c2 = zb[2 * NPH + e];
                    zS[dy + 1] = c1 + 4.f * c0;
                    zD[dy + 1] = c2;
                    zL[dy + 1] = c1 - 2.f * c0;
                }
                yS[dx + 1] = s0(zS);
                yDS[dx + 1] = d1(zS);
                yLS[dx + 1] = l2(zS);
                ySD[dx + 1] = s0(zD);
                yDD[dx + 1] = d1(zD);
                ySL[dx + 1] = s0(zL);
            }
            const float phi = zb[e0];
            const float gxp = d1(yS) * (1.f / 72.f), gyp = s0(yDS) * (1.f / 72.f),
                        gzp = s0(ySD) * (1.f / 72.f);
            const float hxx = l2(yS) * (1.f / 36.f), hyy = s0(yLS) * (1.f / 36.f),
                        hzz = s0(ySL) * (1.f / 36.f);
            const float hxy = d1(yDS) * (1.f / 24.f), hxz = d1(ySD) * (1.f / 24.f),
                        hyz = s0(yDD) * (1.f / 24.f);

            // regularised normal, its divergence and the CSF force
            const float m2 = gxp * gxp + gyp * gyp + gzp * gzp + P.normal_eps2;
            const float im = m2 > 0.f ? rsqrtf(m2) : 0.f;
            float nxv = gxp * im, nyv = gyp * im, nzv = gzp * im;
            const float ghg = gxp * (gxp * hxx + 2.f * (gyp * hxy + gzp * hxz)) +
                              gyp * (gyp * hyy + 2.f * gzp * hyz) + gzp * gzp * hzz;
            const float kappa = (hxx + hyy + hzz) * im - ghg * (im * im * im);
            const float fk = -0.5f * P.sigma * kappa;
            float Fx = fk * gxp, Fy = fk * gyp, Fz = fk * gzp;
            if (inl_cur) {
                Fx = Fy = Fz = 0.f;
                nxv = nyv = nzv = 0.f;
            }

            // collision in Hermite form (Guo forcing: v = u + F / (2 rho))
            const float rho = 1.f + drho, irho = 1.f / rho;
            const float hfx = 0.5f * Fx * irho, hfy = 0.5f * Fy * irho, hfz = 0.5f * Fz * irho;
            const float vx = ux + hfx, vy = uy + hfy, vz = uz + hfz;
            // Pi^neq relative to v: P + rho (u u - v v) = P - rho (u h + h v)
            const float nxx = pxx - rho * (ux * hfx + hfx * vx);
            const float nyy = pyy - rho * (uy * hfy + hfy * vy);
            const float nzz = pzz - rho * (uz * hfz + hfz * vz);
            const float nxy = pxy - rho * (ux * hfy + hfx * vy);
            const float nxz = pxz - rho * (ux * hfz + hfx * vz);
            const float nyz = pyz - rho * (uy * hfz + hfy * vz);
            const float rvx = rho * vx, rvy = rho * vy, rvz = rho * vz;
            // A2 = rho v v + (1-omega) Pi^neq + (1-omega/2)(v F + F v)
            // M  = rho v v / 3 + (1-omega) Pi^neq  (A3 = v M + M v + ... )
            const float exx = rvx * vx, eyy = rvy * vy, ezz = rvz * vz;
            const float exy = rvx * vy, exz = rvx * vz, eyz = rvy * vz;
            const float Mxx = exx * (1.f / 3.f) + om1 * nxx, Myy = eyy * (1.f / 3.f) + om1 * nyy,
                        Mzz = ezz * (1.f / 3.f) + om1 * nzz, Mxy = exy * (1.f / 3.f) + om1 * nxy,
                        Mxz = exz * (1.f / 3.f) + om1 * nxz, Myz = eyz * (1.f / 3.f) + om1 * nyz;
            const float A2xx = exx + om1 * nxx + fo * (2.f * vx * Fx);
            const float A2yy = eyy + om1 * nyy + fo * (2.f * vy * Fy);
            const float A2zz = ezz + om1 * nzz + fo * (2.f * vz * Fz);
            const float A2xy = exy + om1 * nxy + fo * (vx * Fy + Fx * vy);
            const float A2xz = exz + om1 * nxz + fo * (vx * Fz + Fx * vz);
            const float A2yz = eyz + om1 * nyz + fo * (vy * Fz + Fy * vz);

            // Hermite coefficients of the tensor-product basis h_a(cx) h_b(cy) h_c(cz),
            // index 2 pre-multiplied by 2/3:  k_abc
            const float k000 = drho;
            const float k100 = 3.f * (rho * ux + Fx), k010 = 3.f * (rho * uy + Fy),
                        k001 = 3.f * (rho * uz + Fz);
            const float k200 = 3.f * A2xx, k020 = 3.f * A2yy, k002 = 3.f * A2zz;
            const float k110 = 9.f * A2xy, k101 = 9.f * A2xz, k011 = 9.f * A2yz;
            const float k210 = 9.f * (2.f * vx * Mxy + vy * Mxx);
            const float k201 = 9.f * (2.f * vx * Mxz + vz * Mxx);
            const float k120 = 9.f * (2.f * vy * Mxy + vx * Myy);
            const float k021 = 9.f * (2.f * vy * Myz + vz * Myy);
            const float k102 = 9.f * (2.f * vz * Mxz + vx * Mzz);
            const float k012 = 9.f * (2.f * vz * Myz + vy * Mzz);
            const float k111 = 27.f * (vx * Myz + vy * Mxz + vz * Mxy);

            // x sweep: X[qx][g], g = b + 3 c over the (b, c) pairs present
            float X[3][8];
            xsweep(k000, k100, k200, X[0][0], X[1][0], X[2][0]);
            xsweep(k010, k110, k210, X[0][1], X[1][1], X[2][1]);
            xsweep(k020, k120, 0.f, X[0][2], X[1][2], X[2][2]);
            xsweep(k001, k101, k201, X[0][3], X[1][3], X[2][3]);
            xsweep(k011, k111, 0.f, X[0][4], X[1][4], X[2][4]);
            xsweep(k021, 0.f, 0.f, X[0][5], X[1][5], X[2][5]);
            xsweep(k002, k102, 0.f, X[0][6], X[1][6], X[2][6]);
            xsweep(k012, 0.f, 0.f, X[0][7], X[1][7], X[2][7]);

            // y populations of each (qx, c) group; p(+1) and p(-1) go to the
            // rows below and above through shared memory
            float* yb = yx + buf * 20 * NT + tid;
#pragma unroll
            for (int qx = 0; qx < 3; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float b0 = X[qx][3 * c], b1 = X[qx][3 * c + 1];
                    const float b2 = c < 2 ? X[qx][3 * c + 2] : 0.f;
                    const Tri tr = pops3(b0, b1, b2);
                    const int k = 3 * qx + c;
                    yb[(2 * k) * NT] = tr.p;
                    yb[(2 * k + 1) * NT] = tr.m;
                    YZ[k] = tr.z;
                }

            // D3Q7: g_i^post = w_i (B0 + c_i . B1)
            const float ga = P.gamma * (1.f - phi * phi);
            const float b1x = 4.f * phi * vx + ga * nxv;
            const float b1y = 4.f * phi * vy + ga * nyv;
            const float b1z = 4.f * phi * vz + ga * nzv;
            const float fromL = __shfl_up_sync(FULL, phi + b1x, 1);
            const float fromR = __shfl_down_sync(FULL, phi - b1x, 1);
            hx = 0.25f * phi + 0.125f * (fromL + fromR);
            yb[18 * NT] = phi + b1y;
            yb[19 * NT] = phi - b1y;
            vzp = phi + b1z;
            vzm = phi - b1z;
        }
        __syncthreads();

        // (4b)-(5) interior rows: y shift and moments, z shift and moments,
        //          output of plane p - 1.
        if (row_interior) {
            const float* ya = yx + buf * 20 * NT + tid - 32;  // row y - 1
            const float* yc = yx + buf * 20 * NT + tid + 32;  // row y + 1
            float Y[3][3][3];
#pragma unroll
            for (int qx = 0; qx < 3; ++qx)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = 3 * qx + c;
                    const float qp = ya[(2 * k) * NT], qm = yc[(2 * k + 1) * NT];
                    Y[qx][0][c] = qm + YZ[k] + qp;
                    Y[qx][1][c] = qp - qm;
                    Y[qx][2][c] = qp + qm;
                }
            const float hxy = hx + 0.125f * (ya[18 * NT] + yc[19 * NT]);

            // z populations of the (qx, qy) groups 00, 10, 01, 20, 02, 11
            const int gqx[6] = {0, 1, 0, 2, 0, 1}, gqy[6] = {0, 0, 1, 0, 2, 1};
            float O0[6], O1[6], O2[6];
#pragma unroll
            for (int g = 0; g < 6; ++g) {
                const Tri tr = pops3(Y[gqx[g]][gqy[g]][0], Y[gqx[g]][gqy[g]][1], Y[gqx[g]][gqy[g]][2]);
                O0[g] = cPP[g] + cZ[g] + tr.m;
                O1[g] = cPP[g] - tr.m;
                O2[g] = cPP[g] + tr.m;
                cPP[g] = cP[g];
                cP[g] = tr.p;
                cZ[g] = tr.z;
            }
            const float phin = cH + 0.125f * (cVPP + vzm);
            cH = hxy;
            cVPP = cVP;
            cVP = vzp;

            if (p >= z0 + 1 && store_ok) {
                const float s = 1.f / 216.f;
                const float dr = O0[0] * s, jx = O0[1] * s, jy = O0[2] * s, jz = O1[0] * s;
                const float dxx = O0[3] * s, dyy = O0[4] * s, dzz = O2[0] * s;
                const float cxy = O0[5] * s, cxz = O1[1] * s, cyz = O1[2] * s;
                const float rn = 1.f + dr, irn = 1.f / rn;
                const float ux = jx * irn, uy = jy * irn, uz = jz * irn;
                const float val[NFIELDS] = {
                    dr, ux, uy, uz,
                    dxx - (1.f / 3.f) * dr - rn * ux * ux,
                    dyy - (1.f / 3.f) * dr - rn * uy * uy,
                    dzz - (1.f / 3.f) * dr - rn * uz * uz,
                    cxy - rn * ux * uy, cxz - rn * ux * uz, cyz - rn * uy * uz, phin};
                S* o = out + sxy + nxy * (p - 1);
#pragma unroll
                for (int f = 0; f < NFIELDS; ++f) Io<S>::st(o + f * fs, val[f], P.scale[f]);
                sum_rho += Io<S>::round_trip(dr, P.scale[F_DRHO], P.inv_scale[F_DRHO]);
                sum_phi += Io<S>::round_trip(phin, P.scale[F_PHI], P.inv_scale[F_PHI]);
            }
        }
        sgz_cur = sgz_nxt;
        inl_cur = inl_nxt;
        buf ^= 1;
    }
    cp_async_wait<0>();

    // block partials of sum(rho - 1) and sum(phi) in FP64
    double a = sum_rho, b = sum_phi;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(FULL, a, off);
        b += __shfl_xor_sync(FULL, b, off);
    }
    __syncthreads();
    double* red = reinterpret_cast<double*>(yx);
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < NW; ++w) {
            A += red[2 * w];
            B += red[2 * w + 1];
        }
        partials[2 * blk] = A;
        partials[2 * blk + 1] = B;
        if (blk == 0) *t_out = t + 1;
    }
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
    S* dst = st + field * P.fstride;
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
        sp += Io<S>::ld(st + F_PHI * fs + i, P.inv_scale[F_PHI]);
    }
    block_partials<S>(sr, sp, partials);
}

template <typename S>
__global__ void __launch_bounds__(CONV_THREADS) get_field_kernel(const __grid_constant__ StepParams P,
                                                                 const S* __restrict__ st, int field,
                                                                 float* __restrict__ dst) {
    const long long N = (long long)P.nx * P.ny * P.nz;
    const S* src = st + field * P.fstride;
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

template <typename S>
cudaError_t launch_step_t(const StepParams& p, const void* in, void* out, const long long* t_in,
                          long long* t_out, double* partials, cudaStream_t s) {
    constexpr int NW = NW_STEP;
    auto k = step_kernel<NW, S>;
    const LaunchShape sh = step_shape(p, ST_FP32);
    k<<<sh.grid, sh.block, sh.smem, s>>>(p, static_cast<const S*>(in), static_cast<S*>(out), t_in, t_out,
                                         partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t prepare_t() {
    return cudaFuncSetAttribute(step_kernel<NW_STEP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StepSmem<NW_STEP>::BYTES);
}

}  // namespace

cudaError_t prepare_kernels(int storage) {
    switch (storage) {
        case ST_FP32: return prepare_t<float>();
        case ST_FP16: return prepare_t<__half>();
        case ST_BF16: return prepare_t<__nv_bfloat16>();
        default: return cudaErrorInvalidValue;
    }
}

LaunchShape step_shape(const StepParams& p, int /*storage*/) {
    LaunchShape sh;
    sh.nw = NW_STEP;
    const int ty = NW_STEP - 2;
    sh.grid = dim3((p.nx + TX - 1) / TX, (p.ny + ty - 1) / ty, (p.nz + p.tile_z - 1) / p.tile_z);
    sh.block = dim3(32, NW_STEP, 1);
    sh.smem = StepSmem<NW_STEP>::BYTES;
    return sh;
}

int max_partials(const StepParams& p, int storage) {
    const LaunchShape sh = step_shape(p, storage);
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
