// The paper's own GPU design, kept as an ablation of the fused moment-only
// step: populations in HBM and two sweeps per time step (Sec. 2: the moment
// arrays plus one set of population arrays instead of two A-B sets).
//
//   collide_push: for every node of the grid and of its one-node ghost shell,
//     read the stored moments (ghosts by the face rules), the phase field of
//     its 27 neighbours, build the post-collision populations f_i (D3Q27,
//     third-order Hermite form with Guo forcing) and g_k (D3Q7) and write each
//     to the population arrays at x + c_i (Eq. pushLB), when that is in the grid;
//   moments: for every node, read the 27 + 7 populations and write the stored
//     moments rho - 1, u, P, phi and the block partial sums.
//
// Per lattice update: 11 + 34 values read and 34 + 11 written = 360 B in FP32,
// against 88 B for the fused kernel.  The moments stay the state, so I/O,
// sums and checkpoints are the same as for the fused path.  f is stored as the
// deviation f_i - w_i from rest (FP32 precision), g as is.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TS_THREADS = 256;

__device__ __forceinline__ int ts_resolve(int g, int n, int lo, int hi, float& sign, int& inlet) {
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

__device__ __forceinline__ void ts_philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
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

__device__ __forceinline__ float ts_inlet_phi(const StepParams& P, int x, int y) {
    const float dx = (float)x - P.inlet_cx, dy = (float)y - P.inlet_cy;
    return -tanhf((sqrtf(dx * dx + dy * dy) - P.inlet_half_d) * P.inlet_two_over_w);
}

// Stored moments of grid position (gx, gy, gz), ghosts resolved by the face
// rules; inlet ghosts carry the imposed u and phi.
struct Node {
    float drho, u[3], p[6], phi;
    int inlet;
};

__device__ void ts_fetch(const StepParams& P, const float* __restrict__ M, long long t, int gx, int gy, int gz,
                         Node& n) {
    float sx_, sy_, sz_;
    int in = 0;
    const int sx = ts_resolve(gx, P.nx, P.face[0], P.face[1], sx_, in);
    const int sy = ts_resolve(gy, P.ny, P.face[2], P.face[3], sy_, in);
    const int sz = ts_resolve(gz, P.nz, P.face[4], P.face[5], sz_, in);
    const long long i = sx + (long long)P.nx * (sy + (long long)P.ny * sz);
    const long long fs = P.fstride;
    n.drho = __ldg(M + F_DRHO * fs + i);
    for (int a = 0; a < 3; ++a) n.u[a] = __ldg(M + (F_UX + a) * fs + i);
    for (int k = 0; k < 6; ++k) n.p[k] = __ldg(M + (F_PXX + k) * fs + i);
    n.phi = __ldg(M + F_PHI * fs + i);
    n.inlet = in;
    if (in) {
        const float phib = ts_inlet_phi(P, sx, sy);
        const float s = 0.5f * (1.f + phib);
        uint32_t c[4] = {(uint32_t)(sx + P.nx * sy), (uint32_t)((unsigned long long)t & 0xffffffffu),
                         (uint32_t)((unsigned long long)t >> 32), 0u};
        ts_philox(c, P.seed_lo, P.seed_hi);
        for (int k = 0; k < 3; ++k) {
            const float rc = (float)(c[k] >> 8) * (1.f / 16777216.f);
            n.u[k] = s * (P.inlet_u[k] + P.noise_amp * P.inlet_umag * (2.f * rc - 1.f));
        }
        n.phi = phib;
    }
    // mirror images: odd components flip (xx yy zz xy xz yz)
    n.u[0] *= sx_;
    n.u[1] *= sy_;
    n.u[2] *= sz_;
    n.p[3] *= sx_ * sy_;
    n.p[4] *= sx_ * sz_;
    n.p[5] *= sy_ * sz_;
}

__device__ float ts_phi_at(const StepParams& P, const float* __restrict__ M, int gx, int gy, int gz) {
    float s;
    int in = 0;
    const int sx = ts_resolve(gx, P.nx, P.face[0], P.face[1], s, in);
    const int sy = ts_resolve(gy, P.ny, P.face[2], P.face[3], s, in);
    const int sz = ts_resolve(gz, P.nz, P.face[4], P.face[5], s, in);
    if (in) return ts_inlet_phi(P, sx, sy);
    return __ldg(M + F_PHI * P.fstride + sx + (long long)P.nx * (sy + (long long)P.ny * sz));
}

__device__ __forceinline__ float w1(int c) { return c == 0 ? (2.f / 3.f) : (1.f / 6.f); }

__global__ void __launch_bounds__(TS_THREADS) collide_push_kernel(const __grid_constant__ StepParams P,
                                                                  const float* __restrict__ M,
                                                                  float* __restrict__ pops,
                                                                  const long long* __restrict__ t_dev) {
    const int ex = P.nx + 2, ey = P.ny + 2, ez = P.nz + 2;
    const long long total = (long long)ex * ey * ez;
    const long long t = *t_dev;
    const long long fs = P.fstride;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const int gx = (int)(id % ex) - 1, gy = (int)((id / ex) % ey) - 1, gz = (int)(id / ((long long)ex * ey)) - 1;
        Node n;
        ts_fetch(P, M, t, gx, gy, gz, n);
        // interface geometry from the 27-point isotropic stencils
        float g[3] = {0.f, 0.f, 0.f}, h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float F[3] = {0.f, 0.f, 0.f}, nr[3] = {0.f, 0.f, 0.f};
        if (!n.inlet) {
            for (int cz = -1; cz <= 1; ++cz)
                for (int cy = -1; cy <= 1; ++cy)
                    for (int cx = -1; cx <= 1; ++cx) {
                        const float w = w1(cx) * w1(cy) * w1(cz);
                        const float ph = ts_phi_at(P, M, gx + cx, gy + cy, gz + cz);
                        const float wp = w * ph;
                        g[0] += 3.f * wp * cx;
                        g[1] += 3.f * wp * cy;
                        g[2] += 3.f * wp * cz;
                        h[0] += 9.f * wp * (cx * cx - (1.f / 3.f));
                        h[1] += 9.f * wp * (cy * cy - (1.f / 3.f));
                        h[2] += 9.f * wp * (cz * cz - (1.f / 3.f));
                        h[3] += 9.f * wp * (cx * cy);
                        h[4] += 9.f * wp * (cx * cz);
                        h[5] += 9.f * wp * (cy * cz);
                    }
            const float m2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + P.normal_eps2;
            const float im = m2 > 0.f ? rsqrtf(m2) : 0.f;
            for (int a = 0; a < 3; ++a) nr[a] = g[a] * im;
            const float ghg = g[0] * g[0] * h[0] + g[1] * g[1] * h[1] + g[2] * g[2] * h[2] +
                              2.f * (g[0] * g[1] * h[3] + g[0] * g[2] * h[4] + g[1] * g[2] * h[5]);
            const float kappa = (h[0] + h[1] + h[2]) * im - ghg * im * im * im;
            for (int a = 0; a < 3; ++a) F[a] = -0.5f * P.sigma * kappa * g[a];
        }
        // collision in Hermite form (Guo forcing)
        const float rho = 1.f + n.drho, hf = 0.5f / rho;
        float v[3];
        for (int a = 0; a < 3; ++a) v[a] = n.u[a] + hf * F[a];
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        float A2[6], Mt[6];
        const float om1 = 1.f - P.omega, fo = 1.f - 0.5f * P.omega;
        for (int k = 0; k < 6; ++k) {
            const int a = ia[k], b = ib[k];
            const float pn = n.p[k] - rho * (n.u[a] * hf * F[b] + hf * F[a] * v[b]);
            const float e = rho * v[a] * v[b];
            A2[k] = e + om1 * pn + fo * (v[a] * F[b] + F[a] * v[b]);
            Mt[k] = e * (1.f / 3.f) + om1 * pn;
        }
        // tensor-product coefficients C_abc of w_i sum C_abc h_a(cx) h_b(cy) h_c(cz)
        const float c100 = 3.f * (rho * n.u[0] + F[0]), c010 = 3.f * (rho * n.u[1] + F[1]),
                    c001 = 3.f * (rho * n.u[2] + F[2]);
        const float c200 = 4.5f * A2[0], c020 = 4.5f * A2[1], c002 = 4.5f * A2[2];
        const float c110 = 9.f * A2[3], c101 = 9.f * A2[4], c011 = 9.f * A2[5];
        const float c210 = 13.5f * (2.f * v[0] * Mt[3] + v[1] * Mt[0]);
        const float c201 = 13.5f * (2.f * v[0] * Mt[4] + v[2] * Mt[0]);
        const float c120 = 13.5f * (2.f * v[1] * Mt[3] + v[0] * Mt[1]);
        const float c021 = 13.5f * (2.f * v[1] * Mt[5] + v[2] * Mt[1]);
        const float c102 = 13.5f * (2.f * v[2] * Mt[4] + v[0] * Mt[2]);
        const float c012 = 13.5f * (2.f * v[2] * Mt[5] + v[1] * Mt[2]);
        const float c111 = 27.f * (v[0] * Mt[5] + v[1] * Mt[4] + v[2] * Mt[3]);
        // push f_i - w_i to x + c_i
        for (int cz = -1; cz <= 1; ++cz) {
            const int z = gz + cz;
            if (z < 0 || z >= P.nz) continue;
            for (int cy = -1; cy <= 1; ++cy) {
                const int y = gy + cy;
                if (y < 0 || y >= P.ny) continue;
                for (int cx = -1; cx <= 1; ++cx) {
                    const int x = gx + cx;
                    if (x < 0 || x >= P.nx) continue;
                    const float hx2 = cx * cx - (1.f / 3.f), hy2 = cy * cy - (1.f / 3.f), hz2 = cz * cz - (1.f / 3.f);
                    const float dev = n.drho + c100 * cx + c010 * cy + c001 * cz + c200 * hx2 + c020 * hy2 +
                                      c002 * hz2 + c110 * cx * cy + c101 * cx * cz + c011 * cy * cz +
                                      c210 * hx2 * cy + c201 * hx2 * cz + c120 * cx * hy2 + c021 * hy2 * cz +
                                      c102 * cx * hz2 + c012 * cy * hz2 + c111 * cx * cy * cz;
                    const int i = (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1);
                    pops[i * fs + x + (long long)P.nx * (y + (long long)P.ny * z)] = w1(cx) * w1(cy) * w1(cz) * dev;
                }
            }
        }
        // D3Q7: g_k = w_k (phi + c_k . (4 phi v + Gamma (1 - phi^2) n))
        const float ga = P.gamma * (1.f - n.phi * n.phi);
        float b1[3];
        for (int a = 0; a < 3; ++a) b1[a] = 4.f * n.phi * v[a] + ga * nr[a];
        const int dxs[7] = {0, 1, -1, 0, 0, 0, 0}, dys[7] = {0, 0, 0, 1, -1, 0, 0}, dzs[7] = {0, 0, 0, 0, 0, 1, -1};
        for (int k = 0; k < 7; ++k) {
            const int x = gx + dxs[k], y = gy + dys[k], z = gz + dzs[k];
            if (x < 0 || x >= P.nx || y < 0 || y >= P.ny || z < 0 || z >= P.nz) continue;
            const float wk = k == 0 ? 0.25f : 0.125f;
            pops[(27 + k) * fs + x + (long long)P.nx * (y + (long long)P.ny * z)] =
                wk * (n.phi + dxs[k] * b1[0] + dys[k] * b1[1] + dzs[k] * b1[2]);
        }
    }
}

__global__ void __launch_bounds__(TS_THREADS) moments_kernel(const __grid_constant__ StepParams P,
                                                             const float* __restrict__ pops, float* __restrict__ M,
                                                             const long long* __restrict__ t_in,
                                                             long long* __restrict__ t_out,
                                                             double* __restrict__ partials) {
    const long long N = (long long)P.nx * P.ny * P.nz, fs = P.fstride;
    float sr = 0.f, sp = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        float r = 0.f, j[3] = {0.f, 0.f, 0.f}, q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 27; ++k) {
            const int cx = k % 3 - 1, cy = (k / 3) % 3 - 1, cz = k / 9 - 1;
            const float f = __ldg(pops + k * fs + i);
            r += f;
            j[0] += cx * f;
            j[1] += cy * f;
            j[2] += cz * f;
            q[0] += cx * cx * f;
            q[1] += cy * cy * f;
            q[2] += cz * cz * f;
            q[3] += cx * cy * f;
            q[4] += cx * cz * f;
            q[5] += cy * cz * f;
        }
        float phi = 0.f;
#pragma unroll
        for (int k = 0; k < 7; ++k) phi += __ldg(pops + (27 + k) * fs + i);
        // deviations: rho - 1 = sum (f - w); Pi - cs2 I = sum c c (f - w)
        const float rn = 1.f + r, irn = 1.f / rn;
        const float u[3] = {j[0] * irn, j[1] * irn, j[2] * irn};
        M[F_DRHO * fs + i] = r;
        for (int a = 0; a < 3; ++a) M[(F_UX + a) * fs + i] = u[a];
        M[F_PXX * fs + i] = q[0] - (1.f / 3.f) * r - rn * u[0] * u[0];
        M[F_PYY * fs + i] = q[1] - (1.f / 3.f) * r - rn * u[1] * u[1];
        M[F_PZZ * fs + i] = q[2] - (1.f / 3.f) * r - rn * u[2] * u[2];
        M[F_PXY * fs + i] = q[3] - rn * u[0] * u[1];
        M[F_PXZ * fs + i] = q[4] - rn * u[0] * u[2];
        M[F_PYZ * fs + i] = q[5] - rn * u[1] * u[2];
        M[F_PHI * fs + i] = phi;
        sr += r;
        sp += phi;
    }
    __shared__ double ra[TS_THREADS / 32], rb[TS_THREADS / 32];
    double da = sr, db = sp;
    for (int off = 16; off > 0; off >>= 1) {
        da += __shfl_xor_sync(0xffffffffu, da, off);
        db += __shfl_xor_sync(0xffffffffu, db, off);
    }
    if ((threadIdx.x & 31) == 0) {
        ra[threadIdx.x >> 5] = da;
        rb[threadIdx.x >> 5] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < TS_THREADS / 32; ++w) {
            A += ra[w];
            B += rb[w];
        }
        partials[2 * blockIdx.x] = A;
        partials[2 * blockIdx.x + 1] = B;
        if (blockIdx.x == 0) *t_out = *t_in + 1;
    }
}

int ts_blocks(long long n) {
    long long b = (n + TS_THREADS - 1) / TS_THREADS;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

int twosweep_partials(const StepParams& p) { return ts_blocks((long long)p.nx * p.ny * p.nz); }

cudaError_t launch_twosweep_step(const StepParams& p, float* M, float* pops, const long long* t_in,
                                 long long* t_out, double* partials, cudaStream_t s) {
    const long long ext = (long long)(p.nx + 2) * (p.ny + 2) * (p.nz + 2);
    collide_push_kernel<<<ts_blocks(ext), TS_THREADS, 0, s>>>(p, M, pops, t_in);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_kernel<<<twosweep_partials(p), TS_THREADS, 0, s>>>(p, pops, M, t_in, t_out, partials);
    return cudaGetLastError();
}

}  // namespace tslb
