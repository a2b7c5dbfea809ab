/*
 * FP64 CPU oracle of the multicomponent thread-safe lattice Boltzmann step
 * (arXiv 2403.15773).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg are its only users.  It shares no code
 * with the CUDA library.
 *
 * What it computes, step by step, in the paper's order and notation:
 *
 *   (1) moments of the populations at every node (Sec. 2):
 *         rho = sum_i f_i, rho u = sum_i c_i f_i, Pi = sum_i c_i c_i f_i,
 *         phi = sum_i g_i;
 *   (2) interface geometry and the continuum-surface force (Sec. 2.2):
 *         grad phi, n = grad phi / |grad phi| (regularised), kappa = div n,
 *         F = -(sigma/2) kappa grad phi        (phi in [-1, 1]: jump of 2);
 *   (3) the fused stream-collide push (Eq. pushLB), with
 *         f_i^post = f_i^eq(rho, u) + (1 - omega) f_i^neq + (1 - omega/2) S_i,
 *       f^eq the third-order Hermite equilibrium (Eq. eqts), f^neq the Hermite
 *       reconstruction of Eq. neq_final up to third order with the recursive
 *       a3 of Eq. noneqts, S_i Guo's forcing term in second-order Hermite form;
 *       and the D3Q7 phase-field push (Eq. intcapturing, antidiff),
 *         g_i^post = w_i phi (1 + c_i.u / cs7^2) + w_i Gamma (1 - phi^2) c_i.n;
 *   (4) boundaries: every population that enters the domain from outside is
 *       the post-collision population of a ghost node whose moments follow the
 *       face rule (non-equilibrium extrapolation, Eq. original_neq, at the jet
 *       inlet; zero-gradient copy at outflow faces; specular mirror at
 *       free-slip walls; wrap at periodic faces).
 *
 * Readings where the paper is silent or garbled (each one is also listed in
 * the design notes of the repository):
 *   - D3Q27 weights 8/27, 2/27, 1/54, 1/216 and cs2 = 1/3 (Sec. 2, Fig. 2);
 *     D3Q7 weights 1/4 (rest) and 1/8, cs7^2 = 1/4.
 *   - Eq. noneqts drops w_i and the -cs2 delta of H2; read as
 *     f^neq = w_i [H2:a2/(2 cs^4) + H3:a3/(6 cs^6)], a3 = u a2 + a2 u + ... (3 terms).
 *   - a2_neq is the projected Pi - Pi^eq (the stored moment of Sec. 2).
 *   - Forcing: Guo's scheme; u = (rho u_raw + F/2)/rho in f^eq, first-order
 *     non-equilibrium a1 = j - rho u = -F/2 kept in f^neq.
 *   - n = grad phi / sqrt(|grad phi|^2 + eps^2) (eps a parameter, 1e-2 by
 *     default): the unit normal where phi varies, a smooth bounded field where
 *     the gradient vanishes in the bulk; kappa = div n exactly, with isotropic
 *     D3Q27 stencils for grad phi and its Hessian H.
 *   - phi in [-1, 1]; Lambda_i = w_i Gamma (1 - phi^2) c_i.n, Gamma = 1/W gives
 *     the steady profile tanh(2x/W).
 *   - Inlet ghost: rho and P from the adjacent fluid node, u and phi imposed
 *     (smoothed top hat, Philox4x32-10 noise), no interface force, n = 0.
 */
#include "tslb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 27
#define Q7 7

static const double CS2 = 1.0 / 3.0;  /* D3Q27 sound speed squared */
static const double CS2_7 = 0.25;     /* D3Q7: sum_i w_i c_ia c_ib = delta_ab / 4 */

static int C[Q][3];
static double W[Q];
static double H2[Q][3][3];
static double H3[Q][3][3][3];
static const int C7[Q7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                              {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double W7[Q7] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
static int tables_ready = 0;

/* D3Q27 velocities in the order i = (cx+1) + 3 (cy+1) + 9 (cz+1), with the
 * Hermite tensors H2 = c c - cs2 I and
 * H3_abg = c_a c_b c_g - cs2 (c_g d_ab + c_a d_bg + c_b d_ag) (Eq. eqts). */
static void tables(void) {
    if (tables_ready) return;
    for (int i = 0; i < Q; ++i) {
        C[i][0] = i % 3 - 1;
        C[i][1] = (i / 3) % 3 - 1;
        C[i][2] = i / 9 - 1;
        int n2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
        W[i] = n2 == 0 ? 8.0 / 27.0 : n2 == 1 ? 2.0 / 27.0 : n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    }
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                H2[i][a][b] = C[i][a] * C[i][b] - CS2 * (a == b);
                for (int g = 0; g < 3; ++g)
                    H3[i][a][b][g] = C[i][a] * C[i][b] * C[i][g] -
                                     CS2 * (C[i][g] * (a == b) + C[i][a] * (b == g) + C[i][b] * (a == g));
            }
    tables_ready = 1;
}

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications with the round keys bumped by the Weyl constants. */
void orc_philox4x32_10(const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4) {
    uint32_t x0 = ctr4[0], x1 = ctr4[1], x2 = ctr4[2], x3 = ctr4[3];
    uint32_t k0 = key2[0], k1 = key2[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out4[0] = x0;
    out4[1] = x1;
    out4[2] = x2;
    out4[3] = x3;
}

/* Imposed inlet state at lateral node (x, y) and step t: a smoothed top hat
 * phi_B = -tanh(2 (r - D/2) / W), u_B = s (U + xi) with s = (1 + phi_B)/2 and
 * xi_c = a |U| (2 r_c - 1), r_c = (philox_c >> 8) 2^-24 from
 * counter (x + nx y, t_lo, t_hi, 0) and key (seed_lo, seed_hi). */
void orc_inlet_state(const orc_params* p, int x, int y, int64_t t, double* u3, double* phi) {
    double dx = (double)x - p->inlet_cx, dy = (double)y - p->inlet_cy;
    double r = sqrt(dx * dx + dy * dy);
    double phib = -tanh(2.0 * (r - 0.5 * p->inlet_diameter) / p->inlet_width);
    double s = 0.5 * (1.0 + phib);
    uint32_t ctr[4] = {(uint32_t)(x + p->nx * y), (uint32_t)((uint64_t)t & 0xffffffffu),
                       (uint32_t)((uint64_t)t >> 32), 0u};
    uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    double umag = sqrt(p->inlet_u[0] * p->inlet_u[0] + p->inlet_u[1] * p->inlet_u[1] +
                       p->inlet_u[2] * p->inlet_u[2]);
    for (int c = 0; c < 3; ++c) {
        double rc = (double)(out[c] >> 8) * (1.0 / 16777216.0);
        double xi = p->noise_amp * umag * (2.0 * rc - 1.0);
        u3[c] = s * (p->inlet_u[c] + xi);
    }
    *phi = phib;
}

/* --------------------------------------------------------- node algebra */

typedef struct {
    double rho, u[3], P[3][3], phi;
    int inlet;
} node_t;

/* Third-order Hermite equilibrium (Eq. eqts). */
void orc_feq3(double rho, const double* u, double* f27) {
    tables();
    double uu[3][3], uuu[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            uu[a][b] = u[a] * u[b];
            for (int g = 0; g < 3; ++g) uuu[a][b][g] = u[a] * u[b] * u[g];
        }
    for (int i = 0; i < Q; ++i) {
        double cu = 0, h2 = 0, h3 = 0;
        for (int a = 0; a < 3; ++a) {
            cu += C[i][a] * u[a];
            for (int b = 0; b < 3; ++b) {
                h2 += H2[i][a][b] * uu[a][b];
                for (int g = 0; g < 3; ++g) h3 += H3[i][a][b][g] * uuu[a][b][g];
            }
        }
        f27[i] = rho * W[i] * (1.0 + cu / CS2 + h2 / (2.0 * CS2 * CS2) + h3 / (6.0 * CS2 * CS2 * CS2));
    }
}

/* Post-collision populations of one node:
 *   f^post = f^eq(rho, u) + (1 - omega) f^neq + (1 - omega/2) S,
 * u = u_raw + F/(2 rho) (Guo), Pi = rho cs2 I + rho u_raw u_raw + P,
 * a1 = rho u_raw - rho u, a2 = Pi - rho cs2 I - rho u u,
 * a3_abg = u_a a2_bg + u_b a2_ag + u_g a2_ab (Eq. noneqts),
 * f^neq_i = w_i [c.a1/cs2 + H2:a2/(2 cs^4) + H3:a3/(6 cs^6)] (Eq. neq_final),
 * S_i = w_i [c.F/cs2 + H2:(uF + Fu)/(2 cs^4)]. */
static void post_f(const node_t* nd, const double* F, double omega, const double (*a2_ce)[3], double* f) {
    const double rho = nd->rho;
    double u[3], a1[3], a2[3][3], a3[3][3][3], uf[3][3];
    for (int a = 0; a < 3; ++a) {
        u[a] = nd->u[a] + F[a] / (2.0 * rho);
        a1[a] = rho * nd->u[a] - rho * u[a];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double pi_ab = rho * CS2 * (a == b) + rho * nd->u[a] * nd->u[b] + nd->P[a][b];
            a2[a][b] = a2_ce ? a2_ce[a][b] : pi_ab - (rho * CS2 * (a == b) + rho * u[a] * u[b]);
            uf[a][b] = u[a] * F[b] + F[a] * u[b];
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int g = 0; g < 3; ++g)
                a3[a][b][g] = u[a] * a2[b][g] + u[b] * a2[a][g] + u[g] * a2[a][b];
    double feq[Q];
    orc_feq3(rho, u, feq);
    for (int i = 0; i < Q; ++i) {
        double c1 = 0, cF = 0, h2 = 0, h2f = 0, h3 = 0;
        for (int a = 0; a < 3; ++a) {
            c1 += C[i][a] * a1[a];
            cF += C[i][a] * F[a];
            for (int b = 0; b < 3; ++b) {
                h2 += H2[i][a][b] * a2[a][b];
                h2f += H2[i][a][b] * uf[a][b];
                for (int g = 0; g < 3; ++g) h3 += H3[i][a][b][g] * a3[a][b][g];
            }
        }
        double fneq = W[i] * (c1 / CS2 + h2 / (2.0 * CS2 * CS2) + h3 / (6.0 * CS2 * CS2 * CS2));
        double S = W[i] * (cF / CS2 + h2f / (2.0 * CS2 * CS2));
        f[i] = feq[i] + (1.0 - omega) * fneq + (1.0 - 0.5 * omega) * S;
    }
}

void orc_post_populations(double rho, const double* u_raw, const double* pi,
                          const double* force, double omega, double* f27) {
    tables();
    node_t nd;
    nd.rho = rho;
    for (int a = 0; a < 3; ++a) nd.u[a] = u_raw[a];
    nd.P[0][0] = pi[0];
    nd.P[1][1] = pi[1];
    nd.P[2][2] = pi[2];
    nd.P[0][1] = nd.P[1][0] = pi[3];
    nd.P[0][2] = nd.P[2][0] = pi[4];
    nd.P[1][2] = nd.P[2][1] = pi[5];
    nd.phi = 0;
    nd.inlet = 0;
    post_f(&nd, force, 1.0 * omega, NULL, f27);
}

/* Chapman-Enskog non-equilibrium second moment from the momentum of the 27
 * neighbours, j(x + c_i) (i in oracle order): grad j by the isotropic stencil
 * (1/cs2) sum_i w_i c_i j(x + c_i), a2 = -(cs2/omega)(d_a j_b + d_b j_a). */
void orc_ce_neq(const double* j27 /* 27 x 3 */, double omega, double* a2_6) {
    tables();
    double d[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  /* d[a][b] = d_a j_b */
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) d[a][b] += W[i] * C[i][a] * j27[3 * i + b] / CS2;
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) a2_6[k] = -(CS2 / omega) * (d[ia[k]][ib[k]] + d[ib[k]][ia[k]]);
}

/* D3Q7 post-collision populations, tau = 1 (Eq. intcapturing, antidiff). */
static void post_g(double phi, const double* u, const double* nrm, double gamma, double* g) {
    for (int k = 0; k < Q7; ++k) {
        double cu = 0, cn = 0;
        for (int a = 0; a < 3; ++a) {
            cu += C7[k][a] * u[a];
            cn += C7[k][a] * nrm[a];
        }
        g[k] = W7[k] * phi * (1.0 + cu / CS2_7) + W7[k] * gamma * (1.0 - phi * phi) * cn;
    }
}

/* grad phi = (1/cs2) sum_i w_i c_i phi(x + c_i); H = (1/cs^4) sum_i w_i H2_i phi(x + c_i);
 * n = grad phi / m with m = sqrt(|grad phi|^2 + eps^2) (the unit normal of
 * Sec. 2.2, regularised where the gradient vanishes); kappa = div n
 * = tr H / m - grad.H.grad / m^3; F = -(sigma/2) kappa grad phi. */
void orc_interface(const double* phi27, double sigma, double eps, double* grad3,
                   double* hess6, double* normal3, double* kappa, double* force3) {
    tables();
    double g[3] = {0, 0, 0}, h[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a) {
            g[a] += W[i] * C[i][a] * phi27[i] / CS2;
            for (int b = 0; b < 3; ++b) h[a][b] += W[i] * H2[i][a][b] * phi27[i] / (CS2 * CS2);
        }
    double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + eps * eps);
    double n[3] = {0, 0, 0}, ghg = 0, k = 0;
    if (m > 0) {
        for (int a = 0; a < 3; ++a) n[a] = g[a] / m;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) ghg += g[a] * h[a][b] * g[b];
        k = (h[0][0] + h[1][1] + h[2][2]) / m - ghg / (m * m * m);
    }
    for (int a = 0; a < 3; ++a) {
        if (grad3) grad3[a] = g[a];
        if (normal3) normal3[a] = n[a];
        if (force3) force3[a] = -0.5 * sigma * k * g[a];
    }
    if (hess6) {
        hess6[0] = h[0][0];
        hess6[1] = h[1][1];
        hess6[2] = h[2][2];
        hess6[3] = h[0][1];
        hess6[4] = h[0][2];
        hess6[5] = h[1][2];
    }
    if (kappa) *kappa = k;
}

/* ------------------------------------------------------- ghost resolution */

/* Source coordinate of grid coordinate g along an axis of n nodes whose
 * lower/upper faces follow rule lo/hi; only |distance| <= 2 is ever asked. */
static int resolve_axis(int g, int n, int lo, int hi, int* mirror, int* inlet) {
    if (g >= 0 && g < n) return g;
    int kind = g < 0 ? lo : hi;
    switch (kind) {
        case ORC_PERIODIC: return ((g % n) + n) % n;
        case ORC_FREE_SLIP: *mirror = 1; return g < 0 ? -1 - g : 2 * n - 1 - g;
        case ORC_INLET: *inlet = 1; return g < 0 ? 0 : n - 1;
        default: return g < 0 ? 0 : n - 1; /* ORC_OUTFLOW */
    }
}

typedef struct {
    const orc_params* p;
    int64_t t;
    const double *rho, *u, *pi, *phi;
    int64_t N;
} fields_t;

static void fetch_node(const fields_t* fs, int gx, int gy, int gz, node_t* nd) {
    const orc_params* p = fs->p;
    int mx = 0, my = 0, mz = 0, in = 0;
    int sx = resolve_axis(gx, p->nx, p->face[0], p->face[1], &mx, &in);
    int sy = resolve_axis(gy, p->ny, p->face[2], p->face[3], &my, &in);
    int sz = resolve_axis(gz, p->nz, p->face[4], p->face[5], &mz, &in);
    int64_t n = sx + (int64_t)p->nx * (sy + (int64_t)p->ny * sz);
    const int64_t N = fs->N;
    nd->rho = fs->rho[n];
    for (int a = 0; a < 3; ++a) nd->u[a] = fs->u[a * N + n];
    nd->P[0][0] = fs->pi[0 * N + n];
    nd->P[1][1] = fs->pi[1 * N + n];
    nd->P[2][2] = fs->pi[2 * N + n];
    nd->P[0][1] = nd->P[1][0] = fs->pi[3 * N + n];
    nd->P[0][2] = nd->P[2][0] = fs->pi[4 * N + n];
    nd->P[1][2] = nd->P[2][1] = fs->pi[5 * N + n];
    nd->phi = fs->phi[n];
    nd->inlet = in;
    if (in) orc_inlet_state(p, sx, sy, fs->t, nd->u, &nd->phi);
    const double sg[3] = {mx ? -1.0 : 1.0, my ? -1.0 : 1.0, mz ? -1.0 : 1.0};
    for (int a = 0; a < 3; ++a) {
        nd->u[a] *= sg[a];
        for (int b = 0; b < 3; ++b) nd->P[a][b] *= sg[a] * sg[b];
    }
}

static double fetch_phi(const fields_t* fs, int gx, int gy, int gz) {
    const orc_params* p = fs->p;
    int m = 0, in = 0;
    int sx = resolve_axis(gx, p->nx, p->face[0], p->face[1], &m, &in);
    int sy = resolve_axis(gy, p->ny, p->face[2], p->face[3], &m, &in);
    int sz = resolve_axis(gz, p->nz, p->face[4], p->face[5], &m, &in);
    if (in) {
        double u3[3], ph;
        orc_inlet_state(p, sx, sy, fs->t, u3, &ph);
        return ph;
    }
    return fs->phi[sx + (int64_t)p->nx * (sy + (int64_t)p->ny * sz)];
}

/* Post-collision f and g of the node (or ghost) at (gx, gy, gz). */
static void node_post(const fields_t* fs, int gx, int gy, int gz, double* f, double* g) {
    const orc_params* p = fs->p;
    node_t nd;
    fetch_node(fs, gx, gy, gz, &nd);
    double F[3] = {0, 0, 0}, nrm[3] = {0, 0, 0};
    if (!nd.inlet) {
        double phi27[Q];
        for (int i = 0; i < Q; ++i) phi27[i] = fetch_phi(fs, gx + C[i][0], gy + C[i][1], gz + C[i][2]);
        orc_interface(phi27, p->sigma, p->normal_eps, NULL, NULL, nrm, NULL, F);
        for (int a = 0; a < 3; ++a) F[a] += p->ext_force[a];
    }
    double a2[3][3];
    if (p->ce_neq) {
        double j27[3 * Q], a2_6[6];
        for (int i = 0; i < Q; ++i) {
            node_t nb;
            fetch_node(fs, gx + C[i][0], gy + C[i][1], gz + C[i][2], &nb);
            for (int a = 0; a < 3; ++a) j27[3 * i + a] = nb.rho * nb.u[a];
        }
        orc_ce_neq(j27, p->omega, a2_6);
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) a2[ia[k]][ib[k]] = a2[ib[k]][ia[k]] = a2_6[k];
    }
    post_f(&nd, F, p->omega, p->ce_neq ? (const double(*)[3])a2 : NULL, f);
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = nd.u[a] + F[a] / (2.0 * nd.rho);
    post_g(nd.phi, u, nrm, p->gamma, g);
}

/* Stored moments of a population set: rho, u = j/rho, P = Pi - rho cs2 I - rho u u, phi. */
static void moments_of(const double* f, const double* g, double* m11) {
    double rho = 0, j[3] = {0, 0, 0}, pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, phi = 0;
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += C[i][a] * f[i];
            for (int b = 0; b < 3; ++b) pi[a][b] += C[i][a] * C[i][b] * f[i];
        }
    }
    for (int k = 0; k < Q7; ++k) phi += g[k];
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    m11[0] = rho;
    for (int a = 0; a < 3; ++a) m11[1 + a] = u[a];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        int a = ia[k], b = ib[k];
        m11[4 + k] = pi[a][b] - rho * CS2 * (a == b) - rho * u[a] * u[b];
    }
    m11[10] = phi;
}

/* ------------------------------------------------------------ simulation */

struct orc_sim {
    orc_params p;
    int64_t N, t;
    double *f, *fn, *g, *gn;
    double *rho, *u, *pi, *phi;
};

static int valid_params(const orc_params* p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return 0;
    for (int a = 0; a < 3; ++a) {
        int lo = p->face[2 * a], hi = p->face[2 * a + 1];
        int n = a == 0 ? p->nx : a == 1 ? p->ny : p->nz;
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return 0;
        if ((lo == ORC_PERIODIC) != (hi == ORC_PERIODIC)) return 0;
        if (lo != ORC_PERIODIC && n < 2) return 0;
    }
    for (int k = 0; k < 6; ++k)
        if (p->face[k] == ORC_INLET && k != 4) return 0;
    if (!(p->omega > 0.0 && p->omega < 2.0)) return 0;
    if (p->face[4] == ORC_INLET && !(p->inlet_width > 0.0)) return 0;
    if (!(p->normal_eps >= 0.0)) return 0;
    return 1;
}

orc_sim* orc_create(const orc_params* p) {
    tables();
    if (!p || !valid_params(p)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = (int64_t)p->nx * p->ny * p->nz;
    size_t N = (size_t)s->N;
    s->f = (double*)calloc(Q * N, sizeof(double));
    s->fn = (double*)calloc(Q * N, sizeof(double));
    s->g = (double*)calloc(Q7 * N, sizeof(double));
    s->gn = (double*)calloc(Q7 * N, sizeof(double));
    s->rho = (double*)calloc(N, sizeof(double));
    s->u = (double*)calloc(3 * N, sizeof(double));
    s->pi = (double*)calloc(6 * N, sizeof(double));
    s->phi = (double*)calloc(N, sizeof(double));
    if (!s->f || !s->fn || !s->g || !s->gn || !s->rho || !s->u || !s->pi || !s->phi) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f);
    free(s->fn);
    free(s->g);
    free(s->gn);
    free(s->rho);
    free(s->u);
    free(s->pi);
    free(s->phi);
    free(s);
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_set_state(orc_sim* s, const double* rho, const double* u, const double* pi,
                  const double* phi, int64_t t0) {
    tables();
    const int64_t N = s->N;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double un[3] = {u[n], u[N + n], u[2 * N + n]};
        double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (pi) {
            P[0][0] = pi[n];
            P[1][1] = pi[N + n];
            P[2][2] = pi[2 * N + n];
            P[0][1] = P[1][0] = pi[3 * N + n];
            P[0][2] = P[2][0] = pi[4 * N + n];
            P[1][2] = P[2][1] = pi[5 * N + n];
        }
        double feq[Q];
        orc_feq3(rho[n], un, feq);
        for (int i = 0; i < Q; ++i) {
            double h2 = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) h2 += H2[i][a][b] * P[a][b];
            s->f[i * N + n] = feq[i] + W[i] * h2 / (2.0 * CS2 * CS2);
        }
        double zero[3] = {0, 0, 0}, g[Q7];
        post_g(phi[n], un, zero, 0.0, g);
        for (int k = 0; k < Q7; ++k) s->g[k * N + n] = g[k];
    }
    s->t = t0;
    return 0;
}

static void moments_all(orc_sim* s) {
    const int64_t N = s->N;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double f[Q], g[Q7], m[11];
        for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
        for (int k = 0; k < Q7; ++k) g[k] = s->g[k * N + n];
        moments_of(f, g, m);
        s->rho[n] = m[0];
        for (int a = 0; a < 3; ++a) s->u[a * N + n] = m[1 + a];
        for (int k = 0; k < 6; ++k) s->pi[k * N + n] = m[4 + k];
        s->phi[n] = m[10];
    }
}

void orc_step(orc_sim* s, int nsteps) {
    tables();
    const orc_params* p = &s->p;
    const int64_t N = s->N;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    for (int step = 0; step < nsteps; ++step) {
        /* (1) moments of the current populations */
        moments_all(s);
        fields_t fs = {p, s->t, s->rho, s->u, s->pi, s->phi, N};
        /* (2)-(4) every node of the domain and of its one-node ghost shell
         * collides and pushes f_i^post to x + c_i when that lies in the domain */
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
        for (int gz = -1; gz <= nz; ++gz)
            for (int gy = -1; gy <= ny; ++gy) {
                double f[Q], g[Q7];
                for (int gx = -1; gx <= nx; ++gx) {
                    node_post(&fs, gx, gy, gz, f, g);
                    for (int i = 0; i < Q; ++i) {
                        int x = gx + C[i][0], y = gy + C[i][1], z = gz + C[i][2];
                        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                        s->fn[i * N + x + (int64_t)nx * (y + (int64_t)ny * z)] = f[i];
                    }
                    for (int k = 0; k < Q7; ++k) {
                        int x = gx + C7[k][0], y = gy + C7[k][1], z = gz + C7[k][2];
                        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                        s->gn[k * N + x + (int64_t)nx * (y + (int64_t)ny * z)] = g[k];
                    }
                }
            }
        double* tf = s->f;
        s->f = s->fn;
        s->fn = tf;
        double* tg = s->g;
        s->g = s->gn;
        s->gn = tg;
        s->t += 1;
    }
    moments_all(s);
}

void orc_get_moments(const orc_sim* s, double* rho, double* u, double* pi, double* phi) {
    orc_sim* m = (orc_sim*)s;
    moments_all(m);
    const int64_t N = s->N;
    if (rho) memcpy(rho, s->rho, N * sizeof(double));
    if (u) memcpy(u, s->u, 3 * N * sizeof(double));
    if (pi) memcpy(pi, s->pi, 6 * N * sizeof(double));
    if (phi) memcpy(phi, s->phi, N * sizeof(double));
}

/* Neumaier's compensated summation, so that the totals are exact to FP64
 * rounding of each node's own moment. */
typedef struct {
    double sum, comp;
} ksum_t;

static void kadd(ksum_t* k, double x) {
    double t = k->sum + x;
    if (fabs(k->sum) >= fabs(x))
        k->comp += (k->sum - t) + x;
    else
        k->comp += (x - t) + k->sum;
    k->sum = t;
}

void orc_sums(const orc_sim* s, double* mass, double* phi_total, double* momentum3) {
    const int64_t N = s->N;
    ksum_t m = {0, 0}, ph = {0, 0}, j[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t n = 0; n < N; ++n) {
        double rho = 0, jn[3] = {0, 0, 0}, phi = 0;
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * N + n];
            rho += fi;
            for (int a = 0; a < 3; ++a) jn[a] += C[i][a] * fi;
        }
        for (int k = 0; k < Q7; ++k) phi += s->g[k * N + n];
        kadd(&m, rho);
        kadd(&ph, phi);
        for (int a = 0; a < 3; ++a) kadd(&j[a], jn[a]);
    }
    if (mass) *mass = m.sum + m.comp;
    if (phi_total) *phi_total = ph.sum + ph.comp;
    if (momentum3)
        for (int a = 0; a < 3; ++a) momentum3[a] = j[a].sum + j[a].comp;
}

int64_t orc_time(const orc_sim* s) { return s->t; }

int orc_step_sample(const orc_params* p, int64_t t, const double* rho, const double* u,
                    const double* pi, const double* phi, int64_t nsamp, const int64_t* idx,
                    double* out) {
    tables();
    if (!p || !valid_params(p)) return -1;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    fields_t fs = {p, t, rho, u, pi, phi, N};
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t s = 0; s < nsamp; ++s) {
        int64_t n = idx[s];
        if (n < 0 || n >= N) {
            bad = 1;
            continue;
        }
        int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((int64_t)p->nx * p->ny));
        double fin[Q], gin[Q7], f[Q], g[Q7];
        for (int i = 0; i < Q; ++i) {
            node_post(&fs, x - C[i][0], y - C[i][1], z - C[i][2], f, g);
            fin[i] = f[i];
        }
        for (int k = 0; k < Q7; ++k) {
            node_post(&fs, x - C7[k][0], y - C7[k][1], z - C7[k][2], f, g);
            gin[k] = g[k];
        }
        moments_of(fin, gin, out + 11 * s);
    }
    return bad ? -1 : 0;
}

void orc_lattice(double* c27, double* w27, double* c7, double* w7) {
    tables();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c27[3 * i + a] = C[i][a];
        w27[i] = W[i];
    }
    for (int k = 0; k < Q7; ++k) {
        for (int a = 0; a < 3; ++a) c7[3 * k + a] = C7[k][a];
        w7[k] = W7[k];
    }
}
