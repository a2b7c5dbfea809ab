/*
 * FP64 CPU oracle of the multicomponent thread-safe lattice Boltzmann step
 * (Montessori, Hegele, Lauricella, arXiv 2403.15773).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * The oracle keeps the paper's own data layout: 27 D3Q27 populations f_i and
 * 7 D3Q7 populations g_i per node (A-B buffered), and advances them with the
 * literal push form of the fused step (Sec. 2, Eq. pushLB / fullstrcoll),
 * using the third-order equilibrium (Eq. eqts), the recursive third-order
 * non-equilibrium reconstruction (Eq. noneqts), the continuum-surface force
 * and the D3Q7 conservative phase-field update (Sec. 2.2, Eqs. intcapturing,
 * antidiff), and the non-equilibrium-extrapolation boundary closure
 * (Eq. original_neq / neq_final).
 *
 * Arrays crossing this interface are FP64, structure of arrays, x fastest:
 * index n = x + nx*(y + ny*z).  Vector fields are [3][N] (x, y, z blocks),
 * tensors [6][N] in the order xx, yy, zz, xy, xz, yz.
 */
#ifndef TSLB_ORACLE_H
#define TSLB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_INLET = 1, ORC_OUTFLOW = 2, ORC_FREE_SLIP = 3 };

typedef struct {
    int nx, ny, nz;
    double omega;            /* BGK relaxation frequency, nu = cs2 (1/omega - 1/2) */
    double sigma;            /* surface tension */
    double gamma;            /* anti-diffusion strength Gamma (1/W for an interface of width W) */
    int face[6];             /* -x,+x,-y,+y,-z,+z ; ORC_INLET only on -z */
    double inlet_u[3];       /* imposed jet velocity on the nozzle */
    double inlet_diameter;   /* nozzle diameter D (nodes) */
    double inlet_cx, inlet_cy;   /* nozzle centre on the inlet face */
    double inlet_width;      /* W of the smoothed nozzle edge */
    double noise_amp;        /* velocity noise amplitude as a fraction of |inlet_u| */
    uint64_t seed;           /* Philox key of the inlet noise */
    double ext_force[3];     /* test hook: uniform body force added to the interface force */
    double normal_eps;       /* regularisation of the interface normal, n = grad phi / sqrt(|grad phi|^2 + eps^2) */
    int ce_neq;              /* 1: a2_neq from the Chapman-Enskog strain rate of the neighbours'
                                momentum, -(cs2/omega)(d_a j_b + d_b j_a), instead of Pi - Pi^eq */
} orc_params;

typedef struct orc_sim orc_sim;

/* Returns NULL on invalid parameters or allocation failure. */
orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);

/* Populations := third-order equilibrium at (rho, u) plus the second-order
 * Hermite non-equilibrium carrying pi (pi may be NULL = 0); g := D3Q7
 * equilibrium at (phi, u).  Step counter := t0. */
int orc_set_state(orc_sim* s, const double* rho, const double* u,
                  const double* pi, const double* phi, int64_t t0);

/* n fused steps. */
void orc_step(orc_sim* s, int n);

/* Moments of the current populations: rho, u = j/rho, pi = P = Pi - rho cs2 I - rho u u. */
void orc_get_moments(const orc_sim* s, double* rho, double* u, double* pi, double* phi);
void orc_sums(const orc_sim* s, double* mass, double* phi_total, double* momentum3);
int64_t orc_time(const orc_sim* s);
int orc_threads(void);
/* Threads of the later steps (n >= 1; timing only: the results do not depend on it). */
void orc_set_threads(int n);

/* One step evaluated only at the listed nodes, from a full stored state
 * (rho, u, pi, phi over the whole grid at step t).  out: 11 values per sample
 * (rho, ux, uy, uz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz, phi). */
int orc_step_sample(const orc_params* p, int64_t t, const double* rho, const double* u,
                    const double* pi, const double* phi, int64_t nsamp,
                    const int64_t* idx, double* out);

/* Per-node pieces, exported for the unit pins. */
void orc_lattice(double* c27 /*27*3*/, double* w27, double* c7 /*7*3*/, double* w7);
void orc_post_populations(double rho, const double* u_raw, const double* pi,
                          const double* force, double omega, double* f27);
void orc_feq3(double rho, const double* u, double* f27);
void orc_interface(const double* phi27 /* phi(x + c_i), i in oracle order */,
                   double sigma, double eps, double* grad3, double* hess6, double* normal3,
                   double* kappa, double* force3);
void orc_ce_neq(const double* j27, double omega, double* a2_6);
void orc_philox4x32_10(const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4);
void orc_inlet_state(const orc_params* p, int x, int y, int64_t t, double* u3, double* phi);

#ifdef __cplusplus
}
#endif
#endif
