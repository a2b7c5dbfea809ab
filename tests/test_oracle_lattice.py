"""Pins of the oracle's per-node pieces against closed forms and printed values.

Lattice isotropy (Sec. 2, Fig. 2), the Hermite moments of the rebuilt
populations (Eq. LBexp, eqts, noneqts), the interface geometry (Sec. 2.2) and
the Philox4x32-10 generator of the inlet noise.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _frac(x):
    return Fraction(x).limit_denominator(10000)


def test_d3q27_isotropy_exact():
    c, w, _, _ = oracle.lattice()
    wf = [_frac(x) for x in w]
    assert sorted(set(wf)) == [Fraction(1, 216), Fraction(1, 54), Fraction(2, 27), Fraction(8, 27)]
    assert sum(wf) == 1
    ci = c.astype(int)
    assert len({tuple(v) for v in ci}) == 27
    for a in range(3):
        assert sum(wf[i] * ci[i, a] for i in range(27)) == 0
        for b in range(3):
            m2 = sum(wf[i] * ci[i, a] * ci[i, b] for i in range(27))
            assert m2 == (Fraction(1, 3) if a == b else 0)
            for g in range(3):
                assert sum(wf[i] * ci[i, a] * ci[i, b] * ci[i, g] for i in range(27)) == 0
    # fourth moment: cs^4 (d_ab d_gd + d_ag d_bd + d_ad d_bg)
    for a, b, g, d in itertools.product(range(3), repeat=4):
        m4 = sum(wf[i] * ci[i, a] * ci[i, b] * ci[i, g] * ci[i, d] for i in range(27))
        iso = Fraction(1, 9) * ((a == b) * (g == d) + (a == g) * (b == d) + (a == d) * (b == g))
        assert m4 == iso


def test_d3q7_isotropy_exact():
    _, _, c7, w7 = oracle.lattice()
    wf = [_frac(x) for x in w7]
    assert sum(wf) == 1
    ci = c7.astype(int)
    for a in range(3):
        assert sum(wf[k] * ci[k, a] for k in range(7)) == 0
        for b in range(3):
            assert sum(wf[k] * ci[k, a] * ci[k, b] for k in range(7)) == (Fraction(1, 4) if a == b else 0)


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def _moments(f):
    c, _, _, _ = oracle.lattice()
    rho = f.sum()
    j = c.T @ f
    pi = np.einsum("ia,ib,i->ab", c, c, f)
    q = np.einsum("ia,ib,ig,i->abg", c, c, c, f)
    return rho, j, pi, q


def _sym(p6):
    xx, yy, zz, xy, xz, yz = p6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments_third_order(seed):
    """Eq. eqts: rho, rho u, rho cs2 I + rho u u and, on the D3Q27-supported
    third-order components, rho (u u u + cs2 (u d + d u + ...))."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1)
    u = 0.1 * rng.uniform(-1, 1, 3)
    rho_m, j, pi, q = _moments(oracle.feq3(rho, u))
    assert abs(rho_m - rho) < 1e-14
    assert np.allclose(j, rho * u, atol=5e-15, rtol=0)
    assert np.allclose(pi, rho * CS2 * np.eye(3) + rho * np.outer(u, u), atol=5e-15, rtol=0)
    d = np.eye(3)
    for a, b, g in itertools.product(range(3), repeat=3):
        if a == b == g:
            continue  # c^3 = c on D3Q27: the xxx moments are not supported
        exact = rho * (u[a] * u[b] * u[g] + CS2 * (u[a] * d[b, g] + u[b] * d[a, g] + u[g] * d[a, b]))
        assert abs(q[a, b, g] - exact) < 5e-15


@pytest.mark.parametrize("seed", range(6))
def test_post_collision_moments(seed):
    """f^post = f^eq + (1 - omega) f^neq (Eq. LBexp) with Guo forcing:
    mass kept, momentum gains F, Pi relaxes as Pi^eq + (1-omega) Pi^neq plus the
    forcing term (1 - omega/2)(u F + F u), u = u_raw + F/(2 rho)."""
    rng = np.random.default_rng(100 + seed)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1)
    u_raw = 0.08 * rng.uniform(-1, 1, 3)
    p6 = 1e-3 * rng.uniform(-1, 1, 6)
    F = (1e-4 * rng.uniform(-1, 1, 3)) if seed % 2 else np.zeros(3)
    omega = rng.uniform(0.5, 1.99)
    f = oracle.post_populations(rho, u_raw, p6, F, omega)
    rho_m, j, pi, q = _moments(f)
    u = u_raw + F / (2 * rho)
    assert abs(rho_m - rho) < 1e-14
    assert np.allclose(j, rho * u_raw + F, atol=5e-15, rtol=0)
    pi_pre = rho * CS2 * np.eye(3) + rho * np.outer(u_raw, u_raw) + _sym(p6)
    pi_eq = rho * CS2 * np.eye(3) + rho * np.outer(u, u)
    expect = pi_eq + (1 - omega) * (pi_pre - pi_eq) + (1 - omega / 2) * (np.outer(u, F) + np.outer(F, u))
    assert np.allclose(pi, expect, atol=5e-15, rtol=0)
    # third-order: equilibrium part plus (1 - omega) times the recursive a3 (Eq. noneqts)
    a2 = pi_pre - pi_eq
    d = np.eye(3)
    for a, b, g in itertools.product(range(3), repeat=3):
        if a == b == g:
            continue
        q_eq = rho * (u[a] * u[b] * u[g] + CS2 * (u[a] * d[b, g] + u[b] * d[a, g] + u[g] * d[a, b]))
        a3 = u[a] * a2[b, g] + u[b] * a2[a, g] + u[g] * a2[a, b]
        # moment of c_a c_b c_g over the cs2-shifted lower orders of the post state
        j_post = rho * u_raw + F
        a2_post = pi - rho * CS2 * np.eye(3)
        lower = CS2 * (j_post[a] * d[b, g] + j_post[b] * d[a, g] + j_post[g] * d[a, b])
        a3_post = q[a, b, g] - lower
        a3_eq = q_eq - CS2 * rho * (u[a] * d[b, g] + u[b] * d[a, g] + u[g] * d[a, b])
        assert abs(a3_post - (a3_eq + (1 - omega) * a3)) < 5e-15, (a, b, g)
    assert np.all(np.isfinite(a2_post))


def test_omega_one_gives_equilibrium():
    """omega = 1 and F = 0: the post-collision state is the equilibrium itself."""
    u = np.array([0.03, -0.02, 0.05])
    f = oracle.post_populations(1.02, u, np.array([1e-3, -2e-3, 5e-4, 3e-4, -1e-4, 2e-4]),
                                np.zeros(3), 1.0)
    assert np.allclose(f, oracle.feq3(1.02, u), atol=1e-16, rtol=0)


def _phi27(func):
    c, _, _, _ = oracle.lattice()
    return np.array([func(ci) for ci in c])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("eps", [0.0, 1e-2, 0.3])
def test_interface_geometry_quadratic(seed, eps):
    """For phi = a.x + x.B.x/2 the lattice stencils are exact: grad = a, H = B.
    The normal n = grad phi / m, m = sqrt(|grad phi|^2 + eps^2) (eps = 0: the
    unit normal of Sec. 2.2), and its divergence evaluated analytically,
    kappa = div n = tr B / m - a.B.a / m^3; F = -(sigma/2) kappa grad phi."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, 3)
    B = rng.uniform(-1, 1, (3, 3))
    B = B + B.T
    g, h, n, k, F = oracle.interface(_phi27(lambda x: a @ x + 0.5 * x @ B @ x + 0.3), 0.02, eps)
    assert np.allclose(g, a, atol=1e-14)
    assert np.allclose(h, [B[0, 0], B[1, 1], B[2, 2], B[0, 1], B[0, 2], B[1, 2]], atol=1e-14)
    m = math.sqrt(a @ a + eps * eps)
    assert np.allclose(n, a / m, atol=1e-14)
    kappa = np.trace(B) / m - a @ B @ a / m ** 3
    assert abs(k - kappa) < 1e-12
    assert np.allclose(F, -0.01 * kappa * a, atol=1e-14)


def test_interface_divergence_by_finite_differences():
    """kappa equals a centred finite difference of the regularised normal
    field of a smooth non-quadratic phi (independent of the stencil algebra)."""
    eps = 1e-2
    f = lambda x: math.tanh(0.4 * x[0] - 0.3 * x[1] + 0.2 * x[2] + 0.05 * x[0] * x[1])
    def grad_exact(x):
        s = 1 - math.tanh(0.4 * x[0] - 0.3 * x[1] + 0.2 * x[2] + 0.05 * x[0] * x[1]) ** 2
        return s * np.array([0.4 + 0.05 * x[1], -0.3 + 0.05 * x[0], 0.2])
    def normal(x):
        g = grad_exact(x)
        return g / math.sqrt(g @ g + eps * eps)
    # lattice values at spacing h: scale the field so the 27-point stencil sees a smooth function
    hs = 0.05
    g, h, n, k, F = oracle.interface(_phi27(lambda c: f(hs * c)), 1.0, eps * hs)
    # the stencil returns derivatives per lattice unit; convert to per unit length
    kappa_fd = sum((normal(hs * np.eye(3)[a])[a] - normal(-hs * np.eye(3)[a])[a]) / (2 * hs)
                   for a in range(3))
    assert abs(k / hs - kappa_fd) < 2e-3 * max(1.0, abs(kappa_fd))


def test_interface_sphere_sign():
    """phi = +1 inside a sphere: the normal points inward, kappa ~ -2/r, and the
    force points inward (it compresses the droplet, p_in > p_out)."""
    r0 = 20.0
    ctr = np.array([r0, 0.0, 0.0])  # node at distance r0 from the centre on +x
    g, h, n, k, F = oracle.interface(_phi27(lambda x: -np.linalg.norm(x + ctr)), 0.01, 0.0)
    assert n[0] < -0.999
    assert abs(k - (-2.0 / r0)) < 0.01 * 2.0 / r0
    assert F[0] < 0


def test_interface_flat_bulk_regularised():
    """In a uniform phase the regularised normal and the force vanish (up to
    the rounding of the gradient stencil), unlike the bare unit normal."""
    g, h, n, k, F = oracle.interface(np.ones(27), 0.05, 1e-2)
    assert np.max(np.abs(n)) < 1e-13 and np.max(np.abs(F)) < 1e-15


def test_inlet_state_profile_and_noise():
    p = oracle.make_params(64, 64, 8, 1.9, faces=(3, 3, 3, 3, 1, 2), inlet_u=(0, 0, 0.05),
                           inlet_diameter=16, inlet_cx=32, inlet_cy=32, inlet_width=3,
                           noise_amp=0.01, seed=7)
    u_c, phi_c = oracle.inlet_state(p, 32, 32, 0)
    assert phi_c > 0.999 and abs(u_c[2] - 0.05) <= 0.01 * 0.05 * 1.0001
    u_f, phi_f = oracle.inlet_state(p, 0, 0, 0)
    assert phi_f < -0.999 and np.all(np.abs(u_f) < 1e-6)
    # the noise is Philox4x32-10 on counter (x + nx y, t, 0, 0), key (seed) mapped to [0, 1)
    xs = []
    for t in range(200):
        u, _ = oracle.inlet_state(p, 32, 32, t)
        raw = oracle.philox4x32_10([32 + 64 * 32, t, 0, 0], [7, 0])
        r = (raw[:3] >> 8) * 2.0 ** -24
        s = 0.5 * (1 + phi_c)
        assert np.allclose(u, s * (np.array([0, 0, 0.05]) + 0.01 * 0.05 * (2 * r - 1)), atol=1e-17)
        xs.append(u)
    xs = np.array(xs)
    assert np.max(np.abs(xs[:, 0])) <= 0.01 * 0.05
    assert abs(xs[:, 0].mean()) < 0.2 * 0.01 * 0.05  # zero-mean noise
