"""Pins of the oracle's Chapman-Enskog closure (Sec. 2.1, the recursive
regularisation): a2_neq estimated from the strain rate of the momentum field,
-(cs2 / omega)(d_a j_b + d_b j_a), with the gradient taken by the D3Q27
isotropic stencil (1/cs2) sum_i w_i c_i j(x + c_i), in place of the projection
Pi - Pi^eq of the stored moments.

The stencil is pinned by fields whose derivative is known exactly (linear and
quadratic: a symmetric stencil differentiates them exactly) and by its known
truncation on cubics; the prefactor by the projection variant, whose stored
Pi^neq follows the same Chapman-Enskog relation at leading order, and by the
shear-wave viscosity nu = cs2 (1/omega - 1/2) that both closures must give."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_15773_gb300 import inputs

P, FS = oracle.PERIODIC, oracle.FREE_SLIP
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _sim(nx, ny, nz, omega, sigma=0.0, gamma=0.0, faces=(P,) * 6, **kw):
    return oracle.OracleSim(oracle.make_params(nx, ny, nz, omega, sigma, gamma, faces, **kw))


def _j27(func):
    c, _, _, _ = oracle.lattice()
    return np.array([func(ci.astype(float)) for ci in c])


@pytest.mark.parametrize("seed", range(4))
def test_stencil_exact_on_linear_and_quadratic_fields(seed):
    """j(x) = j0 + G x + (x.Hb x)_b: the symmetric stencil returns G exactly
    (the quadratic part is even and drops out), so
    a2_ab = -(cs2/omega)(G_ba + G_ab)."""
    rng = np.random.default_rng(seed)
    j0 = rng.normal(size=3)
    G = rng.normal(size=(3, 3))          # G[b, a] = d_a j_b
    H = rng.normal(size=(3, 3, 3))
    omega = 0.6 + 1.3 * rng.random()
    a2 = oracle.ce_neq(_j27(lambda x: j0 + G @ x + np.einsum("a,bac,c->b", x, H, x)), omega)
    for k, (a, b) in enumerate(PAIRS):
        want = -(1.0 / 3.0) / omega * (G[b, a] + G[a, b])
        assert abs(a2[k] - want) < 1e-14 * (1 + abs(want))


def test_stencil_truncation_on_cubics():
    """Along its own axis the stencil is the central difference, which turns
    x^3 into 1 (= h^2 f'''/6); across the other axes it smooths with the
    1D weights (1/6, 2/3, 1/6), which turns x y^2 into d_x = 1/3."""
    omega = 1.0
    a2 = oracle.ce_neq(_j27(lambda x: np.array([x[0] ** 3, 0.0, 0.0])), omega)
    assert abs(a2[0] - (-(1.0 / 3.0) * 2.0)) < 1e-15
    assert np.all(np.abs(a2[1:]) < 1e-15)
    a2 = oracle.ce_neq(_j27(lambda x: np.array([x[0] * x[1] ** 2, 0.0, 0.0])), omega)
    assert abs(a2[0] - (-(1.0 / 3.0) * 2.0 / 3.0)) < 1e-15
    assert np.all(np.abs(a2[1:]) < 1e-15)
    # a mixed term: j_y = x z -> d_x j_y = z smoothed in z = 0 at the centre
    a2 = oracle.ce_neq(_j27(lambda x: np.array([0.0, x[0] * x[2], 0.0])), omega)
    assert np.all(np.abs(a2) < 1e-15)


def _shear(L, omega, A, ce, steps):
    k = 2 * math.pi / L
    y = np.arange(L)
    u = np.zeros((3, 1, L, 1))
    u[0, 0, :, 0] = A * np.sin(k * y)
    s = _sim(1, L, 1, omega, ce_neq=ce)
    s.set_state(np.ones((1, L, 1)), u, -np.ones((1, L, 1)))
    s.step(steps)
    return s, k, y


@pytest.mark.parametrize("omega", [1.0, 1.6, 1.9])
def test_projection_pi_neq_follows_chapman_enskog(omega):
    """In a decaying shear wave the projection closure's stored Pi^neq_xy is
    -(cs2/omega) d_y j_x to O(k^2): the relation the closure estimates.  A
    prefactor off by cs2^2 (the 1/(omega cs2) one) misses by 9x."""
    L, A = 64, 1e-4
    s, k, y = _shear(L, omega, A, False, 40)
    rho, u, pi, _ = s.moments()
    amp = 2.0 / L * np.sum(u[0, 0, :, 0] * np.sin(k * y))
    pxy = pi[3, 0, :, 0]
    want = -(1.0 / 3.0) / omega * amp * k * np.cos(k * y)
    assert np.max(np.abs(pxy - want)) < 0.03 * np.max(np.abs(want))


@pytest.mark.parametrize("omega", [1.0, 1.6, 1.9])
def test_chapman_enskog_shear_wave_viscosity(omega):
    """u_x = A sin(2 pi y / L) decays at nu k^2, nu = cs2 (1/omega - 1/2), with
    the gradient closure too: its one-step amplification is exactly
    1 - (1 - cos k)/3 - (1 - omega) sin^2 k / (3 omega) = 1 - nu k^2 + O(k^4);
    at omega = 1.9 (nu = 0.009) the k^4 term is 4 % of nu k^2 for L = 64."""
    L, A = 64, 1e-4
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    T = int(round(0.7 / (nu * (2 * math.pi / L) ** 2)))
    s, k, y = _shear(L, omega, A, True, 0)
    amp0 = A
    s.step(T)
    amp1 = 2.0 / L * np.sum(s.moments()[1][0, 0, :, 0] * np.sin(k * y))
    g = 1 - (1 - math.cos(k)) / 3 - (1 - omega) * math.sin(k) ** 2 / (3 * omega)
    assert abs(amp1 / amp0 - g ** T) < 1e-9
    rate = -math.log(amp1 / amp0) / T
    assert abs(rate / (nu * k * k) - 1.0) < 0.05


def test_chapman_enskog_rest_and_uniform_flow_fixed_points():
    s = _sim(5, 4, 6, 1.7, sigma=0.01, gamma=1 / 3, ce_neq=True)
    N = s.N
    s.set_state(np.ones(N), np.zeros(3 * N), np.ones(N))
    s.step(20)
    rho, u, pi, phi = s.moments()
    assert np.max(np.abs(rho - 1)) < 20 * 2.3e-16 and np.max(np.abs(u)) < 1e-16
    u0 = np.array([0.03, -0.02, 0.01])
    s.set_state(np.full(N, 1.01), np.repeat(u0, N), -np.ones(N))
    s.step(3)
    rho, u, pi, phi = s.moments()
    for a in range(3):
        assert np.max(np.abs(u[a] - u0[a])) < 1e-15
    assert np.max(np.abs(pi)) < 1e-15


def test_chapman_enskog_conserves_mass_momentum_phase():
    """Periodic, no surface tension: the closure changes only the second and
    third moments, so mass, momentum and phase are conserved."""
    L = 12
    rho, u, pi, phi = inputs.random_smooth_fields(L, L, L, seed=5, amp_rho=1e-2, amp_u=3e-2,
                                                   amp_pi=0.0)
    phi = np.tanh(3 * phi)
    s = _sim(L, L, L, 1.8, sigma=0.0, gamma=1 / 3, ce_neq=True)
    s.set_state(rho, u, phi)
    m0, p0, j0 = s.sums()
    s.step(30)
    m1, p1, j1 = s.sums()
    # rounding only: one unit roundoff per node and step at most
    bound = 2.3e-16 * L ** 3 * 30
    assert abs(m1 - m0) < bound and abs(p1 - p0) < bound
    assert np.max(np.abs(np.asarray(j1) - np.asarray(j0))) < 1e-13


def test_chapman_enskog_free_slip_equals_mirrored_periodic():
    """The strain estimate at a mirror ghost is the mirror image of the one at
    its source node, so a free-slip box still equals the quarter of the
    mirrored periodic box."""
    L, Lz = 8, 6
    rho, u, pi, phi = inputs.random_smooth_fields(L, L, Lz, seed=12, amp_rho=1e-2, amp_u=2e-2,
                                                   amp_pi=0.0)
    phi = np.tanh(3 * (phi + 0.2))
    small = _sim(L, L, Lz, 1.7, sigma=0.02, gamma=1 / 3.0, faces=(FS, FS, FS, FS, P, P),
                 ce_neq=True)
    small.set_state(rho, u, phi)

    def ext(a):
        return np.concatenate([np.concatenate([a, np.flip(a, -1)], -1),
                               np.flip(np.concatenate([a, np.flip(a, -1)], -1), -2)], -2)

    sx = np.ones((Lz, 2 * L, 2 * L))
    sx[:, :, L:] = -1
    sy = np.ones((Lz, 2 * L, 2 * L))
    sy[:, L:, :] = -1
    U = np.stack([ext(u[0]) * sx, ext(u[1]) * sy, ext(u[2])])
    big = _sim(2 * L, 2 * L, Lz, 1.7, sigma=0.02, gamma=1 / 3.0, ce_neq=True)
    big.set_state(ext(rho), U, ext(phi))
    small.step(12)
    big.step(12)
    a, b = small.moments(), big.moments()
    assert np.max(np.abs(a[0] - b[0][:, :L, :L])) < 1e-14
    for k in range(3):
        assert np.max(np.abs(a[1][k] - b[1][k][:, :L, :L])) < 1e-14
    assert np.max(np.abs(a[3] - b[3][:, :L, :L])) < 1e-13


def test_chapman_enskog_departs_from_projection_at_order_k2():
    """The two closures agree at leading order: a smooth periodic droplet run
    both ways differs by much less than the flow it carries."""
    w = inputs.droplet_workload(24, radius=7.0, sigma=0.01)
    rho, u, phi = w.fields()
    runs = []
    for ce in (False, True):
        s = _sim(24, 24, 24, w.omega, sigma=w.sigma, gamma=1 / w.width, ce_neq=ce)
        s.set_state(rho, u, phi)
        s.step(60)
        runs.append(s.moments())
    du = np.max(np.abs(runs[0][1] - runs[1][1]))
    umax = np.max(np.abs(runs[0][1]))
    assert umax > 0 and du < 0.3 * umax
    assert np.max(np.abs(runs[0][3] - runs[1][3])) < 1e-3
