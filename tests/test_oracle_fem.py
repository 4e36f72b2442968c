"""Pins for the oracle's finite-element layer (CPU only).

Each test checks the oracle against something other than itself: closed-form
stencils worked out by hand from the P1 element matrices, structural facts
the paper states (Sec. 2: M SPD, K SPSD with the constants as null space,
M_E symmetric), an independent quadrature (collapsed Gauss--Legendre) of the
nonlinear integrals, constant-state reductions and a finite-difference check
of the Jacobian of eqn newton against the residual.
"""
import itertools
import math

import numpy as np
import pytest

from oracle.fem import (Mesh, Params, System, double_well_integral, mass_matrix, me_matrix, nonlinear_term,
                        stiffness_matrix)


def center_index(dim, n):
    c = n // 2
    return sum(c * (n + 1) ** a for a in range(dim))


def offset_index(dim, n, off):
    return sum(off[a] * (n + 1) ** a for a in range(dim))


@pytest.mark.parametrize("dim,n", [(2, 3), (2, 6), (3, 2), (3, 4)])
def test_structure(dim, n):
    mesh = Mesh(dim, n)
    M, K = mass_matrix(mesh), stiffness_matrix(mesh)
    one = np.ones(mesh.nv)
    assert abs(one @ M @ one - 1.0) < 1e-14              # 1^T M 1 = |Omega|
    assert np.abs(K @ one).max() < 1e-13                 # constants span null(K)
    assert abs(M - M.T).max() == 0 and abs(K - K.T).max() == 0
    em = np.linalg.eigvalsh(M.toarray())
    ek = np.linalg.eigvalsh(K.toarray())
    assert em.min() > 0                                  # M SPD
    assert abs(ek[0]) < 1e-12 and ek[1] > 1e-6           # K SPSD, one zero eigenvalue


def test_interior_stencil_2d():
    # Hand-derived from the right-triangle element matrices:
    # K = 5-point [4, -1 x 4]; M = h^2/2 on the diagonal, h^2/12 on +-x, +-y, +-(1,1).
    n = 6
    h = 1.0 / n
    mesh = Mesh(2, n)
    M, K = mass_matrix(mesh).toarray(), stiffness_matrix(mesh).toarray()
    c = center_index(2, n)
    m_exp = {(0, 0): h * h / 2}
    k_exp = {(0, 0): 4.0}
    for off in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        m_exp[off] = h * h / 12
        k_exp[off] = -1.0
    for off in [(1, 1), (-1, -1)]:
        m_exp[off] = h * h / 12
    for off in itertools.product((-1, 0, 1), repeat=2):
        j = c + offset_index(2, n, off)
        assert M[c, j] == pytest.approx(m_exp.get(off, 0.0), abs=1e-16)
        assert K[c, j] == pytest.approx(k_exp.get(off, 0.0), abs=1e-14)
    assert np.count_nonzero(M[c]) == 7 and np.count_nonzero(np.abs(K[c]) > 1e-14) == 5


def test_interior_stencil_3d_kuhn():
    # Kuhn tetrahedra (6 per cube around the main diagonal); counting the
    # tetrahedra on each edge: M = 0.4 h^3 diag, h^3/20 on +-e_i and +-(1,1,1),
    # h^3/30 on +-(e_i + e_j); K = h [6, -1 on +-e_i], zero on the diagonals.
    n = 4
    h = 1.0 / n
    mesh = Mesh(3, n)
    M, K = mass_matrix(mesh).toarray(), stiffness_matrix(mesh).toarray()
    c = center_index(3, n)
    m_exp, k_exp = {(0, 0, 0): 0.4 * h ** 3}, {(0, 0, 0): 6 * h}
    for a in range(3):
        e = [0, 0, 0]
        e[a] = 1
        for s in (1, -1):
            off = tuple(s * x for x in e)
            m_exp[off] = h ** 3 / 20
            k_exp[off] = -h
    for s in (1, -1):
        m_exp[(s, s, s)] = h ** 3 / 20
        for a, b in [(0, 1), (0, 2), (1, 2)]:
            off = [0, 0, 0]
            off[a] = off[b] = s
            m_exp[tuple(off)] = h ** 3 / 30
    for off in itertools.product((-1, 0, 1), repeat=3):
        j = c + offset_index(3, n, off)
        assert M[c, j] == pytest.approx(m_exp.get(off, 0.0), abs=1e-17)
        assert K[c, j] == pytest.approx(k_exp.get(off, 0.0), abs=1e-14)


def test_corner_rows_2d():
    # Vertex (0,0) lies in the two triangles of cell (0,0) only:
    # M_00 = 2 * 2|T|/12 = h^2/6, neighbours (1,0), (0,1): |T|/12 each,
    # (1,1): 2|T|/12; K_00 = 1, K to (1,0) and (0,1) = -1/2, to (1,1) = 0.
    n = 5
    h = 1.0 / n
    mesh = Mesh(2, n)
    M, K = mass_matrix(mesh).toarray(), stiffness_matrix(mesh).toarray()
    T = h * h / 2
    assert M[0, 0] == pytest.approx(h * h / 6, abs=1e-17)
    assert M[0, 1] == pytest.approx(T / 12, abs=1e-17)
    assert M[0, n + 1] == pytest.approx(T / 12, abs=1e-17)
    assert M[0, n + 2] == pytest.approx(2 * T / 12, abs=1e-17)
    assert K[0, 0] == pytest.approx(1.0) and K[0, 1] == pytest.approx(-0.5)
    assert K[0, n + 1] == pytest.approx(-0.5) and abs(K[0, n + 2]) < 1e-15
    # the opposite corner (n,n) lies in one triangle only (the upper one of cell n-1,n-1... both)
    last = mesh.nv - 1
    assert M[last].sum() == pytest.approx(one_cell_share(h), abs=1e-17)


def one_cell_share(h):
    # corner (n,n) touches both triangles of its cell: row sum = int phi = 2 * |T|/3
    return 2 * (h * h / 2) / 3


# --------------------------------------------------------------------------
# independent quadrature: collapsed (Duffy) Gauss--Legendre on the reference simplex
# --------------------------------------------------------------------------
def duffy_rule(dim, q=6):
    g, w = np.polynomial.legendre.leggauss(q)
    g, w = 0.5 * (g + 1), 0.5 * w
    pts, wts = [], []
    if dim == 2:
        for s, ws in zip(g, w):
            for t, wt in zip(g, w):
                pts.append((s, t * (1 - s)))
                wts.append(ws * wt * (1 - s))
    else:
        for s, ws in zip(g, w):
            for t, wt in zip(g, w):
                for r, wr in zip(g, w):
                    pts.append((s, t * (1 - s), r * (1 - s) * (1 - t)))
                    wts.append(ws * wt * wr * (1 - s) ** 2 * (1 - t))
    pts = np.array(pts)
    lam = np.concatenate([1 - pts.sum(1, keepdims=True), pts], axis=1)   # barycentrics
    return lam, np.array(wts)          # weights sum to the reference volume 1/d!


@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_nonlinear_integrals_vs_quadrature(dim, n):
    rng = np.random.default_rng(7)
    mesh = Mesh(dim, n)
    u = rng.uniform(-1.2, 1.2, mesh.nv)
    lam, wts = duffy_rule(dim)
    ME = np.zeros((mesh.nv, mesh.nv))
    N = np.zeros(mesh.nv)
    Mq = np.zeros((mesh.nv, mesh.nv))
    for s, vol in zip(mesh.simplices, mesh.volume):
        uh = lam @ u[s]
        scale = math.factorial(dim) * vol
        for a in range(dim + 1):
            N[s[a]] += scale * np.sum(wts * (uh ** 3 - uh) * lam[:, a])
            for b in range(dim + 1):
                ME[s[a], s[b]] += scale * np.sum(wts * (3 * uh ** 2 - 1) * lam[:, a] * lam[:, b])
                Mq[s[a], s[b]] += scale * np.sum(wts * lam[:, a] * lam[:, b])
    assert np.abs(me_matrix(mesh, u).toarray() - ME).max() < 1e-15
    assert np.abs(nonlinear_term(mesh, u) - N).max() < 1e-15
    assert np.abs(mass_matrix(mesh).toarray() - Mq).max() < 1e-16
    assert abs(me_matrix(mesh, u) - me_matrix(mesh, u).T).max() < 1e-18   # M_E symmetric


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_constant_state_reductions(dim, n):
    mesh = Mesh(dim, n)
    M = mass_matrix(mesh)
    a = -0.37
    u = np.full(mesh.nv, a)
    assert np.abs(me_matrix(mesh, u) - (3 * a * a - 1) * M).max() < 1e-17
    assert np.abs(nonlinear_term(mesh, u) - (a ** 3 - a) * (M @ np.ones(mesh.nv))).max() < 1e-17


@pytest.mark.parametrize("dim,n,theta", [(2, 5, 1.0), (2, 4, 0.5), (3, 3, 0.5)])
def test_jacobian_is_derivative_of_residual(dim, n, theta):
    rng = np.random.default_rng(3)
    sysm = System(Mesh(dim, n), Params(0.05, 80.0, 0.1, theta, 3e-3))
    nv = sysm.mesh.nv
    u_n, w_n = rng.uniform(-1, 1, nv), rng.uniform(-1, 1, nv)
    u, w = rng.uniform(-1, 1, nv), rng.uniform(-1, 1, nv)
    v = rng.standard_normal(2 * nv)
    J = sysm.jacobian(u)
    eps = 1e-4
    Fp = sysm.residual(u_n, w_n, u + eps * v[:nv], w + eps * v[nv:])
    Fm = sysm.residual(u_n, w_n, u - eps * v[:nv], w - eps * v[nv:])
    fd = (Fp - Fm) / (2 * eps)
    assert np.linalg.norm(J @ v - fd) <= 1e-7 * np.linalg.norm(fd)


def test_initial_w_solves_okb():
    rng = np.random.default_rng(11)
    sysm = System(Mesh(2, 6), Params(0.04, 100.0, 0.0, 1.0, 1e-4))
    u0 = rng.uniform(-0.5, 0.5, sysm.mesh.nv)
    w0 = sysm.initial_w(u0)
    F = sysm.residual(u0, w0, u0, w0)
    assert np.linalg.norm(F[sysm.mesh.nv:]) < 1e-15
    a = 0.25                                   # constant state: w0 = a^3 - a
    w_c = sysm.initial_w(np.full(sysm.mesh.nv, a))
    assert np.abs(w_c - (a ** 3 - a)).max() < 1e-14


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 4)])
def test_initial_w_chebyshev_equals_lu(dim, n):
    """Both solvers of the okb projection reach the same w0 (to round-off)."""
    sysm = System(Mesh(dim, n), Params(0.05, 50.0, 0.1, 0.5, 1e-3))
    u0 = 0.1 + 0.5 * np.random.default_rng(4).uniform(-1, 1, sysm.mesh.nv)
    a, b = sysm.initial_w(u0), sysm.initial_w(u0, solver="chebyshev")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


# --------------------------------------------------------------------------
# the Ohta--Kawasaki energy (Sec. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_double_well_integral_vs_quadrature(dim, n):
    """int (1 - u_h^2)^2 against the independent collapsed Gauss--Legendre rule
    (exact for the degree-4 integrand)."""
    u = np.random.default_rng(8).uniform(-1.3, 1.3, Mesh(dim, n).nv)
    mesh = Mesh(dim, n)
    lam, wts = duffy_rule(dim)
    ref = 0.0
    for s, vol in zip(mesh.simplices, mesh.volume):
        uh = lam @ u[s]
        ref += math.factorial(dim) * vol * np.sum(wts * (1 - uh ** 2) ** 2)
    assert abs(double_well_integral(mesh, u) - ref) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_energy_of_constant_state(dim, n):
    """u = c: no gradient, f = u - m is constant so its mean-free part vanishes,
    and the double well integrates to (1 - c^2)^2 |Omega| / 4 with |Omega| = 1."""
    c = 0.3
    sysm = System(Mesh(dim, n), Params(0.05, 70.0, -0.2, 0.5, 1e-3))
    E = sysm.energy(np.full(sysm.mesh.nv, c))
    assert abs(E["gradient"]) < 1e-15 and abs(E["nonlocal"]) < 1e-14
    assert abs(E["double_well"] - 0.25 * (1 - c * c) ** 2) < 1e-15


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_energy_of_a_discrete_eigenmode(dim, n):
    """u = m + a v with K v = lam M v (so 1^T M v = 0 for lam > 0): the inverse
    Neumann Laplacian of a v is a v / lam, so
        gradient = eps^2/2 a^2 lam v^T M v,   nonlocal = sigma/2 a^2 v^T M v / lam,
    closed forms that do not go through the oracle's bordered solve."""
    import scipy.linalg as sla
    eps, sigma, m, a = 0.06, 120.0, 0.15, 0.4
    sysm = System(Mesh(dim, n), Params(eps, sigma, m, 0.5, 1e-3))
    lam, Q = sla.eigh(sysm.K.toarray(), sysm.M.toarray())
    for k in (1, 3, len(lam) // 2):
        v = Q[:, k]
        vMv = v @ (sysm.M @ v)
        E = sysm.energy(m + a * v)
        assert abs(E["gradient"] - 0.5 * eps ** 2 * a * a * lam[k] * vMv) <= 1e-12 * E["gradient"]
        assert abs(E["nonlocal"] - 0.5 * sigma * a * a * vMv / lam[k]) <= 1e-10 * E["nonlocal"]


def test_energy_decreases_along_implicit_timesteps():
    """The Ohta--Kawasaki equation is the H^{-1} gradient flow of E (Sec. 1);
    with theta = 1 and a small step the discrete energy decreases every step
    (the 32^2 workload's parameters, a larger initial perturbation)."""
    from oracle.solvers import Options, timestep
    rng = np.random.default_rng(12)
    sysm = System(Mesh(2, 16), Params(0.04, 100.0, 0.0, 1.0, 1e-4))
    u = 0.3 * rng.uniform(-1, 1, sysm.mesh.nv)
    w = sysm.initial_w(u)
    prev = sysm.energy(u)["total"]
    for _ in range(4):
        u, w, info = timestep(sysm, u, w, Options(linear="direct", newton_atol=1e-12, newton_extra=1))
        e = sysm.energy(u)["total"]
        assert info["converged"] and e < prev
        prev = e
