"""Pins for the oracle's solvers (CPU only).

Checks against closed forms and the paper's statements:
  * the Chebyshev iterate equals the closed-form error polynomial
    T_k((th - lambda)/de)/T_k(th/de) applied through an eigendecomposition;
  * diag(M)^{-1} M has its spectrum in [1/2, (d+2)/2] (element bound);
  * linear interpolation is exact on linears and the coarse operators are the
    Galerkin products P^T A_f P;
  * a V-cycle equals its error-propagation operator built from dense
    smoother polynomials and exact coarse corrections;
  * with exact A^{-1} and S^{-1}, GMRES converges in two iterations (Sec. 2);
  * eig(S~^{-1} S) are real (Lemma 1) and obey Lemma 2's bounds for SPD K;
  * the preconditioned operator has eigenvalues {1} and eig(S~^{-1} S) (Sec. 3);
  * [A 0; C S~] applied to the exact-mode preconditioner output returns v;
  * FGMRES agrees with dense LU of J (Sec. 2, eqn newton);
  * a timestep keeps the mean law (u_bar - m)(1 + dt th sig) = (u_bar_n - m)(1 - dt (1-th) sig)
    and maps a constant state to its closed form;
  * a small discrete eigenmode K v = lam M v is multiplied per timestep by the
    theta-method's amplification factor (1 - (1-th) dt mu)/(1 + th dt mu),
    mu = lam (eps^2 lam - 1) + sig, which pins the explicit (1 - theta) part of
    the residual (invisible to the mean law and the constant state, since K 1 = 0).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fem import Mesh, Params, System, mass_matrix, me_matrix, stiffness_matrix
from oracle.solvers import (Multigrid, Options, Preconditioner, chebyshev, fgmres, level_sizes,
                            mass_interval, prolongation, timestep)


def cheb_poly(k, t):
    return np.polynomial.chebyshev.Chebyshev.basis(k)(t)


def cheb_error_matrix(A, k, lo, hi):
    """Dense p_k(D^{-1}A) with p_k(l) = T_k((th-l)/de)/T_k(th/de)."""
    d = A.diagonal()
    Dh = np.sqrt(d)
    B = (A / Dh[:, None]) / Dh[None, :]
    lam, Q = np.linalg.eigh(B)
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    p = cheb_poly(k, (th - lam) / de) / cheb_poly(k, th / de)
    return (Q * p) @ Q.T / Dh[:, None] * Dh[None, :]


@pytest.mark.parametrize("dim,n,k", [(2, 5, 1), (2, 5, 4), (2, 6, 10), (3, 3, 7)])
def test_chebyshev_matches_polynomial(dim, n, k):
    rng = np.random.default_rng(k)
    mesh = Mesh(dim, n)
    A = (mass_matrix(mesh) + 0.02 * stiffness_matrix(mesh)).toarray()
    lo, hi = 0.3, 0.5 * (dim + 2)
    xs = rng.standard_normal(mesh.nv)
    x0 = rng.standard_normal(mesh.nv)
    b = A @ xs
    x = chebyshev(A, 1.0 / A.diagonal(), b, x0, k, lo, hi)
    E = cheb_error_matrix(A, k, lo, hi)
    assert np.linalg.norm((x - xs) - E @ (x0 - xs)) <= 1e-12 * np.linalg.norm(x0 - xs)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_mass_jacobi_interval(dim, n):
    M = mass_matrix(Mesh(dim, n)).toarray()
    lam = sla.eigh(M, np.diag(M.diagonal()), eigvals_only=True)
    lo, hi = mass_interval(dim)
    assert lam.min() >= lo - 1e-12 and lam.max() <= hi + 1e-12
    assert lam.max() > 0.8 * hi            # the bound is nearly attained


@pytest.mark.parametrize("dim,nc", [(2, 3), (2, 4), (3, 2)])
def test_prolongation(dim, nc):
    P = prolongation(dim, nc)
    fine, coarse = Mesh(dim, 2 * nc), Mesh(dim, nc)
    rng = np.random.default_rng(1)
    coef = rng.standard_normal(dim + 1)
    lin = lambda X: coef[0] + X @ coef[1:]
    assert np.abs(P @ lin(coarse.coords) - lin(fine.coords)).max() < 1e-14
    for asm in (mass_matrix, stiffness_matrix):
        Af, Ac = asm(fine), asm(coarse)
        assert np.abs((P.T @ Af @ P - Ac).toarray()).max() < 1e-14 * max(1, abs(Ac).max())


def vcycle_error_operator(mg, level):
    A = mg.A[level].toarray()
    if level == len(mg.sizes) - 1:
        return np.zeros_like(A)
    Spre = cheb_error_matrix(A, mg.nu_pre, mg.lo, mg.hi)
    Spost = cheb_error_matrix(A, mg.nu_post, mg.lo, mg.hi)
    P = mg.P[level].toarray()
    Ac = mg.A[level + 1].toarray()
    Ec = vcycle_error_operator(mg, level + 1)
    Bc = (np.eye(len(Ac)) - Ec) @ np.linalg.inv(Ac)     # one coarse V-cycle from zero
    return Spost @ (np.eye(len(A)) - P @ Bc @ P.T @ A) @ Spre


@pytest.mark.parametrize("dim,n,gamma,cycles", [(2, 16, 4e-3, 1), (2, 16, 4e-3, 3), (3, 8, 1e-2, 2)])
def test_vcycle_error_propagation(dim, n, gamma, cycles):
    mg = Multigrid(dim, n, gamma)
    assert len(mg.sizes) >= 2
    E = vcycle_error_operator(mg, 0)
    A = mg.A[0].toarray()
    rng = np.random.default_rng(2)
    b = rng.standard_normal(len(A))
    xs = np.linalg.solve(A, b)
    x = mg.solve(b, cycles)
    e = -xs
    for _ in range(cycles):
        e = E @ e
    assert np.linalg.norm((x - xs) - e) <= 1e-11 * np.linalg.norm(xs)
    assert np.linalg.norm(x - xs) <= 0.2 ** cycles * np.linalg.norm(xs)


def test_level_sizes():
    assert level_sizes(1024) == [1024, 512, 256, 128, 64, 32, 16, 8, 4]     # 9 levels
    assert level_sizes(32) == [32, 16, 8, 4]
    assert level_sizes(96) == [96, 48, 24, 12, 6, 3]
    assert level_sizes(17) == [17]


def small_system(dim=2, n=6, seed=0, amp=0.9, **kw):
    rng = np.random.default_rng(seed)
    p = dict(eps=0.04, sigma=100.0, m=0.0, theta=1.0, dt=1e-3)
    p.update(kw)
    sysm = System(Mesh(dim, n), Params(**p))
    u = rng.uniform(-amp, amp, sysm.mesh.nv)
    return sysm, u, rng


def test_exact_preconditioner_two_iterations():
    sysm, u, rng = small_system()
    J = sysm.jacobian(u)
    P = Preconditioner(sysm, u, mode="exact", schur="exact")
    f = rng.standard_normal(2 * sysm.mesh.nv)
    x, its, rel = fgmres(lambda z: J @ z, P.apply, f, restart=30, rtol=1e-10)
    assert its == 2 and rel < 1e-10


def dense_schur(sysm, u, tau=0.0):
    M = sysm.M.toarray()
    K = sysm.K.toarray() + tau * M
    ME = me_matrix(sysm.mesh, u).toarray()
    p = sysm.p
    Mi = np.linalg.inv(M)
    S = M + p.eps ** 2 * p.c * K @ Mi @ K + p.c * ME @ Mi @ K
    Sh = M + p.eps * np.sqrt(p.c) * K
    St = Sh @ Mi @ Sh
    return M, K, ME, S, St


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_lemmas_1_and_2(dim, n):
    sysm, u, _ = small_system(dim, n, seed=4, amp=1.0, dt=2e-3)
    p = sysm.p
    M, K, ME, S, St = dense_schur(sysm, u)
    # eqn schurapprox: S~ = M + eps^2 c K M^-1 K + 2 eps sqrt(c) K
    Mi = np.linalg.inv(M)
    assert np.abs(St - (M + p.eps ** 2 * p.c * K @ Mi @ K + 2 * p.eps * np.sqrt(p.c) * K)).max() < 1e-13
    lam = np.linalg.eigvals(np.linalg.solve(St, S))
    assert np.abs(lam.imag).max() < 1e-8                          # Lemma 1
    # Lemma 2 with K perturbed to SPD
    M, K, ME, S, St = dense_schur(sysm, u, tau=1e-6)
    lam = np.linalg.eigvals(np.linalg.solve(St, S)).real
    mu = sla.eigh(ME, M, eigvals_only=True)
    lm, lp = min(mu.min(), 0.0), max(mu.max(), 0.0)
    lo = 0.5 + np.sqrt(p.c) * lm / (2 * p.eps)
    hi = 1.0 + np.sqrt(p.c) * lp / (2 * p.eps)
    assert lm < 0 < lp                                            # both signs exercised
    assert lam.min() >= lo - 1e-10 and lam.max() < hi


def test_block_preconditioned_spectrum():
    sysm, u, _ = small_system(2, 4, seed=5, dt=2e-3)
    nv = sysm.mesh.nv
    A, B, C, D = (x.toarray() for x in sysm.blocks(u))
    _, _, _, S, St = dense_schur(sysm, u)
    J = np.block([[A, B], [C, D]])
    Pm = np.block([[A, np.zeros_like(B)], [C, St]])
    lam = np.sort_complex(np.linalg.eigvals(np.linalg.solve(Pm, J)))
    expect = np.sort_complex(np.concatenate([np.ones(nv), np.linalg.eigvals(np.linalg.solve(St, S))]))
    assert np.abs(lam - expect).max() < 1e-8


@pytest.mark.parametrize("mode,k_R", [("inexact", 1), ("inexact", 2), ("exact", 1)])
def test_fgmres_records_its_arnoldi_decomposition(mode, k_R):
    """The recorded cycle is the (unique) Arnoldi decomposition of J P^{-1}
    from v_0 = f / ||f||: Z = P^{-1} V, V orthonormal, Hbar upper Hessenberg
    with positive subdiagonal and J Z = V Hbar; these conditions determine
    Hbar (implicit Q theorem).  Restart 4 gives several cycles."""
    sysm, u, rng = small_system(2, 6, seed=11, dt=2e-3)
    J = sysm.jacobian(u)
    P = Preconditioner(sysm, u, mode=mode, k_R=k_R)
    f = rng.standard_normal(2 * sysm.mesh.nv)
    for restart in (4, 30):
        cycles = []
        x, its, rel = fgmres(lambda z: J @ z, P.apply, f, restart=restart, rtol=1e-8, cycles=cycles)
        assert sum(c["H"].shape[1] for c in cycles) == its
        assert len(cycles) == (1 if restart == 30 else -(-its // restart))
        c = cycles[0]
        H, V, Z = c["H"], c["V"], c["Z"]
        m = H.shape[1]
        assert H.shape == (m + 1, m) and V.shape[1] == m + 1 and Z.shape[1] == m
        assert np.abs(V[:, 0] - f / np.linalg.norm(f)).max() < 1e-15
        assert np.abs(V.T @ V - np.eye(m + 1)).max() < 1e-6         # MGS: O(eps cond) loss
        for j in range(m):
            assert np.array_equal(Z[:, j], P.apply(V[:, j]))
        assert np.all(np.tril(H, -2) == 0) and np.all(np.diag(H, -1) > 0)
        assert np.abs(J @ Z - V @ H).max() < 1e-12 * np.abs(J @ Z).max()


def test_ritz_values_recover_the_schur_spectrum():
    """Sec. 3: eig(J P^{-1}) = {1} and eig(S~^{-1} S) for exact A^{-1} and
    S~^{-1}.  Once the Krylov space is invariant the Ritz values of the cycle
    contain every eigenvalue of S~^{-1} S (real: Lemma 1)."""
    sysm, u, rng = small_system(2, 3, seed=3, amp=1.0, dt=2e-3)
    J = sysm.jacobian(u)
    P = Preconditioner(sysm, u, mode="exact")
    f = rng.standard_normal(2 * sysm.mesh.nv)
    cycles = []
    fgmres(lambda z: J @ z, P.apply, f, restart=63, rtol=1e-15, max_its=63, cycles=cycles)
    H = cycles[0]["H"]
    m = H.shape[1]
    ritz = np.linalg.eigvals(H[:m, :m])
    _, _, _, S, St = dense_schur(sysm, u)
    lam = np.linalg.eigvals(np.linalg.solve(St, S))
    assert np.abs(lam.imag).max() < 1e-8
    assert max(np.abs(ritz - l).min() for l in lam.real) < 1e-9


@pytest.mark.parametrize("k_R", [1, 2])
def test_exact_mode_preconditioner_inverts_block_triangle(k_R):
    sysm, u, rng = small_system(2, 5, seed=6, dt=2e-3)
    nv = sysm.mesh.nv
    A, B, C, D = (x.toarray() for x in sysm.blocks(u))
    _, _, _, S, St = dense_schur(sysm, u)
    v = rng.standard_normal(2 * nv)
    z = Preconditioner(sysm, u, mode="exact", k_R=k_R).apply(v)
    z1, z2 = z[:nv], z[nv:]
    assert np.allclose(A @ z1, v[:nv], rtol=0, atol=1e-12 * np.abs(v).max())
    if k_R == 1:
        assert np.allclose(C @ z1 + St @ z2, v[nv:], rtol=0, atol=1e-11 * np.abs(v).max())
    else:
        # two Richardson steps on S z2 = t from zero: z2 = (2 S~^-1 - S~^-1 S S~^-1) t
        t = v[nv:] - C @ z1
        Sti = np.linalg.inv(St)
        assert np.allclose(z2, (2 * Sti - Sti @ S @ Sti) @ t, rtol=0, atol=1e-9 * np.abs(z2).max())


def test_inexact_preconditioner_structure():
    sysm, u, rng = small_system(2, 8, seed=8, dt=2e-3)
    nv = sysm.mesh.nv
    P = Preconditioner(sysm, u, mode="inexact", q_A=10, n_V=2)
    v = rng.standard_normal(2 * nv)
    z = P.apply(v)
    M = sysm.M.toarray()
    Ainv = (np.eye(nv) - cheb_error_matrix(M, 10, 0.5, 2.0)) @ np.linalg.inv(M) / sysm.p.a11
    E = vcycle_error_operator(P.mg, 0)
    Sh = P.mg.A[0].toarray()
    Shinv = (np.eye(nv) - E @ E) @ np.linalg.inv(Sh)
    C = P.Cblk.toarray()
    z1 = Ainv @ v[:nv]
    z2 = Shinv @ M @ Shinv @ (v[nv:] - C @ z1)
    assert np.allclose(z, np.concatenate([z1, z2]), rtol=0, atol=1e-10 * np.abs(z).max())


def test_fgmres_matches_dense_lu_17():
    sysm, u, rng = small_system(2, 16, seed=9, amp=0.8, dt=1e-4)
    J = sysm.jacobian(u)
    f = rng.standard_normal(2 * sysm.mesh.nv)
    xd = np.linalg.solve(J.toarray(), f)
    P = Preconditioner(sysm, u, mode="inexact")
    x, its, rel = fgmres(lambda z: J @ z, P.apply, f, restart=30, rtol=1e-12)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    # restarted (short restart) reaches the same answer
    x2, its2, rel2 = fgmres(lambda z: J @ z, P.apply, f, restart=4, rtol=1e-12)
    assert its2 >= its and np.linalg.norm(x2 - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("dim,n,theta", [(2, 8, 0.5), (2, 8, 1.0), (3, 4, 0.5)])
def test_timestep_mean_law(dim, n, theta):
    rng = np.random.default_rng(10)
    p = Params(0.05, 150.0, 0.2, theta, 5e-4)
    sysm = System(Mesh(dim, n), p)
    u0 = 0.2 + 0.3 * rng.uniform(-1, 1, sysm.mesh.nv)
    w0 = sysm.initial_w(u0)
    opts = Options(restart=30, gmres_rtol=1e-12, newton_atol=1e-14, newton_extra=1)
    u1, w1, info = timestep(sysm, u0, w0, opts)
    assert info["converged"]
    ubar = lambda x: np.ones(sysm.mesh.nv) @ (sysm.M @ x)
    lhs = (ubar(u1) - p.m) * (1 + p.dt * p.theta * p.sigma)
    rhs = (ubar(u0) - p.m) * (1 - p.dt * (1 - p.theta) * p.sigma)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_timestep_constant_state():
    p = Params(0.03, 200.0, -0.1, 0.5, 1e-3)
    sysm = System(Mesh(2, 6), p)
    a = 0.35
    u0 = np.full(sysm.mesh.nv, a)
    w0 = sysm.initial_w(u0)
    opts = Options(gmres_rtol=1e-12, newton_atol=1e-16, newton_extra=1)
    u1, w1, info = timestep(sysm, u0, w0, opts)
    r = (1 - p.dt * (1 - p.theta) * p.sigma) / (1 + p.dt * p.theta * p.sigma)
    assert np.abs(u1 - (p.m + (a - p.m) * r)).max() < 1e-13
    assert np.abs(w1 - (u1 ** 3 - u1)).max() < 1e-13


def test_timestep_matches_direct_newton():
    import ok_inputs as oi
    wl = oi.SMALL_2D
    sysm = System(Mesh(wl.dim, wl.n), Params(wl.eps, wl.sigma, wl.m, wl.theta, wl.dt))
    u0 = oi.initial_u(wl)
    w0 = sysm.initial_w(u0)
    a = timestep(sysm, u0, w0, Options(gmres_rtol=1e-10, newton_atol=1e-10, newton_extra=1))
    b = timestep(sysm, u0, w0, Options(linear="direct", newton_atol=1e-10, newton_extra=1))
    for x, y in zip(a[:2], b[:2]):
        assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


# --------------------------------------------------------------------------
# the theta-method's explicit part (Sec. 2: theta-method in time for eqn oka)
# --------------------------------------------------------------------------
def _generalised_mode(sysm, target):
    """A discrete eigenpair K v = lam M v (dense, tiny grids) with lam near `target`."""
    lam, Q = sla.eigh(sysm.K.toarray(), sysm.M.toarray())
    k = int(np.argmin(np.abs(lam - target)))
    v = Q[:, k]
    return lam[k], v / np.abs(v).max()


@pytest.mark.parametrize("dim,n,theta", [(2, 6, 0.5), (2, 6, 1.0), (2, 6, 0.3), (3, 3, 0.5)])
def test_timestep_amplifies_an_eigenmode_by_the_theta_method_factor(dim, n, theta):
    """Small-amplitude eigenmode through two whole timesteps.

    For m = 0 and |u| << 1, N(u) = -M u + O(|u|^3), so with K v = lam M v the
    semi-discrete system reduces on span{v} to the scalar ODE a' = -mu a with
    w = (eps^2 lam - 1) a and mu = lam (eps^2 lam - 1) + sigma.  The
    theta-method maps a_n to R a_n with the textbook amplification factor
        R = (1 - (1 - theta) dt mu) / (1 + theta dt mu).
    Both the implicit and the explicit (weight 1 - theta) parts of eqn oka
    enter R; a dropped or sign-flipped K w_n or sigma M (u_n - m) term in the
    residual changes it by O(dt lam b) or O(dt sigma), far above the O(a^2)
    linearisation error checked here.
    """
    eps, sigma, dt = 0.2, 10.0, 1e-3
    sysm = System(Mesh(dim, n), Params(eps, sigma, 0.0, theta, dt))
    lam, v = _generalised_mode(sysm, 120.0)
    mu = lam * (eps ** 2 * lam - 1.0) + sigma
    R = (1.0 - (1.0 - theta) * dt * mu) / (1.0 + theta * dt * mu)
    assert abs(R) > 0.05 and abs(R - 1.0) > 0.05          # the step visibly changes the mode
    a0 = 1e-5
    u, w = a0 * v, (eps ** 2 * lam - 1.0) * a0 * v
    opts = Options(linear="direct", newton_atol=0.0, newton_rtol=1e-11, newton_extra=1)
    a = a0
    for _ in range(2):
        u, w, info = timestep(sysm, u, w, opts)
        assert info["converged"]
        a = R * a
        assert np.linalg.norm(u - a * v) <= 1e-7 * abs(a) * np.linalg.norm(v)
        assert np.linalg.norm(w - (eps ** 2 * lam - 1.0) * a * v) <= 1e-7 * abs(a) * np.linalg.norm(v)


@pytest.mark.parametrize("theta", [0.25, 0.5, 1.0])
def test_residual_at_the_previous_state_is_the_full_explicit_step(theta):
    """At (u, w) = (u_n, w_n) the theta weights add up to one, so for every
    theta  F1 = dt [K w_n + sigma M (u_n - m)]  and  F2 = M w_n - eps^2 K u_n - N(u_n)."""
    rng = np.random.default_rng(21)
    p = Params(0.07, 40.0, 0.15, theta, 3e-3)
    sysm = System(Mesh(2, 5), p)
    nv = sysm.mesh.nv
    un, wn = rng.uniform(-1, 1, nv), rng.uniform(-1, 1, nv)
    F = sysm.residual(un, wn, un, wn)
    ref_theta1 = System(Mesh(2, 5), Params(p.eps, p.sigma, p.m, 1.0, p.dt)).residual(un, wn, un, wn)
    assert np.abs(F - ref_theta1).max() <= 1e-14 * np.abs(F).max()
    # and the theta = 1 value is independent of (u_n, w_n) beyond the M (u - u_n) term:
    ua, wa = rng.uniform(-1, 1, nv), rng.uniform(-1, 1, nv)
    F1 = System(Mesh(2, 5), Params(p.eps, p.sigma, p.m, 1.0, p.dt)).residual(ua, wa, un, wn)[:nv]
    assert np.abs(F1 - (F[:nv] + sysm.M @ (un - ua))).max() <= 1e-14 * np.abs(F1).max()


def test_large_coarse_level_is_solved_exactly():
    """A coarsest level above 5000 unknowns (2D n = 150 -> 75: 76^2) is solved by
    sparse LU: the coarse solve satisfies S_hat x = b to round-off, like the
    dense solve of the small coarse levels."""
    mg = Multigrid(2, 150, 3e-3, coarse_max=4)
    assert mg.sizes == [150, 75] and mg.coarse_lu is not None
    b = np.random.default_rng(5).standard_normal(76 * 76)
    x = mg.coarse_solve(b)
    A = mg.A[-1]
    assert np.abs(A @ x - b).max() <= 1e-13 * (abs(A) @ np.abs(x)).max()      # backward error
    assert np.abs(A @ x - b).max() <= 1e-9 * np.abs(b).max()
    small = Multigrid(2, 16, 3e-3, coarse_max=4)
    xs = small.coarse_solve(b[:25])
    assert np.linalg.norm(small.A[-1] @ xs - b[:25]) <= 1e-12 * np.linalg.norm(b[:25])
