"""Oracle finite elements: meshes, assembled matrices, residual and Jacobian.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation (Sec. 2 of Farrell & Pearson): continuous piecewise-linear
(P1) elements for both u and w on Omega = (0,1)^d, homogeneous Neumann
conditions (eqn okbcs), theta-method in time.  Every integral is computed
exactly with the simplex monomial rule

    int_T  prod_a lambda_a^{k_a}  dx  =  d! |T| prod_a k_a! / (d + sum_a k_a)!

applied term by term to the polynomial integrand; no quadrature points.

Meshes: n cells per side.  2D squares are cut along their (0,0)-(1,1)
diagonal into two right triangles; 3D cubes are cut into the 6 Kuhn
tetrahedra that share the (0,0,0)-(1,1,1) diagonal.  Vertex (i,j[,k]) has
index i + (n+1) j [+ (n+1)^2 k], x fastest.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# mesh
# --------------------------------------------------------------------------
class Mesh:
    """Uniform simplicial mesh of the unit square or cube (Sec. 4: Omega)."""

    def __init__(self, dim: int, n: int):
        if dim not in (2, 3) or n < 1:
            raise ValueError("dim must be 2 or 3 and n >= 1")
        self.dim, self.n = dim, n
        self.nv = (n + 1) ** dim
        side = np.arange(n + 1, dtype=np.float64) / n
        if dim == 2:
            yy, xx = np.meshgrid(side, side, indexing="ij")
            self.coords = np.stack([xx.ravel(), yy.ravel()], axis=1)
        else:
            zz, yy, xx = np.meshgrid(side, side, side, indexing="ij")
            self.coords = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        self.simplices = self._simplices()
        self._geometry()

    def index(self, *ijk):
        n1 = self.n + 1
        out = 0
        for axis, v in enumerate(ijk):
            out = out + np.asarray(v) * n1 ** axis
        return out

    def _simplices(self) -> np.ndarray:
        n, d = self.n, self.dim
        cells = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"),
                         axis=-1).reshape(-1, d)[:, ::-1]  # columns x, y, (z)

        def corner(offset):
            return self.index(*[cells[:, a] + offset[a] for a in range(d)])

        simp = []
        if d == 2:
            simp.append(np.stack([corner((0, 0)), corner((1, 0)), corner((1, 1))], 1))
            simp.append(np.stack([corner((0, 0)), corner((1, 1)), corner((0, 1))], 1))
        else:
            for perm in itertools.permutations(range(3)):
                path = [np.zeros(3, dtype=int)]
                for axis in perm:
                    nxt = path[-1].copy()
                    nxt[axis] = 1
                    path.append(nxt)
                simp.append(np.stack([corner(tuple(p)) for p in path], 1))
        return np.concatenate(simp, axis=0)

    def _geometry(self):
        d = self.dim
        X = self.coords[self.simplices]                       # (ns, d+1, d)
        A = np.concatenate([np.ones(X.shape[:2] + (1,)), X], axis=2)
        self.volume = np.abs(np.linalg.det(A)) / math.factorial(d)
        C = np.linalg.inv(A)                                  # columns: lambda_a
        self.grad = np.transpose(C[:, 1:, :], (0, 2, 1))      # (ns, d+1, d)


# --------------------------------------------------------------------------
# exact simplex integrals
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def monomial_factor(d: int, idx: tuple) -> float:
    """int_T prod_{a in idx} lambda_a dx / |T| for a tuple of local indices."""
    counts = [idx.count(a) for a in range(d + 1)]
    num = math.factorial(d) * math.prod(math.factorial(k) for k in counts)
    return num / math.factorial(d + sum(counts))


def _assemble(mesh: Mesh, local: np.ndarray) -> sp.csr_matrix:
    """Sum element matrices local[(ns, d+1, d+1)] into a CSR matrix."""
    s = mesh.simplices
    k = s.shape[1]
    rows = np.repeat(s, k, axis=1).ravel()
    cols = np.tile(s, (1, k)).ravel()
    A = sp.coo_matrix((local.ravel(), (rows, cols)), shape=(mesh.nv, mesh.nv))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def _assemble_vector(mesh: Mesh, local: np.ndarray) -> np.ndarray:
    out = np.zeros(mesh.nv)
    np.add.at(out, mesh.simplices.ravel(), local.ravel())
    return out


def mass_matrix(mesh: Mesh) -> sp.csr_matrix:
    """M_ij = int phi_i phi_j (Sec. 2, after eqn newton)."""
    d = mesh.dim
    loc = np.empty((len(mesh.volume), d + 1, d + 1))
    for a in range(d + 1):
        for b in range(d + 1):
            loc[:, a, b] = mesh.volume * monomial_factor(d, (a, b))
    return _assemble(mesh, loc)


def stiffness_matrix(mesh: Mesh) -> sp.csr_matrix:
    """K_ij = int grad phi_i . grad phi_j, the Neumann Laplacian (Sec. 2)."""
    g = mesh.grad
    loc = mesh.volume[:, None, None] * np.einsum("sad,sbd->sab", g, g)
    return _assemble(mesh, loc)


def me_matrix(mesh: Mesh, u: np.ndarray) -> sp.csr_matrix:
    """(M_E)_ij = int (3 u_h^2 - 1) phi_i phi_j for the P1 function u_h (Sec. 2).

    u_h^2 = sum_{c,e} u_c u_e lambda_c lambda_e on each simplex, integrated
    exactly against lambda_a lambda_b.
    """
    d = mesh.dim
    us = u[mesh.simplices]                                    # (ns, d+1)
    vol = mesh.volume
    loc = np.zeros((len(vol), d + 1, d + 1))
    r = range(d + 1)
    for a in r:
        for b in r:
            acc = np.zeros(len(vol))
            for c in r:
                for e in r:
                    acc += 3.0 * us[:, c] * us[:, e] * monomial_factor(d, (a, b, c, e))
            acc -= monomial_factor(d, (a, b))
            loc[:, a, b] = vol * acc
    return _assemble(mesh, loc)


def nonlinear_term(mesh: Mesh, u: np.ndarray) -> np.ndarray:
    """N(u)_i = int (u_h^3 - u_h) phi_i, the weak form of u(u^2-1) in eqn okb."""
    d = mesh.dim
    us = u[mesh.simplices]
    vol = mesh.volume
    loc = np.zeros((len(vol), d + 1))
    r = range(d + 1)
    for a in r:
        acc = np.zeros(len(vol))
        for c in r:
            for e in r:
                for f in r:
                    acc += us[:, c] * us[:, e] * us[:, f] * monomial_factor(d, (a, c, e, f))
        for c in r:
            acc -= us[:, c] * monomial_factor(d, (a, c))
        loc[:, a] = vol * acc
    return _assemble_vector(mesh, loc)


def double_well_integral(mesh: Mesh, u: np.ndarray) -> float:
    """int (1 - u_h^2)^2 dx for the P1 function u_h, exact: on each simplex
    1 - 2 u_h^2 + u_h^4 with u_h = sum_a u_a lambda_a expanded term by term."""
    d = mesh.dim
    us = u[mesh.simplices]
    vol = mesh.volume
    r = range(d + 1)
    sq = np.zeros(len(vol))
    for a in r:
        for b in r:
            sq += us[:, a] * us[:, b] * monomial_factor(d, (a, b))
    qu = np.zeros(len(vol))
    for a in r:
        for b in r:
            for c in r:
                for e in r:
                    qu += us[:, a] * us[:, b] * us[:, c] * us[:, e] * monomial_factor(d, (a, b, c, e))
    return float(np.sum(vol * (1.0 - 2.0 * sq + qu)))


# --------------------------------------------------------------------------
# the discrete Ohta--Kawasaki system
# --------------------------------------------------------------------------
class Params:
    """eps, sigma, m, theta, dt of eqns oka/okb and the theta-method."""

    def __init__(self, eps, sigma, m, theta, dt):
        self.eps, self.sigma, self.m, self.theta, self.dt = (
            float(eps), float(sigma), float(m), float(theta), float(dt))

    @property
    def a11(self) -> float:
        """Scale of the (1,1) block: 1 + dt theta sigma (eqn newton)."""
        return 1.0 + self.dt * self.theta * self.sigma

    @property
    def c(self) -> float:
        """c = dt theta / (1 + dt theta sigma) (after eqn schur)."""
        return self.dt * self.theta / self.a11

    @property
    def gamma(self) -> float:
        """eps sqrt(c), the stiffness weight in S_hat = M + eps sqrt(c) K."""
        return self.eps * math.sqrt(self.c)


class System:
    """Assembled constant matrices of one (mesh, params) pair."""

    def __init__(self, mesh: Mesh, params: Params):
        self.mesh, self.p = mesh, params
        self.M = mass_matrix(mesh)
        self.K = stiffness_matrix(mesh)
        self.one = np.ones(mesh.nv)

    def residual(self, u_n, w_n, u, w) -> np.ndarray:
        """F(u, w) whose Jacobian is J of eqn newton; Newton solves J d = -F.

        F1 = M(u - u_n) + dt theta [K w + sigma M (u - m)]
                        + dt (1 - theta) [K w_n + sigma M (u_n - m)]   (eqn oka)
        F2 = M w - eps^2 K u - N(u)                                     (eqn okb)
        """
        p, M, K = self.p, self.M, self.K
        mvec = p.m * self.one
        F1 = (M @ (u - u_n)
              + p.dt * p.theta * (K @ w + p.sigma * (M @ (u - mvec)))
              + p.dt * (1.0 - p.theta) * (K @ w_n + p.sigma * (M @ (u_n - mvec))))
        F2 = M @ w - p.eps ** 2 * (K @ u) - nonlinear_term(self.mesh, u)
        return np.concatenate([F1, F2])

    def blocks(self, u):
        """A, B, C, D of J = [[A, B], [C, D]] (eqn newton)."""
        p = self.p
        A = p.a11 * self.M
        B = p.dt * p.theta * self.K
        C = -p.eps ** 2 * self.K - me_matrix(self.mesh, u)
        D = self.M
        return A, B, C, D

    def jacobian(self, u) -> sp.csr_matrix:
        A, B, C, D = self.blocks(u)
        return sp.bmat([[A, B], [C, D]], format="csr")

    def s_hat(self) -> sp.csr_matrix:
        """S_hat = M + eps sqrt(c) K (the factor of eqn outer_approx)."""
        return (self.M + self.p.gamma * self.K).tocsr()

    def energy(self, u) -> dict:
        """The Ohta--Kawasaki free energy (Sec. 1) of the P1 function u_h:

            E = 1/2 int ( eps^2 |grad u|^2 + 1/2 (1 - u^2)^2
                          + sigma |(-Delta_N)^{-1/2} (u - m)|^2 ) dx.

        gradient = eps^2/2 u^T K u;  double_well = 1/4 int (1 - u_h^2)^2 (exact);
        nonlocal = sigma/2 (f, phi)_{L2} with f = u - m less its mean (the
        inverse Neumann Laplacian acts on mean-free data) and phi the
        mean-free solution of K phi = M f, solved exactly (sparse LU of K
        bordered by the mean constraint 1^T M phi = 0).
        """
        import scipy.sparse.linalg as spla
        p, M, K = self.p, self.M, self.K
        lm = M @ self.one                                   # 1^T M (lumped masses)
        f = u - p.m
        f = f - (lm @ f) / (lm @ self.one)
        nv = self.mesh.nv
        A = sp.bmat([[K, sp.csr_matrix(lm[:, None])], [sp.csr_matrix(lm[None, :]), None]], format="csc")
        phi = spla.spsolve(A, np.concatenate([M @ f, [0.0]]))[:nv]
        grad = 0.5 * p.eps ** 2 * float(u @ (K @ u))
        well = 0.25 * double_well_integral(self.mesh, u)
        nonl = 0.5 * p.sigma * float(f @ (M @ phi))
        return {"gradient": grad, "double_well": well, "nonlocal": nonl, "total": grad + well + nonl}

    def initial_w(self, u0, solver: str = "lu") -> np.ndarray:
        """w0 from eqn okb: the L2 projection M w0 = eps^2 K u0 + N(u0).

        solver "lu": sparse LU of M; "chebyshev": 80 Jacobi-preconditioned
        Chebyshev steps on the interval [1/2, (d+2)/2] that holds the spectrum
        of diag(M)^{-1} M (error factor below 1e-30, i.e. round-off), for
        grids where the LU's fill makes it slow.
        """
        rhs = self.p.eps ** 2 * (self.K @ u0) + nonlinear_term(self.mesh, u0)
        if solver == "chebyshev":
            from .solvers import chebyshev, mass_interval
            lo, hi = mass_interval(self.mesh.dim)
            return chebyshev(self.M, 1.0 / self.M.diagonal(), rhs, np.zeros_like(rhs), 80, lo, hi)
        import scipy.sparse.linalg as spla
        return spla.spsolve(self.M.tocsc(), rhs)
