"""Oracle solvers: Chebyshev, multigrid, block preconditioner, FGMRES, Newton.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Farrell & Pearson, Sec. 2-4:
  * Newton on the theta-scheme residual; each step solves J d = -F (eqn newton);
  * right-preconditioned restarted flexible GMRES (Saad, SISC 1993);
  * preconditioner P^{-1} = diag(A~^{-1}, S~^{-1}) [I 0; -C A~^{-1} I] (eqn prec,
    Sec. 3 with A~), S~^{-1} = S_hat^{-1} M S_hat^{-1} (eqn schurinv),
    S_hat = M + eps sqrt(c) K (eqn outer_approx);
  * A~^{-1}: Chebyshev semi-iteration on A = (1 + dt theta sigma) M (Sec. 2-3),
    here Jacobi-preconditioned on the interval [1/2, (d+2)/2] that holds the
    spectrum of diag(M)^{-1} M for P1 simplices;
  * S_hat^{-1}: n_V multigrid V-cycles (Sec. 2 and 4 use algebraic multigrid;
    here read as geometric multigrid on the nested uniform meshes,
    Chebyshev--Jacobi smoothing, linear interpolation, exact coarsest solve);
  * optional k_R = 2: two Richardson steps on S with S~^{-1} (Sec. 4).
Each routine is written in the order of its textbook definition, with no
fusion or reordering, so it can be checked by eye.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Mesh, Params, System, mass_matrix, stiffness_matrix


# --------------------------------------------------------------------------
# Chebyshev semi-iteration (Golub & Varga 1961; Saad, Iterative Methods, 12.3)
# --------------------------------------------------------------------------
def chebyshev(A, dinv, b, x0, steps, lo, hi):
    """`steps` Chebyshev steps for A x = b, preconditioner diag(A)^{-1}.

    For eigenvalues of D^{-1}A in [lo, hi], with centre th = (hi+lo)/2 and
    half-width de = (hi-lo)/2, the error after k steps is
        e_k = T_k((th - D^{-1}A)/de) / T_k(th/de) e_0.
    Three-term form:  r_0 = b - A x_0,  d_0 = D^{-1} r_0 / th,  rho_0 = de/th;
        x_{k+1} = x_k + d_k
        r_{k+1} = r_k - A d_k
        rho_{k+1} = 1 / (2 th/de - rho_k)
        d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / de) D^{-1} r_{k+1}.
    """
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    d = dinv * r / th
    rho = de / th
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        r = r - A @ d
        rho_new = 1.0 / (2.0 * th / de - rho)
        d = rho_new * rho * d + (2.0 * rho_new / de) * (dinv * r)
        rho = rho_new
    return x


def mass_interval(dim: int):
    """Spectrum bounds of diag(M)^{-1} M for P1 simplices: [1/2, (d+2)/2]."""
    return 0.5, 0.5 * (dim + 2)


# --------------------------------------------------------------------------
# geometric multigrid for S_hat = M + gamma K
# --------------------------------------------------------------------------
def level_sizes(n: int, coarse_max: int = 4):
    """n, n/2, ... halving while even and above coarse_max."""
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] > coarse_max:
        sizes.append(sizes[-1] // 2)
    return sizes


def prolongation(dim: int, nc: int) -> sp.csr_matrix:
    """Linear interpolation from the mesh with nc cells to the one with 2 nc.

    Fine vertex 2i + b (b in {0,1}^d) is the midpoint of the coarse edge from
    i to i + b, so its value is (x_i + x_{i+b}) / 2 (x_i itself when b = 0).
    """
    nf = 2 * nc
    n1f, n1c = nf + 1, nc + 1
    fine = np.arange(n1f ** dim)
    f = [(fine // n1f ** a) % n1f for a in range(dim)]      # x, y, (z) of each fine vertex
    i = [fa // 2 for fa in f]
    b = [fa % 2 for fa in f]
    ci = sum(i[a] * n1c ** a for a in range(dim))
    cj = sum((i[a] + b[a]) * n1c ** a for a in range(dim))
    at_coarse = sum(b) == 0
    # at a coarse vertex: weight 1 on x_i; elsewhere 1/2 on x_i and 1/2 on x_{i+b}
    rows = np.concatenate([fine, fine[~at_coarse]])
    cols = np.concatenate([ci, cj[~at_coarse]])
    vals = np.concatenate([np.where(at_coarse, 1.0, 0.5), np.full((~at_coarse).sum(), 0.5)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n1f ** dim, n1c ** dim))


class Multigrid:
    """V-cycles for S_hat = M + gamma K on the nested uniform meshes."""

    def __init__(self, dim, n, gamma, nu_pre=2, nu_post=2, smooth_lo_frac=0.25,
                 coarse_max=4):
        self.dim, self.gamma = dim, gamma
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.hi = 0.5 * (dim + 2)            # Gershgorin bound of D^{-1}(M + gamma K)
        self.lo = smooth_lo_frac * self.hi
        self.sizes = level_sizes(n, coarse_max)
        self.A, self.dinv, self.P = [], [], []
        for nl in self.sizes:
            mesh = Mesh(dim, nl)
            A = (mass_matrix(mesh) + gamma * stiffness_matrix(mesh)).tocsr()
            self.A.append(A)
            self.dinv.append(1.0 / A.diagonal())
        for nl in self.sizes[1:]:
            self.P.append(prolongation(dim, nl))
        # the coarsest level is solved exactly: dense LU when small, sparse LU
        # for the large odd coarse levels of n = c 2^k with c odd and large
        if self.A[-1].shape[0] <= 5000:
            self.coarse, self.coarse_lu = self.A[-1].toarray(), None
        else:
            self.coarse, self.coarse_lu = None, spla.splu(self.A[-1].tocsc())

    def coarse_solve(self, b):
        if self.coarse_lu is not None:
            return self.coarse_lu.solve(b)
        return np.linalg.solve(self.coarse, b)

    def vcycle(self, level, b, x):
        A = self.A[level]
        if level == len(self.sizes) - 1:
            return self.coarse_solve(b)
        x = chebyshev(A, self.dinv[level], b, x, self.nu_pre, self.lo, self.hi)
        r = b - A @ x
        P = self.P[level]
        xc = self.vcycle(level + 1, P.T @ r, np.zeros(P.shape[1]))
        x = x + P @ xc
        x = chebyshev(A, self.dinv[level], b, x, self.nu_post, self.lo, self.hi)
        return x

    def solve(self, b, cycles):
        """`cycles` V-cycles from x = 0 (each one starts from the last iterate)."""
        x = np.zeros_like(b)
        for _ in range(cycles):
            x = self.vcycle(0, b, x)
        return x


# --------------------------------------------------------------------------
# block lower-triangular preconditioner (eqn prec, outer_approx, schurinv)
# --------------------------------------------------------------------------
class Preconditioner:
    """z = P^{-1} v with P = [A~ 0; C S~].

    mode "inexact": A~^{-1} = q_A Chebyshev steps on M divided by (1 + dt theta sigma),
                    S_hat^{-1} = n_V V-cycles;
    mode "exact":   A^{-1} and S_hat^{-1} by sparse LU (the ideal setting of Sec. 3).
    k_R = 1 applies S~^{-1}; k_R = 2 does two Richardson steps on S from zero.
    """

    def __init__(self, system: System, u_k, mode="inexact", q_A=10, n_V=5, k_R=1,
                 nu_pre=2, nu_post=2, smooth_lo_frac=0.25, schur="matching", coarse_max=4):
        self.sys, self.mode = system, mode
        self.q_A, self.n_V, self.k_R = q_A, n_V, k_R
        p, dim = system.p, system.mesh.dim
        self.Ablk, self.Bblk, self.Cblk, _ = system.blocks(u_k)
        self.M = system.M
        self.dinv_M = 1.0 / self.M.diagonal()
        self.lo_M, self.hi_M = mass_interval(dim)
        self.nv = system.mesh.nv
        self.schur = schur
        if mode == "exact":
            self.A_lu = spla.splu(self.Ablk.tocsc())
            self.Shat_lu = spla.splu(system.s_hat().tocsc())
            if schur == "exact":
                S = (self.M - self.Cblk @ spla.spsolve(self.Ablk.tocsc(), self.Bblk.tocsc())).toarray()
                self.S_exact = sla.lu_factor(S)
        else:
            self.mg = Multigrid(dim, system.mesh.n, p.gamma, nu_pre, nu_post, smooth_lo_frac, coarse_max)

    def A_inv(self, r):
        if self.mode == "exact":
            return self.A_lu.solve(r)
        x = chebyshev(self.M, self.dinv_M, r, np.zeros_like(r), self.q_A, self.lo_M, self.hi_M)
        return x / self.sys.p.a11

    def Shat_inv(self, r):
        if self.mode == "exact":
            return self.Shat_lu.solve(r)
        return self.mg.solve(r, self.n_V)

    def S_tilde_inv(self, t):
        """S~^{-1} t = S_hat^{-1} M S_hat^{-1} t (eqn schurinv)."""
        if self.schur == "exact":
            return sla.lu_solve(self.S_exact, t)
        return self.Shat_inv(self.M @ self.Shat_inv(t))

    def S_apply(self, y):
        """S y = D y - C A~^{-1} B y (Schur complement with the A~^{-1} in use)."""
        return self.M @ y - self.Cblk @ self.A_inv(self.Bblk @ y)

    def apply(self, v):
        r1, r2 = v[:self.nv], v[self.nv:]
        y1 = self.A_inv(r1)
        t = r2 - self.Cblk @ y1
        y2 = self.S_tilde_inv(t)
        if self.k_R == 2:
            y2 = y2 + self.S_tilde_inv(t - self.S_apply(y2))
        return np.concatenate([y1, y2])


# --------------------------------------------------------------------------
# right-preconditioned restarted flexible GMRES (Saad 1993)
# --------------------------------------------------------------------------
def fgmres(J_apply, P_apply, f, restart=30, rtol=1e-10, max_its=1000, cycles=None):
    """Solve J x = f from x_0 = 0.  Returns (x, iterations, true rel. residual).

    Arnoldi with modified Gram--Schmidt on w = J z_j, z_j = P^{-1} v_j; the
    iterate is x_0 + Z_m y with y = argmin || beta e_1 - H_m y ||.  Stops when
    that least-squares residual is <= rtol ||f||; at every restart and at exit
    the true residual f - J x is recomputed.

    `cycles`: if a list, every restart cycle of m steps appends a dict with
    its Arnoldi relation J Z_m = V_{m+1} Hbar_m: "H" = Hbar_m ((m+1) x m),
    "V" = [v_0 .. v_m] (v_m absent after a breakdown), "Z" = [z_0 .. z_{m-1}].
    Recording changes no arithmetic.
    """
    fnorm = np.linalg.norm(f)
    x = np.zeros_like(f)
    if fnorm == 0.0:
        return x, 0, 0.0
    r = f.copy()
    beta = fnorm
    its = 0
    while beta > rtol * fnorm and its < max_its:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        y = None
        for j in range(restart):
            z = P_apply(V[j])
            Z.append(z)
            w = J_apply(z)
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            its += 1
            rhs = np.zeros(j + 2)
            rhs[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], rhs, rcond=None)
            est = np.linalg.norm(rhs - H[:j + 2, :j + 1] @ y)
            breakdown = H[j + 1, j] <= 1e-300
            if not breakdown:
                V.append(w / H[j + 1, j])
            if est <= rtol * fnorm or its >= max_its or breakdown:
                break
        if cycles is not None:
            m = len(Z)
            cycles.append({"H": H[:m + 1, :m].copy(), "V": np.column_stack(V), "Z": np.column_stack(Z)})
        x = x + np.column_stack(Z) @ y
        r = f - J_apply(x)
        beta = np.linalg.norm(r)
    return x, its, beta / fnorm


# --------------------------------------------------------------------------
# Newton and the theta-method timestep (Sec. 2, eqn newton)
# --------------------------------------------------------------------------
class Options:
    def __init__(self, restart=30, gmres_rtol=1e-10, max_gmres=1000, q_A=10, n_V=5,
                 k_R=1, nu_pre=2, nu_post=2, newton_atol=1e-10, newton_rtol=0.0,
                 max_newton=25, newton_extra=0, linear="fgmres", prec_mode="inexact", coarse_max=4):
        self.restart, self.gmres_rtol, self.max_gmres = restart, gmres_rtol, max_gmres
        self.q_A, self.n_V, self.k_R = q_A, n_V, k_R
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.newton_atol, self.newton_rtol = newton_atol, newton_rtol
        self.max_newton, self.newton_extra = max_newton, newton_extra
        self.linear, self.prec_mode = linear, prec_mode
        self.coarse_max = coarse_max


def linear_solve(system: System, u_k, rhs, opts: Options):
    """One Newton linear solve J(u_k) d = rhs.  Returns (d, gmres its, rel. res.)."""
    J = system.jacobian(u_k)
    if opts.linear == "direct":
        d = spla.spsolve(J.tocsc(), rhs)
        return d, 0, np.linalg.norm(rhs - J @ d) / max(np.linalg.norm(rhs), 1e-300)
    P = Preconditioner(system, u_k, opts.prec_mode, opts.q_A, opts.n_V, opts.k_R,
                       opts.nu_pre, opts.nu_post, coarse_max=opts.coarse_max)
    return fgmres(lambda z: J @ z, P.apply, rhs, opts.restart, opts.gmres_rtol, opts.max_gmres)


def timestep(system: System, u_n, w_n, opts: Options):
    """Newton from (u_n, w_n) to the theta-scheme solution at the next time.

    Stops when ||F||_2 <= max(newton_atol, newton_rtol ||F_0||_2), then takes
    `newton_extra` further steps.  Returns (u, w, info dict).
    """
    nv = system.mesh.nv
    u, w = u_n.copy(), w_n.copy()
    F = system.residual(u_n, w_n, u, w)
    r0 = np.linalg.norm(F)
    newton, gmres_its, extra = 0, [], 0
    history = [r0]
    converged = False
    while True:
        fn = np.linalg.norm(F)
        if fn <= max(opts.newton_atol, opts.newton_rtol * r0):
            converged = True
            if extra >= opts.newton_extra:
                break
            extra += 1
        if newton >= opts.max_newton:
            break
        d, its, _ = linear_solve(system, u, -F, opts)
        gmres_its.append(its)
        u = u + d[:nv]
        w = w + d[nv:]
        newton += 1
        F = system.residual(u_n, w_n, u, w)
        history.append(np.linalg.norm(F))
    return u, w, dict(newton=newton, gmres=gmres_its, converged=converged,
                      residuals=history)


def make_system(dim, n, eps, sigma, m, theta, dt) -> System:
    return System(Mesh(dim, n), Params(eps, sigma, m, theta, dt))
