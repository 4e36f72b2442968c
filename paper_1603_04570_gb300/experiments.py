"""Iteration counts of the paper's Sec. 4 experiments on this solver.

Sec. 4 reports the average number of outer Krylov iterations per Newton step
(Table 1: the mesh refined at fixed parameters; Table 2: eps -> 0 with
dx = eps / 2 and dt = eps^2).  Flat counts are the preconditioner's claim.
This module runs the same experiments through the library:

    python -m paper_1603_04570_gb300.experiments table1 [--sizes 50 100 200 400] [--steps 3]
    python -m paper_1603_04570_gb300.experiments table2 [--sizes 100 200 400] [--steps 3]
    python -m paper_1603_04570_gb300.experiments refine2d [--sizes 128 256 512 1024] [--steps 2]
    python -m paper_1603_04570_gb300.experiments spectrum [--workloads 2d_n1024 3d_n128] [--steps 2]
    python -m paper_1603_04570_gb300.experiments energy [--workloads 2d_n1024 3d_n128] [--steps 5]

`energy` monitors the Ohta--Kawasaki free energy (Sec. 1) along the
trajectory: its interfacial, double-well and nonlocal terms after each
timestep (ok_energy), with the mean of u; the equations are the H^{-1}
gradient flow of that energy, so it decreases while the mean relaxes to m.

`spectrum` estimates eig(J P^{-1}) (Sec. 3: 1 and eig(S~^{-1} S)) at full
size from the Arnoldi matrix of FGMRES cycles: after each timestep, the Ritz
values of the step's last Newton solve, and of one solve of a seeded random
right-hand side at the new state, against Lemma 2's interval enclosed with
l_- >= -1 and l_+ <= 3 max u^2 - 1 (the range of 3 u_h^2 - 1, which bounds
eig(M^{-1} M_E)).  k_R = 1, so the Schur approximation is the one the lemmas
are about.

Paper setting (Table 1): unit cube, m = 0.4, eps = 0.02, sigma = 100,
theta = 0.5, dt = eps^2, u0 = m + cos(2 pi x) cos(2 pi y) cos(2 pi z) / 50,
ten Chebyshev steps for A~^{-1}, two Richardson steps of S~^{-1} (k_R = 2),
five V-cycles per S_hat^{-1}.  The paper does not state its Krylov and Newton
tolerances; its solver (FEniCS over PETSc) defaults to a relative Krylov
tolerance of 1e-5 and a relative Newton tolerance of 1e-8, which these runs
use unless --gmres-rtol is given.  Meshes: the paper's own, n = 50 2^k cells
per side (Table 1: 50, 100, 200, 400; the 800 row needs about 1e9 DoF, more
than one GPU holds with FGMRES(30)); Table 2 takes dx = eps / 2, i.e.
n = 2 / eps = 100, 200, 400 for eps = 0.02, 0.01, 0.005.  The geometric
hierarchy halves n while it is even, down to the 26^3 level of n = 25,
which is solved by Chebyshev iteration to round-off (it is too large for the
dense inverse).  Each line printed is a JSON record; --markdown prints a
table.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import ok_inputs as oi

from . import OK_FP64, OK_MIXED, Grid


def run(wl: oi.Workload, steps: int, k_R: int = 2, precision: int = OK_MIXED, gmres_rtol: float = 1e-5,
        newton_rtol: float = 1e-8, **opts) -> dict:
    """`steps` timesteps of workload `wl`; FGMRES and Newton counts."""
    import torch
    o = dict(restart=wl.restart, gmres_rtol=gmres_rtol, newton_atol=1e-300, newton_rtol=newton_rtol,
             precision=precision, k_R=k_R, q_A=10, n_V=5)
    o.update(opts)
    with Grid(wl.dim, wl.n, wl.eps, wl.sigma, wl.m, wl.theta, wl.dt, **o) as g:
        u = torch.from_numpy(oi.initial_u(wl)).cuda()
        w = torch.empty_like(u)
        g.init_w(u, w)
        torch.cuda.synchronize()
        its = newton = 0
        per_step = []
        t0 = time.perf_counter()
        for _ in range(steps):
            info = g.timestep(u, w)
            its += info.gmres_its
            newton += info.newton_its
            per_step.append(info.gmres_its / max(info.newton_its, 1))
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
    return dict(workload=wl.name, dim=wl.dim, n=wl.n, dofs=wl.dofs, eps=wl.eps, dt=wl.dt, steps=steps,
                k_R=k_R, precision="fp64" if precision == OK_FP64 else "mixed", gmres_rtol=gmres_rtol,
                newton_steps=newton, gmres_its=its, its_per_newton=its / max(newton, 1),
                its_per_newton_by_step=per_step, seconds=seconds)


def table1(sizes, steps, k_R, **kw):
    for n in sizes:
        yield run(oi.scaled(oi.PAPER_3D, n), steps, k_R, **kw)


def table2(steps, k_R, ns=(100, 200, 400), **kw):
    # dx = eps / 2: eps = 2 / n, dt = eps^2
    for n in ns:
        eps = 2.0 / n
        yield run(oi.scaled(oi.PAPER_3D, n, eps=eps, dt=eps * eps), steps, k_R, **kw)


def refine2d(sizes, steps, k_R, **kw):
    for n in sizes:
        wl = dataclasses.replace(oi.scaled(oi.LARGE_2D, n))
        yield run(wl, steps, k_R, coarse_max=32 if n >= 128 else 4, **kw)


def _ritz_record(g, wl, u, label, its):
    import numpy as np
    ritz = g.ritz_values()
    c = wl.dt * wl.theta / (1 + wl.dt * wl.theta * wl.sigma)
    lp = max(3.0 * float((u * u).max()) - 1.0, 0.0)
    lo, hi = 0.5 - c ** 0.5 / (2 * wl.eps), 1.0 + c ** 0.5 * lp / (2 * wl.eps)
    re = np.sort(ritz.real)
    return dict(solve=label, gmres_its=its, ritz_count=len(ritz), ritz_re_min=float(re[0]), ritz_re_max=float(re[-1]),
                ritz_im_max=float(np.abs(ritz.imag).max()), dist_to_1=float(np.abs(ritz - 1.0).min()),
                lemma2_lo=lo, lemma2_hi=hi, outside=int(np.sum((ritz.real < lo) | (ritz.real >= hi))),
                smallest=[round(float(x), 5) for x in re[:4]], largest=[round(float(x), 5) for x in re[-3:]])


def spectrum(names, steps, precision=OK_MIXED, restart=60):
    """Ritz values of eig(J P^{-1}) after each of `steps` timesteps."""
    import numpy as np
    import torch
    for name in names:
        wl = oi.PAPER_3D if name == "paper_3d" else oi.WORKLOADS[name]
        if name == "paper_3d":
            wl = oi.scaled(wl, 128)
        o = dict(restart=restart, gmres_rtol=wl.gmres_rtol, k_R=1, precision=precision,
                 newton_atol=wl.newton_tols[0], newton_rtol=wl.newton_tols[1])
        if wl.dim == 2 and wl.n >= 128:
            o["coarse_max"] = 32
        with Grid(wl.dim, wl.n, wl.eps, wl.sigma, wl.m, wl.theta, wl.dt, **o) as g:
            u = torch.from_numpy(oi.initial_u(wl)).cuda()
            w = torch.empty_like(u)
            g.init_w(u, w)
            f = torch.from_numpy(np.random.default_rng(7).standard_normal(wl.dofs)).cuda()
            x = torch.empty_like(f)
            for step in range(1, steps + 1):
                info = g.timestep(u, w)
                rec = dict(workload=wl.name, dofs=wl.dofs, step=step, newton_steps=info.newton_its,
                           precision="fp64" if precision == OK_FP64 else "mixed")
                yield {**rec, **_ritz_record(g, wl, u, "newton", info.last_gmres_its)}
                si = g.solve_linear(u, f, x, check=False)
                yield {**rec, **_ritz_record(g, wl, u, "random_rhs", si.gmres_its)}


def energy(names, steps, precision=OK_MIXED):
    """The energy's three terms after each of `steps` timesteps."""
    import torch
    for name in names:
        wl = oi.WORKLOADS[name]
        o = dict(restart=wl.restart, gmres_rtol=wl.gmres_rtol, precision=precision,
                 newton_atol=wl.newton_tols[0], newton_rtol=wl.newton_tols[1])
        if wl.dim == 2 and wl.n >= 128:
            o["coarse_max"] = 32
        with Grid(wl.dim, wl.n, wl.eps, wl.sigma, wl.m, wl.theta, wl.dt, **o) as g:
            u = torch.from_numpy(oi.initial_u(wl)).cuda()
            w = torch.empty_like(u)
            g.init_w(u, w)
            for step in range(steps + 1):
                if step:
                    g.timestep(u, w)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                terms, total = g.energy(u)
                yield {"workload": wl.name, "dofs": wl.dofs, "step": step, "t": step * wl.dt, "energy": total,
                       "interfacial": terms[0], "double_well": terms[1], "nonlocal": terms[2],
                       "mean_u": float(u.mean()), "energy_ms": 1e3 * (time.perf_counter() - t0)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("experiment", choices=["table1", "table2", "refine2d", "spectrum", "energy"])
    ap.add_argument("--workloads", nargs="*", default=None, help="spectrum: 2d_n1024, 3d_n128, paper_3d, ...")
    ap.add_argument("--sizes", type=int, nargs="*", default=None)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--k-r", type=int, default=None, help="1: S~^{-1}; 2: two Richardson steps (paper)")
    ap.add_argument("--gmres-rtol", type=float, default=1e-5)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--markdown", action="store_true")
    a = ap.parse_args(argv)
    prec = OK_FP64 if a.fp64 else OK_MIXED
    if a.experiment == "table1":
        rows = table1(a.sizes or [50, 100, 200, 400], a.steps, a.k_r or 2, precision=prec, gmres_rtol=a.gmres_rtol)
    elif a.experiment == "table2":
        rows = table2(a.steps, a.k_r or 2, ns=tuple(a.sizes or (100, 200, 400)), precision=prec,
                      gmres_rtol=a.gmres_rtol)
    elif a.experiment == "spectrum":
        rows = spectrum(a.workloads or ["2d_n1024", "paper_3d"], a.steps, precision=prec)
    elif a.experiment == "energy":
        rows = energy(a.workloads or ["2d_n1024", "3d_n128"], a.steps, precision=prec)
    else:
        rows = refine2d(a.sizes or [128, 256, 512, 1024], a.steps, a.k_r or 1, precision=prec,
                        gmres_rtol=a.gmres_rtol)
    out = []
    for r in rows:
        out.append(r)
        print(json.dumps(r), flush=True)
    if a.markdown and a.experiment == "energy":
        print("\n| workload | step | t | E | interfacial | double well | nonlocal | mean u | ok_energy ms |")
        print("|---|---|---|---|---|---|---|---|---|")
        for r in out:
            print(f"| {r['workload']} | {r['step']} | {r['t']:.2e} | {r['energy']:.9e} | {r['interfacial']:.6e} | "
                  f"{r['double_well']:.9e} | {r['nonlocal']:.6e} | {r['mean_u']:.9f} | {r['energy_ms']:.1f} |")
    elif a.markdown and a.experiment == "spectrum":
        print("\n| workload | step | solve | FGMRES its | Ritz Re min | Ritz Re max | max |Im| | dist to 1 | "
              "Lemma 2 enclosure | outside |")
        print("|---|---|---|---|---|---|---|---|---|---|")
        for r in out:
            print(f"| {r['workload']} | {r['step']} | {r['solve']} | {r['gmres_its']} | {r['ritz_re_min']:.4f} | "
                  f"{r['ritz_re_max']:.4f} | {r['ritz_im_max']:.2e} | {r['dist_to_1']:.1e} | "
                  f"[{r['lemma2_lo']:.4f}, {r['lemma2_hi']:.4f}) | {r['outside']} |")
    elif a.markdown:
        print("\n| n | DoF | eps | dt | k_R | rtol | Newton steps | FGMRES its | its / Newton |")
        print("|---|---|---|---|---|---|---|---|---|")
        for r in out:
            print(f"| {r['n']} | {r['dofs']:,} | {r['eps']:.4g} | {r['dt']:.3g} | {r['k_R']} | {r['gmres_rtol']:g} | "
                  f"{r['newton_steps']} | {r['gmres_its']} | {r['its_per_newton']:.2f} |")


if __name__ == "__main__":
    main()
