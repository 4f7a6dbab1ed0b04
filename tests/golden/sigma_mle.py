"""The FP64 oracle's maximum-likelihood resolution for the sigma-fit data.

The data of the sigma fit: the first N_FIT events of the 2 mm adjoint workload
(seed 4, true sigma_z = 10 mm, sigma_dl = 42 mm), windows of CUT = 5 sigma
rebuilt at every sigma, and the image held at the true phantom rasterised at
the pixel centres, scaled so that sum_l s_l rho_l = N_FIT.  The list-mode
Poisson log-likelihood (the function whose EM step is Eq. iter)
    L(sigma) = sum_j log D_j(sigma) - sum_l s_l rho_l,
    D_j = sum_l P(e_j|l; sigma) s_l rho_l   (Eq. kernel for P),
is maximised over u = (log sigma_z, log sigma_dl) by Newton's method: the
gradient is the oracle's analytic one (dL/du = sigma * dL/dsigma, pinned
against FP64 central differences), the Hessian its central difference with
step H in u.

``python tests/golden/sigma_mle.py [N]`` writes sigma_mle_adjoint_2mm_n<N>.txt
beside this file (N defaults to N_FIT, the sigma fit's event count; the full
1e6-event set gives the estimate with the smaller statistical spread); it
calls only the oracle.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FIT = 100_000
CUT = 5.0
TRUTH = (10.0, 42.0)
H = 1e-3


def golden_path(n_events: int = N_FIT) -> str:
    return os.path.join(HERE, f"sigma_mle_adjoint_2mm_n{n_events}.txt")


def fit_data(n_events: int = N_FIT):
    """(workload, events, rho) of the sigma fit; rho uses the oracle's s."""
    import oracle
    from oracle import Setup
    from synth import make_workload
    w = make_workload("adjoint_2mm", cut=CUT, n_events=n_events)
    ev = w.events()
    s = oracle.sensitivity(Setup.from_workload(w))
    rho = w.phantom().rasterize(w.ny, w.nz, w.R, w.L)
    rho = rho * (w.n_events / float((s * rho).sum()))
    return w, ev, rho


def loglik_and_grad_u(w, ev, rho, u):
    """(L, dL/du) at u = log(sigma), windows of CUT sigma at that sigma."""
    import oracle
    from oracle import Setup
    sz, sl = np.exp(u)
    st = Setup.from_workload(w, sigma_z=float(sz), sigma_dl=float(sl))
    L, _, gs = oracle.loglik_grad(st, ev, rho, want_rho=False)
    return L, np.asarray(gs) * np.array([sz, sl])


def oracle_mle(w, ev, rho, start=TRUTH, tol=1e-7, max_steps=8, central=True,
               final_hessian=True):
    """Newton's method from `start` (the Hessian taken once at the start, by
    central or forward differences; the iteration converges to the zero of
    the analytic gradient either way); returns (sigma_hat, grad_u at it,
    Hessian in u at the start or, with final_hessian, at sigma_hat,
    gradient evaluations)."""
    u = np.log(np.asarray(start, dtype=np.float64))
    evals = 0

    def hessian(u, g0=None):
        nonlocal evals
        Hm = np.zeros((2, 2))
        for k in range(2):
            e = np.zeros(2)
            e[k] = H
            gp = loglik_and_grad_u(w, ev, rho, u + e)[1]
            evals += 1
            if central:
                gm = loglik_and_grad_u(w, ev, rho, u - e)[1]
                evals += 1
                Hm[:, k] = (gp - gm) / (2 * H)
            else:
                Hm[:, k] = (gp - g0) / H
        return 0.5 * (Hm + Hm.T)

    _, g = loglik_and_grad_u(w, ev, rho, u)
    evals += 1
    Hm = hessian(u, g)
    for _ in range(max_steps):
        step = -np.linalg.solve(Hm, g)
        u = u + step
        _, g = loglik_and_grad_u(w, ev, rho, u)
        evals += 1
        if np.max(np.abs(step)) < tol:
            break
    if final_hessian:
        Hm = hessian(u, g)
    return np.exp(u), g, Hm, evals


def read_golden(n_events: int = N_FIT):
    """The stored maximiser: dict with n_events, cut, sigma_z, sigma_dl."""
    out = {}
    with open(golden_path(n_events)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else N_FIT
    w, ev, rho = fit_data(n)
    sig, g, Hm, evals = oracle_mle(w, ev, rho)
    with open(golden_path(n), "w") as f:
        f.write("# Maximum-likelihood (sigma_z, sigma_dl) of the FP64 oracle on the sigma-fit\n"
                "# data (tests/golden/sigma_mle.py: the first n_events events of the 2 mm\n"
                "# adjoint workload, windows of cut sigma, rho = the true phantom).  Written\n"
                "# by that script, which calls only the oracle.\n")
        f.write(f"n_events = {n}\ncut = {CUT}\n")
        f.write(f"sigma_z = {sig[0]:.9f}\nsigma_dl = {sig[1]:.9f}\n")
        f.write(f"# distance from the truth (10, 42) mm: {sig[0] / TRUTH[0] - 1:+.4%}, "
                f"{sig[1] / TRUTH[1] - 1:+.4%}\n")
        f.write(f"# |dL/du| at the maximiser: {np.abs(g).max():.3g}; Hessian eigenvalues "
                f"{np.linalg.eigvalsh(Hm)[0]:.4g}, {np.linalg.eigvalsh(Hm)[1]:.4g}; "
                f"{evals} gradient evaluations\n")
        sd = np.sqrt(np.diag(np.linalg.inv(-Hm)))
        f.write(f"# statistical spread (inverse Hessian): {sd[0]:.4f}, {sd[1]:.4f} in log sigma\n")
    print(sig, g, np.linalg.eigvalsh(Hm), evals)


if __name__ == "__main__":
    main()
