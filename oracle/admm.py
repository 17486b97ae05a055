"""ADMM-TV with the LSP of Algorithm 1 and of Algorithm 2, FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Problem (Eq. 1): min_u 1/2 ||L u - d||^2 + alpha ||u||_TV, split with the
constraint grad u = psi (Section 2, "ADMM").  One outer iteration runs the
four phases the paper names: LSP (u update), RSP (psi update), the update of
the multiplier lambda, and the update of the penalty rho (with the residuals
r and s).

Readings (the paper gives the step order, not the rules):

* LSP objective: 1/2 ||L u - d||^2 + rho/2 ||grad u - g||^2 with
  g = psi - lambda / rho (first line of Algorithms 1 and 2).  Its gradient is
  G = Re L^H (L u - d) - rho div(grad u - g); "-rho nabla(g' - g)" in the
  listings is read as -rho div(g' - g) with g' = grad u.
* CG(u, G, G_prev): nonlinear CG with the Dai-Yuan direction
  beta = ||G||^2 / <p, G - G_prev> (restarted at p = -G on the first inner
  step, as G_prev <- 0 in the listings) and an exact line search on the
  quadratic, gamma = -<G, p> / (||L p||^2 + rho ||grad p||^2).
* Algorithm 2 works in the frequency domain: d_hat = F_2D d once, residual
  d_hat' - d_hat with d_hat' = L_hat u, and data weight 1/(h w) so that,
  by Parseval (F_2D F*_2D = I, Section 4.2), every quantity equals
  Algorithm 1's.
* RSP: psi = shrink_iso(grad u + lambda / rho, alpha / rho).
* lambda <- lambda + rho (grad u - psi).
* Penalty (residual balancing, mu = 10, factor 2): r = ||grad u - psi||,
  s = rho ||div(psi - psi_old)||; rho doubles if r > 10 s, halves if
  s > 10 r.  lambda is unscaled, so it needs no rescaling.
"""

from __future__ import annotations

import numpy as np

from . import lamino, tv


def _dot(a, b) -> float:
    return float(np.vdot(a, b).real)


def lsp(u, d, psi, lam, rho, geom, n_inner, form="alg2", dhat=None):
    """One LSP solve.  ``form`` = "alg1" (space domain, Algorithm 1) or
    "alg2" (frequency domain after operation cancellation, Algorithm 2)."""
    g = psi - lam / rho
    G_prev = None
    p = None
    hw = geom.h * geom.w
    if form == "alg2" and dhat is None:
        dhat = lamino.f_2d(d)
    for i in range(n_inner):
        # forward pass
        if form == "alg1":
            resid = lamino.lam_forward(u, geom) - d
        else:
            resid = lamino.lhat(u, geom) - dhat
        g1 = tv.grad(u)
        # adjoint pass
        if form == "alg1":
            data_grad = lamino.lam_adjoint(resid, geom)
        else:
            data_grad = lamino.lhat_adj(resid, geom) / hw
        G = data_grad - rho * tv.div(g1 - g)
        # CG update
        if i == 0:
            p = -G
        else:
            beta = _dot(G, G) / _dot(p, G - G_prev)
            p = -G + beta * p
        if form == "alg1":
            Lp = lamino.lam_forward(p, geom)
            Lp2 = _dot(Lp, Lp)
        else:
            Lp = lamino.lhat(p, geom)
            Lp2 = _dot(Lp, Lp) / hw
        gp = tv.grad(p)
        gamma = -_dot(G, p) / (Lp2 + rho * _dot(gp, gp))
        u = u + gamma * p
        G_prev = G
    return u


def objective(u, d, geom, alpha) -> float:
    r = lamino.lam_forward(u, geom) - d
    return 0.5 * _dot(r, r) + alpha * tv.tv(u)


def admm(d, geom, alpha, rho, n_outer, n_inner=4, adapt_rho=True, form="alg2", u0=None,
         callback=None):
    """ADMM-TV from u = 0, psi = lambda = 0.  Returns (u, info) where info
    holds per-outer-iteration objective, rho (before its update), r, s."""
    shape = (geom.n1, geom.n0, geom.n2)
    u = np.zeros(shape) if u0 is None else np.array(u0, dtype=np.float64)
    psi = np.zeros((3,) + shape)
    lam = np.zeros((3,) + shape)
    dhat = lamino.f_2d(d) if form == "alg2" else None
    info = {"objective": [], "rho": [], "r": [], "s": []}
    for k in range(n_outer):
        info["rho"].append(rho)
        u = lsp(u, d, psi, lam, rho, geom, n_inner, form=form, dhat=dhat)
        gu = tv.grad(u)
        psi_old = psi
        psi = tv.shrink_iso(gu + lam / rho, alpha / rho)
        lam = lam + rho * (gu - psi)
        r = float(np.linalg.norm((gu - psi).ravel()))
        s = rho * float(np.linalg.norm(tv.div(psi - psi_old).ravel()))
        info["r"].append(r)
        info["s"].append(s)
        if adapt_rho:
            if r > 10.0 * s:
                rho *= 2.0
            elif s > 10.0 * r:
                rho *= 0.5
        info["objective"].append(objective(u, d, geom, alpha))
        if callback is not None:
            callback(k, u, psi, lam, rho)
    info["rho_final"] = rho
    return u, info
