"""Pins for the oracle's LSP (Algorithms 1 and 2) and ADMM-TV.

* The LSP's CG reaches the solution of the dense normal equations of its
  quadratic (built column by column from the operator).
* Algorithm 1 (space domain) and Algorithm 2 (frequency domain after
  cancelling F_2D F*_2D) give the same iterates up to rounding.
* The LSP quadratic decreases at every inner CG step.
* ADMM-TV converges to the minimiser of 1/2 ||L u - d||^2 + alpha TV(u)
  found by an independent quasi-Newton solve of the smoothed objective.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import admm, lamino, tv
from oracle.lamino import Geometry

n1, n0, n2, h, w, T = 8, 4, 8, 8, 8, 8
N = n1 * n0 * n2


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(30)
    g = Geometry(n1=n1, n0=n0, n2=n2, h=h, w=w, theta=np.arange(T) * 2 * np.pi / T,
                 phi=np.deg2rad(30.0))
    A = np.stack([lamino.lhat(e.reshape(n1, n0, n2), g).ravel() for e in np.eye(N)], axis=1)
    D = np.zeros((3 * N, N))
    idx = np.arange(N).reshape(n1, n0, n2)
    for a in range(3):
        for i in np.ndindex((n1, n0, n2)):
            if i[a] + 1 < (n1, n0, n2)[a]:
                j = list(i)
                j[a] += 1
                D[a * N + idx[i], idx[tuple(j)]] += 1.0
                D[a * N + idx[i], idx[i]] -= 1.0
    u_true = rng.uniform(0, 1, (n1, n0, n2))
    d = lamino.lam_forward(u_true, g) + 0.01 * rng.standard_normal((T, h, w))
    psi = 0.1 * rng.standard_normal((3, n1, n0, n2))
    lam = 0.1 * rng.standard_normal((3, n1, n0, n2))
    return dict(g=g, A=A, D=D, d=d, psi=psi, lam=lam)


def _lsp_quadratic(t, u, rho):
    hw = h * w
    r = t["A"] @ u.ravel() - lamino.f_2d(t["d"]).ravel()
    gv = (t["psi"] - t["lam"] / rho).ravel()
    q = t["D"] @ u.ravel() - gv
    return 0.5 * np.vdot(r, r).real / hw + 0.5 * rho * q @ q


def test_lsp_cg_reaches_normal_equation_solution(tiny):
    rho = 0.5
    A, D = tiny["A"], tiny["D"]
    hw = h * w
    gv = (tiny["psi"] - tiny["lam"] / rho).ravel()
    H = (A.conj().T @ A).real / hw + rho * D.T @ D
    b = (A.conj().T @ lamino.f_2d(tiny["d"]).ravel()).real / hw + rho * D.T @ gv
    u_star = np.linalg.solve(H, b)
    u = admm.lsp(np.zeros((n1, n0, n2)), tiny["d"], tiny["psi"], tiny["lam"], rho, tiny["g"], 100)
    assert np.linalg.norm(u.ravel() - u_star) <= 1e-10 * np.linalg.norm(u_star)


def test_lsp_quadratic_decreases_every_inner_step(tiny):
    rho = 0.5
    vals = [_lsp_quadratic(tiny, np.zeros((n1, n0, n2)), rho)]
    for k in range(1, 7):
        u = admm.lsp(np.zeros((n1, n0, n2)), tiny["d"], tiny["psi"], tiny["lam"], rho, tiny["g"], k)
        vals.append(_lsp_quadratic(tiny, u, rho))
    assert all(b < a for a, b in zip(vals, vals[1:]))


def test_algorithm1_equals_algorithm2(tiny):
    u0 = np.random.default_rng(31).standard_normal((n1, n0, n2))
    a = admm.lsp(u0, tiny["d"], tiny["psi"], tiny["lam"], 0.7, tiny["g"], 4, form="alg1")
    b = admm.lsp(u0, tiny["d"], tiny["psi"], tiny["lam"], 0.7, tiny["g"], 4, form="alg2")
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)
    ua, _ = admm.admm(tiny["d"], tiny["g"], 0.02, 0.5, 3, 4, form="alg1")
    ub, _ = admm.admm(tiny["d"], tiny["g"], 0.02, 0.5, 3, 4, form="alg2")
    assert np.linalg.norm(ua - ub) <= 1e-11 * np.linalg.norm(ub)


def test_admm_reaches_tv_minimiser(tiny):
    alpha, eps = 0.02, 1e-6
    g, d, D = tiny["g"], tiny["d"], tiny["D"]

    def f(x):
        u = x.reshape(n1, n0, n2)
        r = lamino.lam_forward(u, g) - d
        gu = (D @ x).reshape(3, -1)
        mag = np.sqrt((gu ** 2).sum(0) + eps ** 2)
        grad = lamino.lam_adjoint(r, g).ravel() + alpha * (D.T @ (gu / mag).ravel())
        return 0.5 * np.vdot(r, r).real + alpha * mag.sum(), grad

    ref = minimize(f, np.zeros(N), jac=True, method="L-BFGS-B",
                   options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    u, info = admm.admm(d, g, alpha, 0.5, 60, 4)
    assert abs(info["objective"][-1] - ref.fun) <= 2e-6 * ref.fun
    assert np.linalg.norm(u.ravel() - ref.x) <= 2e-3 * np.linalg.norm(ref.x)
    # the reported objective is the one of Eq. 1
    r = lamino.lam_forward(u, g) - d
    assert info["objective"][-1] == pytest.approx(0.5 * np.vdot(r, r).real + alpha * tv.tv(u), rel=1e-12)


def test_admm_fixed_rho_objective_non_increasing(tiny):
    _, info = admm.admm(tiny["d"], tiny["g"], 0.02, 0.5, 20, 4, adapt_rho=False)
    ob = np.array(info["objective"])
    assert np.all(np.diff(ob) <= 1e-6 * ob[0])
    assert info["rho"] == [0.5] * 20


def test_penalty_rule_balances_residuals(tiny):
    _, info = admm.admm(tiny["d"], tiny["g"], 0.02, 64.0, 6, 4)
    # a large rho makes the dual residual dominate, so rho must fall
    assert info["rho_final"] < 64.0
    for k in range(5):
        r, s, rho, nxt = info["r"][k], info["s"][k], info["rho"][k], info["rho"][k + 1]
        assert nxt == (2 * rho if r > 10 * s else 0.5 * rho if s > 10 * r else rho)


def test_objective_gradient_matches_finite_differences():
    # P7: the gradient Re L^H (L u - d) + alpha * (-div(grad u / |grad u|_eps)) of
    # 1/2 ||L u - d||^2 + alpha TV_eps(u) against central differences (also a
    # check of L^H against L)
    from paper_2511_01893_b300 import inputs
    n = 16
    g = Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=inputs.angles(12), phi=np.deg2rad(20.0))
    u0 = inputs.ellipsoid_phantom(n, n, 12, seed=1236).numpy()
    d = lamino.lam_forward(u0, g)
    u = 0.5 * u0 + 0.1 * np.random.default_rng(1).standard_normal(u0.shape)
    alpha, eps = 1e-2, 0.1

    def f(x):
        r = lamino.lam_forward(x, g) - d
        gg = tv.grad(x)
        return 0.5 * np.vdot(r, r).real + alpha * np.sum(np.sqrt((gg * gg).sum(0) + eps * eps))

    r = lamino.lam_forward(u, g) - d
    gg = tv.grad(u)
    G = lamino.lam_adjoint(r, g) + alpha * (-tv.div(gg / np.sqrt((gg * gg).sum(0) + eps * eps)))
    v = np.random.default_rng(2).standard_normal(u.shape)
    h = 1e-4
    fd = (f(u + h * v) - f(u - h * v)) / (2 * h)
    assert abs(fd - np.vdot(G, v)) <= 1e-9 * np.linalg.norm(G) * np.linalg.norm(v)
