"""Pins for oracle.pcg (Algorithm 1, Section 3)."""

import numpy as np
import pytest

from oracle import pcg, sketch


def _spd(m, cond, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    ev = np.geomspace(1.0, cond, m)
    return (U * ev) @ U.T, ev


def test_cg_iterates_minimise_energy_error_over_krylov_space():
    # definition of CG: z^j = argmin over K_j(B, rhs) of ||z - z*||_B
    m = 12
    B, _ = _spd(m, 50.0, seed=1)
    rhs = np.random.default_rng(2).standard_normal(m)
    zstar = np.linalg.solve(B, rhs)
    for t in range(1, 8):
        tr = pcg.cg(lambda z: B @ z, rhs, t)
        K = np.column_stack([np.linalg.matrix_power(B, i) @ rhs for i in range(t)])
        Qk, _ = np.linalg.qr(K)
        coef = np.linalg.solve(Qk.T @ B @ Qk, Qk.T @ rhs)
        zk = Qk @ coef
        assert np.allclose(tr.z, zk, rtol=1e-8, atol=1e-10 * np.linalg.norm(zstar))


def test_cg_reaches_exact_solution():
    # m steps in exact arithmetic; a few more in floating point
    m = 10
    B, _ = _spd(m, 30.0, seed=3)
    rhs = np.random.default_rng(4).standard_normal(m)
    tr = pcg.cg(lambda z: B @ z, rhs, 2 * m, tol=1e-13 * np.linalg.norm(rhs))
    assert tr.iterations <= m + 3
    assert np.allclose(tr.z, np.linalg.solve(B, rhs), rtol=1e-10)


def test_chebyshev_residual_is_scaled_chebyshev_polynomial():
    # r^t = T_t((theta - B)/delta) r^0 / T_t(theta/delta), checked in B's eigenbasis
    m = 9
    B, ev = _spd(m, 20.0, seed=5)
    lo, hi = 0.9, 22.0
    rhs = np.random.default_rng(6).standard_normal(m)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    w, U = np.linalg.eigh(B)
    for t in range(0, 7):
        tr = pcg.chebyshev(lambda z: B @ z, rhs, lo, hi, t)
        Tt = np.cos(t * np.arccos(np.clip((theta - w) / delta, -1, 1)))
        Tden = np.cosh(t * np.arccosh(theta / delta))
        expect = U @ ((Tt / Tden) * (U.T @ rhs))
        r = rhs - B @ tr.z
        assert np.allclose(r, expect, atol=1e-10 * np.linalg.norm(rhs))


@pytest.mark.parametrize("kappa", [1.5, 3.0, 10.0])
def test_chebyshev_bound_eq_cs(kappa):
    m = 40
    B, ev = _spd(m, kappa, seed=7)
    rhs = np.random.default_rng(8).standard_normal(m)
    tr = pcg.chebyshev(lambda z: B @ z, rhs, ev[0], ev[-1], 15)
    for t, r in enumerate(tr.res_norms):
        assert r <= pcg.chebyshev_bound(kappa, t) * tr.res_norms[0] * (1 + 1e-9)


def test_chebyshev_bound_closed_form_values():
    # U = (2+zeta)/(2-zeta) with zeta = 1/2 gives U = 5/3; eq. cs2 chain: bound <= zeta^t
    U = 5.0 / 3.0
    for t in range(1, 10):
        assert pcg.chebyshev_bound(U, t) <= 0.5 ** t
    assert pcg.chebyshev_bound(4.0, 1) == pytest.approx(2.0 / (3.0 + 1.0 / 3.0))


def test_preconditioner_whitens_q():
    rng = np.random.default_rng(9)
    m, w = 6, 40
    ADW = rng.standard_normal((m, w)) * np.geomspace(1, 1e3, m)[:, None]
    pre = pcg.preconditioner(ADW)
    Q = ADW @ ADW.T
    assert np.allclose(pre.Q_mhalf @ Q @ pre.Q_mhalf, np.eye(m), atol=1e-9)
    assert np.allclose(pre.Q_mhalf, pre.Q_mhalf.T)
    assert np.allclose(pre.Q_inv, np.linalg.inv(Q), rtol=1e-8)


def test_identity_sketch_makes_cg_one_step():
    # w = n, W = I: Q = A D^2 A^T, B = I, CG converges in one iteration
    rng = np.random.default_rng(10)
    m, n = 5, 30
    A = rng.standard_normal((m, n))
    d = rng.uniform(0.1, 10, n)
    pre = pcg.preconditioner(A * d)
    M = (A * d * d) @ A.T
    Bmat = pre.Q_mhalf @ M @ pre.Q_mhalf
    assert np.allclose(Bmat, np.eye(m), atol=1e-10)
    p = rng.standard_normal(m)
    tr = pcg.cg(lambda z: Bmat @ z, pre.Q_mhalf @ p, 5, tol=1e-12 * np.linalg.norm(p))
    assert tr.iterations == 1
    assert np.allclose(pre.Q_mhalf @ tr.z, np.linalg.solve(M, p), rtol=1e-9)


def _band_case(m, n, w, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    d = np.exp(rng.uniform(-3, 3, n))
    W = sketch.gaussian_matrix(seed, 0, 0, n, w)
    pre = pcg.preconditioner((A * d) @ W)
    sv = np.linalg.svd(pre.Q_mhalf @ (A * d), compute_uv=False)
    return A, d, pre, sv


def test_lemma_3_1_band_at_large_w():
    # zeta = 1/2: (1 + zeta/2)^-1 <= sigma_i^2(Q^{-1/2} A D) <= (1 - zeta/2)^-1
    zeta = 0.5
    _, _, _, sv = _band_case(m=6, n=3000, w=1200, seed=11)
    assert sv.min() ** 2 >= 1.0 / (1.0 + zeta / 2)
    assert sv.max() ** 2 <= 1.0 / (1.0 - zeta / 2)


def test_marchenko_pastur_edges_at_w_4m():
    # sigma_i(Q^{-1/2} A D) = 1/sigma_i(V^T W); V^T W is m x w Gaussian with
    # N(0,1/w) entries, whose singular values fill 1 +- sqrt(m/w)
    m, w = 64, 256
    _, _, _, sv = _band_case(m=m, n=3000, w=w, seed=12)
    r = np.sqrt(m / w)
    inv = 1.0 / sv
    assert inv.min() > (1 - r) * 0.85 and inv.max() < (1 + r) * 1.1
    assert inv.min() < (1 - r) * 1.25 and inv.max() > (1 + r) * 0.9


def test_cg_residual_monotone_with_contraction_eq_rec():
    # Lemma 3.2 with Lemma 3.1: ||f^(j)|| <= (kappa^2 - 1)/2 ||f^(j-1)||
    m, n, w = 6, 3000, 1200
    A, d, pre, sv = _band_case(m, n, w, seed=13)
    kappa2 = (sv.max() / sv.min()) ** 2
    assert kappa2 < 3.0
    M = (A * d * d) @ A.T
    Bmat = pre.Q_mhalf @ M @ pre.Q_mhalf
    p = np.random.default_rng(14).standard_normal(m)
    tr = pcg.cg(lambda z: Bmat @ z, pre.Q_mhalf @ p, 5)
    rates = np.array(tr.res_norms[1:]) / np.array(tr.res_norms[:-1])
    assert (rates <= (kappa2 - 1) / 2 + 1e-12).all()
    # and the zeta form of eq. rec for zeta = 1/2
    assert (rates <= pcg.cg_contraction(0.5) + 1e-12).all()


@pytest.mark.parametrize("zeta", [0.1, 0.5, 0.9])
def test_contraction_is_lemma_3_2_rate_at_the_lemma_3_1_band_edges(zeta):
    # Lemma 3.1's band [(1 + zeta/2)^-1, (1 - zeta/2)^-1] for the squared
    # singular values gives kappa^2 = (1 + zeta/2)/(1 - zeta/2), and Lemma
    # 3.2's rate (kappa^2 - 1)/2 at that kappa is the eq. rec contraction
    kappa2 = (1.0 / (1.0 - zeta / 2)) / (1.0 / (1.0 + zeta / 2))
    assert pcg.cg_contraction(zeta) == pytest.approx((kappa2 - 1) / 2, rel=1e-14)
    assert pcg.cg_contraction(zeta) < 1.0


def test_theory_tolerance_and_iteration_count():
    n, gamma, sigma = 1000, 0.9, 0.5
    mu = 0.3
    tol = pcg.theory_inner_tol(mu, n, gamma, sigma)
    # sqrt(3 n mu) * tol = gamma sigma mu / 4
    assert np.sqrt(3 * n * mu) * tol == pytest.approx(gamma * sigma * mu / 4)
    t = pcg.inner_iteration_count(n, gamma, sigma)
    psi = 4 * np.sqrt(6) * (1 + sigma / np.sqrt(1 - gamma)) / (gamma * sigma)
    # Lemma 4.4: sqrt(6) n zeta^t (1 + sigma/sqrt(1-gamma)) <= gamma sigma / 4
    assert np.sqrt(6) * n * 0.5 ** t * (1 + sigma / np.sqrt(1 - gamma)) <= gamma * sigma / 4
    assert np.sqrt(6) * n * 0.5 ** (t - 1) * (1 + sigma / np.sqrt(1 - gamma)) > gamma * sigma / 4
    assert t == int(np.ceil(np.log(n * psi) / np.log(2)))


def test_lanczos_interval_recovers_the_spectrum():
    # The Chebyshev interval comes from the Lanczos tridiagonal that CG's
    # coefficients define.  Independent construction: Rayleigh-Ritz on an
    # orthonormal basis of the Krylov space K_k(B, rhs), whose extreme Ritz
    # values must equal those of the tridiagonal for every k, and after
    # k = m steps are the extreme eigenvalues of B.
    from oracle import ipm
    m = 8
    B, ev = _spd(m, 40.0, seed=15)
    rhs = np.random.default_rng(16).standard_normal(m)
    for k in range(1, m + 1):
        alphas, betas = ipm._cg_coeffs(lambda z: B @ z, rhs, k)
        lo, hi = ipm.lanczos_interval(alphas, betas)
        K = np.column_stack([np.linalg.matrix_power(B, i) @ rhs for i in range(k)])
        Qk, _ = np.linalg.qr(K)
        ritz = np.linalg.eigvalsh(Qk.T @ B @ Qk)
        assert lo == pytest.approx(ritz[0], rel=1e-7)
        assert hi == pytest.approx(ritz[-1], rel=1e-7)
        assert ev[0] * (1 - 1e-9) <= lo and hi <= ev[-1] * (1 + 1e-9)
    assert lo == pytest.approx(ev[0], rel=1e-8) and hi == pytest.approx(ev[-1], rel=1e-8)
