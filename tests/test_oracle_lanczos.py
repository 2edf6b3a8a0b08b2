"""Pins for the oracle's adaptive Lanczos exponential (Sec. VI.B, Eqs. 36-38)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import hamiltonian as ham
from oracle.lanczos import exp_tridiag_e1, expm_lanczos
from oracle.mesh import Mesh


def _tiny(p=2, n=(2, 3, 2), seed=1):
    br = [np.linspace(-1.5, 1.5, k + 1) for k in n]
    m = Mesh(*br, p)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-2, 1, size=(m.n_elem, m.nq ** 3))
    return m, v


def _rand(n, k, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    return a / np.linalg.norm(a, axis=1, keepdims=True)


def test_exp_tridiag_matches_expm():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(9)
    b = rng.uniform(0.1, 1.0, 8)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    y = exp_tridiag_e1(a, b, 0.7)
    ref = scipy.linalg.expm(-0.7j * T)[:, 0]
    np.testing.assert_allclose(y, ref, atol=1e-14)


@pytest.mark.parametrize("tau", [0.05, 0.3, 1.0])
def test_lanczos_matches_dense_expm(tau):
    m, v = _tiny()
    H = ham.dense_Hbar(m, v)
    psi = _rand(m.N_int, 3, 2)
    out, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, tau, 1e-10, 64)
    ref = (scipy.linalg.expm(-1j * tau * H) @ psi.T).T
    assert np.abs(out - ref).max() < 1e-9
    assert all(len(k) == 1 for k in info["k"])      # no sub-steps needed
    # unitarity
    np.testing.assert_allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-10)


def test_tolerance_controls_error():
    m, v = _tiny(p=3)
    H = ham.dense_Hbar(m, v)
    psi = _rand(m.N_int, 1, 4)
    ref = scipy.linalg.expm(-1j * 0.5 * H) @ psi[0]
    errs, ks = [], []
    for tol in (1e-4, 1e-7, 1e-10):
        out, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, 0.5, tol, 200)
        errs.append(np.linalg.norm(out[0] - ref))
        ks.append(info["k"][0][0])
        assert errs[-1] < 10 * tol
    assert ks[0] < ks[1] < ks[2]


def test_eigenvector_breaks_down_with_exact_phase():
    m, v = _tiny(p=2)
    H = ham.dense_Hbar(m, v)
    lam, S = np.linalg.eigh(H)
    psi = S[:, 3][None, :].astype(complex)
    out, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, 0.8, 1e-10, 64)
    assert info["k"][0] == [1]
    np.testing.assert_allclose(out[0], np.exp(-0.8j * lam[3]) * psi[0], atol=1e-12)


def test_substeps_compose_to_the_same_exponential():
    m, v = _tiny(p=3)
    H = ham.dense_Hbar(m, v)
    psi = _rand(m.N_int, 2, 6)
    out, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, 2.0, 1e-10, 8)
    ref = (scipy.linalg.expm(-2.0j * H) @ psi.T).T
    nsub = max(len(k) for k in info["k"])
    assert nsub > 1
    assert np.abs(out - ref).max() < 10 * nsub * 1e-10


def test_k_fixed_replays_adaptive_choice():
    m, v = _tiny(p=2)
    psi = _rand(m.N_int, 2, 8)
    f = lambda x: ham.apply_H(m, v, x)
    out, info = expm_lanczos(f, psi, 0.4, 1e-10, 64)
    ks = [k[0] for k in info["k"]]
    out2, info2 = expm_lanczos(f, psi, 0.4, 1e-10, 64, k_fixed=ks)
    np.testing.assert_array_equal(out, out2)


def test_reorthogonalized_lanczos_keeps_the_basis_orthonormal_and_matches_expm():
    """CGS2 re-orthogonalization: same exponential, orthonormal basis to rounding even
    where the three-term recurrence loses orthogonality (long run, wide spectrum)."""
    import scipy.linalg
    from oracle.lanczos import expm_lanczos
    rng = np.random.default_rng(4)
    n = 300
    lam = np.concatenate([np.linspace(0, 1, n - 5), [40, 60, 80, 120, 200]])
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    H = (U * lam) @ U.conj().T
    psi = (rng.standard_normal((1, n)) + 1j * rng.standard_normal((1, n)))
    psi /= np.linalg.norm(psi)
    ref = scipy.linalg.expm(-1j * 0.2 * H) @ psi[0]
    out, _ = expm_lanczos(lambda x: H @ x, psi, 0.2, 1e-12, 120, reorth=True)
    assert np.abs(out[0] - ref).max() < 1e-10

    def basis(reorth, k=60):
        q = psi[0] / np.linalg.norm(psi[0])
        Q, beta = [q], 0.0
        prev = np.zeros_like(q)
        for j in range(k):
            w = H @ Q[j]
            a = np.vdot(Q[j], w).real
            w = w - a * Q[j] - beta * prev
            if reorth:
                Qm = np.array(Q)
                for _ in range(2):
                    w = w - Qm.T @ (Qm.conj() @ w)
            beta = np.linalg.norm(w)
            prev = Q[j]
            Q.append(w / beta)
        Qm = np.array(Q)
        return np.abs(Qm.conj() @ Qm.T - np.eye(len(Q))).max()

    assert basis(True) < 1e-13
    assert basis(False) > 1e-6      # the plain recurrence drifts on this spectrum
