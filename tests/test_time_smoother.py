"""CPU checks of the host model that chooses the multigrid-in-time smoother
(ptp_time_cycle_rho, ptp_choose_time_smoother; no GPU call).

On a spatial eigenmode with eigenvalue lambda of L x = lambda M x, the
periodic implicit-Euler system of a time level with N steps is the circulant
P = (1 + kappa) I - S (S the cyclic shift x^{n-1}), kappa = tau lambda.  The
test writes the error propagation of the V(pre, post) cycle as a dense
matrix from its definition (damped Jacobi, pair-sum restriction, injection,
exact last level) and takes its spectral radius with numpy's eigenvalue
routine, against which the library's power-iteration estimate is checked.
Special cases pin the dense construction itself: kappa -> infinity leaves
the smoother alone, and one exact level gives a zero error."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def ptp():
    from paper_2502_21013_gb300 import build
    build.build()
    from paper_2502_21013_gb300 import ptp as mod
    return mod


def circulant(N, kappa):
    S = np.roll(np.eye(N), 1, axis=0)   # (S x)^n = x^{n-1}
    return (1.0 + kappa) * np.eye(N) - S


def cycle_matrix(Nl, kappa0, pre, post, omega):
    """Error propagation E of one V-cycle on level 0 (b = 0)."""
    def level(l):
        N = Nl[l]
        k = kappa0 * Nl[0] / N
        P = circulant(N, k)
        if l == len(Nl) - 1:
            return np.zeros((N, N))
        Es = np.eye(N) - omega / (1.0 + k) * P
        R = np.zeros((N // 2, N))
        for m in range(N // 2):
            R[m, 2 * m] = R[m, 2 * m + 1] = 1.0
        Pc = circulant(N // 2, 2 * k)
        Ec = level(l + 1)
        # coarse correction with the coarse cycle's own error: x_c = (I - E_c) P_c^{-1} R r
        C = np.eye(N) - R.T @ (np.eye(N // 2) - Ec) @ np.linalg.solve(Pc, R @ P)
        return np.linalg.matrix_power(Es, post) @ C @ np.linalg.matrix_power(Es, pre)
    return level(0)


def rho_dense(Nl, kappa0, pre, post, omega):
    return float(np.max(np.abs(np.linalg.eigvals(cycle_matrix(Nl, kappa0, pre, post, omega)))))


def test_dense_construction_special_cases():
    # Galerkin identity of the hierarchy: R P(kappa) R^T = P(2 kappa) on N / 2 steps
    N, k = 8, 0.37
    R = np.zeros((N // 2, N))
    for m in range(N // 2):
        R[m, 2 * m] = R[m, 2 * m + 1] = 1.0
    assert np.allclose(R @ circulant(N, k) @ R.T, circulant(N // 2, 2 * k))
    # one exact level: the cycle is the solve
    assert rho_dense([4], 0.3, 1, 0, 0.9) == 0.0
    # kappa -> infinity: D^-1 P -> I, each sweep leaves (1 - omega) of the error,
    # and the exact coarse correction of a pair-constant error removes it
    assert abs(rho_dense([8, 4, 2, 1], 1e9, 1, 0, 0.5) - 0.5) < 1e-6


@pytest.mark.parametrize("Nl", [[16, 8, 4, 2, 1], [32, 16, 8, 4, 2], [12, 6, 3]])
@pytest.mark.parametrize("kappa", [1e-4, 0.05, 0.7, 5.0])
@pytest.mark.parametrize("pre,post,omega", [(1, 0, 0.95), (1, 0, 0.5), (1, 1, 0.5), (1, 1, 0.8), (2, 1, 0.7)])
def test_cycle_rho_matches_dense_eigenvalues(ptp, Nl, kappa, pre, post, omega):
    ref = rho_dense(Nl, kappa, pre, post, omega)
    got = ptp.time_cycle_rho(Nl, kappa, pre, post, omega)
    assert abs(got - ref) <= 0.02 * ref + 1e-6, (got, ref)


def test_v10_cycle_amplifies_transport_modes(ptp):
    """The reason for the choice: V(1,0) with omega near 1 grows slow modes
    (kappa -> 0) several-fold, and damps well for kappa >= 1."""
    H = [64, 32, 16, 8, 4, 2, 1]
    assert ptp.time_cycle_rho(H, 1e-5, 1, 0, 0.95) > 3.0
    assert ptp.time_cycle_rho(H, 1.0, 1, 0, 0.95) < 0.5
    assert ptp.time_cycle_rho(H, 1e-5, 1, 1, 0.5) < 0.8


def test_choice(ptp):
    H = [256, 128, 64, 32, 16, 8, 4, 2, 1]
    # the bench problem's kappa_min (about 1.07 on the 257x257 square, N = 256)
    post, omega, rho = ptp.choose_time_smoother(H, 0.9 * 1.07)
    assert (post, omega) == (0, 0.95) and rho <= 0.6
    # the paper's transformer (kappa_min about 8e-4): no V(1,0) reaches the
    # target, V(1,1) with omega 0.5 has the least work per digit
    post, omega, rho = ptp.choose_time_smoother(H, 8e-4)
    assert (post, omega) == (1, 0.5)
    assert rho == pytest.approx(rho_dense([32, 16, 8, 4, 2, 1], 8e-4 * 8, 1, 1, 0.5), rel=0.5)
    # every candidate returned with rho <= 0.6 has rho <= 0.6 at every kappa >= kappa_min
    for kmin in (0.05, 0.2, 0.6):
        post, omega, rho = ptp.choose_time_smoother(H, kmin)
        assert rho <= 0.6
        for k in kmin * 2.0 ** np.arange(0, 8):
            assert ptp.time_cycle_rho(H, k, 1, post, omega) <= 0.6 + 1e-9
    # fixed values are kept
    post, omega, _ = ptp.choose_time_smoother(H, 8e-4, post=0)
    assert post == 0
    post, omega, _ = ptp.choose_time_smoother(H, 8e-4, omega=0.7)
    assert omega == 0.7


def test_bad_hierarchy_is_rejected(ptp):
    with pytest.raises(ptp.PtpError):
        ptp.time_cycle_rho([16, 6, 3], 1.0, 1, 0, 0.9)
    with pytest.raises(ptp.PtpError):
        ptp.choose_time_smoother([], 1.0)
