"""The synthetic input recipes: each generator builds the Hamiltonian or features it
states, and returns its lowest orbitals with orthonormal columns (the precondition of
Eq. 1).  Checked against the stated structure (bonds, boundary conditions, on-site
ranges, Hermiticity) and by residuals H U = U E with E the lowest eigenvalues."""
import numpy as np
import pytest

from paper_2109_07358_gb300 import workloads as w


def _check_lowest(H, U, N):
    E = np.linalg.eigvalsh(H)
    Ew = np.real(np.einsum("ij,ik,kj->j", U.conj(), H, U))
    assert np.allclose(U.conj().T @ U, np.eye(N), atol=1e-10)
    assert np.allclose(H @ U, U * Ew, atol=1e-9)          # eigenvectors
    assert np.allclose(np.sort(Ew), E[:N], atol=1e-9)    # the N lowest


def test_square_lattice_recipe():
    nx, ny = 5, 4
    H = w.square_lattice_hamiltonian(nx, ny, seed=3)
    L = nx * ny
    assert np.allclose(H, H.conj().T)
    assert np.allclose(np.diag(H), 0)
    nb = 0
    for a in range(L):
        for b in range(L):
            ax, ay, bx, by = a // ny, a % ny, b // ny, b % ny
            bond = abs(ax - bx) + abs(ay - by) == 1          # open: no wrap-around bonds
            if bond:
                nb += 1
                assert abs(abs(H[a, b]) - 1) < 1e-14             # -e^{i theta}
            else:
                assert H[a, b] == 0
    assert nb == 2 * ((nx - 1) * ny + nx * (ny - 1))
    phases = np.angle(-H[np.triu_indices(L, 1)][np.abs(H[np.triu_indices(L, 1)]) > 0])
    assert np.unique(np.round(phases, 12)).size == nb // 2    # one random phase per bond
    U = w.square_lattice(nx, ny, 7, seed=3)
    _check_lowest(H, U, 7)
    assert np.array_equal(U, w.square_lattice(nx, ny, 7, seed=3))  # seeded


def test_square_lattice_phases_are_uniform():
    from scipy.stats import kstest

    H = w.square_lattice_hamiltonian(24, 24, seed=0)
    iu = np.triu_indices(H.shape[0], 1)
    t = H[iu][np.abs(H[iu]) > 0]
    theta = np.mod(np.angle(-t), 2 * np.pi)
    assert kstest(theta / (2 * np.pi), "uniform").pvalue > 1e-3


@pytest.mark.parametrize("L,N,W", [(200, 30, 1.0), (64, 64, 2.0)])
def test_anderson_chain_recipe(L, N, W):
    d = w.anderson_onsite(L, W, seed=4)
    assert d.min() >= -W and d.max() <= W
    H = np.diag(d) - np.eye(L, k=1) - np.eye(L, k=-1)     # open chain, hopping -1
    U = w.anderson_chain(L, N, W, seed=4)
    assert U.dtype == np.float64
    _check_lowest(H, U, N)


def test_anderson_square_recipe():
    H = w.anderson_square_hamiltonian(4, 4, 2.0, seed=0)
    assert np.allclose(H, H.T)
    off = H - np.diag(np.diag(H))
    assert set(np.unique(off)) <= {-1.0, 0.0} and (off == -1).sum() == 2 * 24  # 24 bonds of a 4x4 open lattice
    assert np.abs(np.diag(H)).max() <= 2.0
    _check_lowest(H, w.anderson_hubbard_4x4(W=2.0, seed=0), 4)


def test_haar_is_orthonormal_and_seeded():
    for cplx in (False, True):
        U = w.haar(50, 12, seed=7, complex_=cplx)
        assert np.iscomplexobj(U) == cplx
        assert np.allclose(U.conj().T @ U, np.eye(12), atol=1e-12)
        assert np.array_equal(U, w.haar(50, 12, seed=7, complex_=cplx))
        assert not np.allclose(U, w.haar(50, 12, seed=8, complex_=cplx))


def test_lensemble_features_and_orbitals():
    Phi = w.lensemble_features(300, 40, seed=2)
    assert np.allclose(np.linalg.norm(Phi, axis=1), 1.0)    # unit-norm rows
    U = w.lensemble_orbitals(Phi, 10)
    assert np.allclose(U.T @ U, np.eye(10), atol=1e-12)
    # the top-10 left singular vectors span the leading eigenspace of C = Phi Phi^T
    C = Phi @ Phi.T
    lam = np.linalg.eigvalsh(C)[::-1][:10]
    assert np.allclose(np.sort(np.diag(U.T @ C @ U))[::-1], lam, atol=1e-9)


def test_serving_and_batch_sizes_follow_their_ranges():
    for L, D, N, s in w.serving_requests(200, seed=1):
        assert 500 <= L <= 20000 and 64 <= D <= 512 and 5 <= N <= min(200, D) and 1 <= s <= 32
    sizes = w.batch_sizes(256, seed=0)
    assert len(sizes) == 256
    for L, N in sizes:
        assert 256 <= L <= 8192 and 16 <= N <= min(1024, L // 4)


def test_quality_features_are_log_normal_scaled():
    from scipy.stats import kstest

    alpha = 0.08
    Phi = w.lensemble_quality_features(4000, 16, alpha, seed=3)
    z = 2 * np.log(np.linalg.norm(Phi, axis=1) / alpha)      # q_i = alpha exp(z_i / 2)
    assert kstest(z, "norm").pvalue > 1e-3
    lam, V = w.lensemble_spectrum(Phi)
    assert np.all(np.diff(lam) <= 1e-12) and lam.size == 16  # descending, rank D
    assert np.allclose(Phi @ (Phi.T @ V), V * lam, atol=1e-9)
