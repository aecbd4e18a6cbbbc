"""Seeded synthetic inputs for fast fermion sampling (arXiv 2109.07358).

Every generator returns an L x N matrix U with orthonormal columns (U^dagger U = 1,
the condition stated with Eq. 1), plus the sizes of the workload.  The module holds
the inputs only: it contains none of the sampling arithmetic, so the CPU oracle and
the CUDA path can both consume its outputs without sharing any of the method.

Workloads (sizes are parameters; the defaults are the ones the tests and the bench use):

* ``open_chain``      1D open chain, hopping -1: closed-form sine orbitals.
* ``square_lattice``  nx x ny open square lattice, bond phases uniform in [0, 2 pi).
* ``anderson_chain``  1D open Anderson chain, on-site energies uniform in [-W, W]
                      (the Hamiltonian of Eq. 5, one spin species).
* ``haar``            Haar-random orbitals: QR of a Gaussian matrix.
* ``batch_sizes``     log-uniform (L, N) pairs for many independent instances.
* ``lensemble_orbitals``  top-N left singular vectors of unit-norm Gaussian
                      feature rows (stand-in for the sentence embeddings of the
                      text-summarisation example; the real data is not available).
* ``double_well``     the double-well chain of the supplementary double-well section.
* ``anderson_square`` 2D open Anderson model (Eq. 5), one spin species; with
                      ``gutzwiller_csr`` (Eq. 4) it gives the Anderson-Hubbard
                      Slater-Jastrow workload (``anderson_hubbard_4x4``).
* ``neighbour_jastrow_csr``  nearest-neighbour density-density Jastrow parameters.

Matrices are float64 / complex128 and C-contiguous (row-major L x N).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def open_chain(L: int, N: int) -> np.ndarray:
    """Lowest-N orbitals of H = -sum_j (c_j^+ c_{j+1} + h.c.) on an open chain of L sites.

    phi_n(j) = sqrt(2/(L+1)) sin(pi n j / (L+1)), j = 1..L, n = 1..N; energies
    -2 cos(pi n/(L+1)) are increasing in n, so columns are in energy order.
    """
    j = np.arange(1, L + 1)[:, None]
    n = np.arange(1, N + 1)[None, :]
    return np.ascontiguousarray(np.sqrt(2.0 / (L + 1)) * np.sin(np.pi * n * j / (L + 1)))


def open_chain_hamiltonian(L: int) -> np.ndarray:
    H = np.zeros((L, L))
    i = np.arange(L - 1)
    H[i, i + 1] = -1.0
    H[i + 1, i] = -1.0
    return H


def square_lattice_hamiltonian(nx: int, ny: int, seed: int = 0) -> np.ndarray:
    """Open nx x ny square lattice; bond (a, b) with a < b gets H_ab = -exp(i theta_ab),
    H_ba = conj(H_ab), theta_ab ~ U[0, 2 pi).  Site index a = ix * ny + iy.  Bonds are
    drawn in the order: all +x bonds (row-major over (ix, iy)), then all +y bonds."""
    r = _rng(seed)
    L = nx * ny
    H = np.zeros((L, L), np.complex128)
    ix, iy = np.meshgrid(np.arange(nx - 1), np.arange(ny), indexing="ij")
    a = (ix * ny + iy).ravel()
    b = ((ix + 1) * ny + iy).ravel()
    jx, jy = np.meshgrid(np.arange(nx), np.arange(ny - 1), indexing="ij")
    a2 = (jx * ny + jy).ravel()
    b2 = (jx * ny + jy + 1).ravel()
    A = np.concatenate([a, a2])
    Bb = np.concatenate([b, b2])
    theta = r.uniform(0.0, 2.0 * np.pi, size=A.size)
    t = -np.exp(1j * theta)
    H[A, Bb] = t
    H[Bb, A] = np.conj(t)
    return H


def _lowest(H: np.ndarray, N: int) -> np.ndarray:
    import scipy.linalg as sl

    w, v = sl.eigh(H, subset_by_index=[0, N - 1], driver="evr")
    return np.ascontiguousarray(v)


def square_lattice(nx: int, ny: int, N: int, seed: int = 0) -> np.ndarray:
    """Lowest-N orbitals (complex128, L = nx*ny) of ``square_lattice_hamiltonian``."""
    return _lowest(square_lattice_hamiltonian(nx, ny, seed), N)


def anderson_onsite(L: int, W: float = 1.0, seed: int = 0) -> np.ndarray:
    return _rng(seed).uniform(-W, W, size=L)


def anderson_chain(L: int, N: int, W: float = 1.0, seed: int = 0) -> np.ndarray:
    """Lowest-N orbitals (real) of H = -sum_j (c_j^+ c_{j+1} + h.c.) + sum_j w_j n_j,
    open boundaries, w_j ~ U[-W, W]."""
    import scipy.linalg as sl

    d = anderson_onsite(L, W, seed)
    e = -np.ones(L - 1)
    try:
        w, v = sl.eigh_tridiagonal(d, e, select="i", select_range=(0, N - 1), lapack_driver="stemr")
    except Exception:  # pragma: no cover - older LAPACK without stemr selection
        H = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        return _lowest(H, N)
    return np.ascontiguousarray(v)


def anderson_square_hamiltonian(nx: int, ny: int, W: float = 1.0, seed: int = 0) -> np.ndarray:
    """One spin species of the 2D Anderson model of Eq. 5 on an open nx x ny square
    lattice: hopping -1 on nearest-neighbour bonds, on-site w_i ~ U[-W, W] (site index
    a = ix * ny + iy, energies drawn in site order)."""
    L = nx * ny
    H = np.diag(_rng(seed).uniform(-W, W, size=L))
    for ix in range(nx):
        for iy in range(ny):
            a = ix * ny + iy
            if ix + 1 < nx:
                H[a, a + ny] = H[a + ny, a] = -1.0
            if iy + 1 < ny:
                H[a, a + 1] = H[a + 1, a] = -1.0
    return H


def anderson_square(nx: int, ny: int, N: int, W: float = 1.0, seed: int = 0) -> np.ndarray:
    """Lowest-N orbitals (real, L = nx*ny) of ``anderson_square_hamiltonian``."""
    return _lowest(anderson_square_hamiltonian(nx, ny, W, seed), N)


def gutzwiller_csr(L: int, V: float):
    """The Gutzwiller factor of Eq. 4 as Jastrow parameters over 2L spin-orbitals
    (up-spin orbital i, down-spin orbital L + i): v_{i, L+i} = v_{L+i, i} = V/2, so that
    1/2 sum_ij v_ij n_i n_j = (V/2) sum_i n_{i up} n_{i down}.  Returns CSR arrays
    (row pointers int64, columns int32, values float64), one entry per row."""
    rowptr = np.arange(2 * L + 1, dtype=np.int64)
    col = np.concatenate([np.arange(L, 2 * L), np.arange(L)]).astype(np.int32)
    val = np.full(2 * L, V / 2.0)
    return rowptr, col, val


def neighbour_jastrow_csr(nx: int, ny: int, V: float):
    """A density-density Jastrow on an open nx x ny lattice (one orbital per site):
    v_ab = V/2 on every nearest-neighbour bond (both directions).  CSR arrays as
    ``gutzwiller_csr``."""
    rows = []
    for ix in range(nx):
        for iy in range(ny):
            nb = []
            if ix > 0:
                nb.append((ix - 1) * ny + iy)
            if iy > 0:
                nb.append(ix * ny + iy - 1)
            if iy + 1 < ny:
                nb.append(ix * ny + iy + 1)
            if ix + 1 < nx:
                nb.append((ix + 1) * ny + iy)
            rows.append(nb)
    rowptr = np.zeros(nx * ny + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    return rowptr, col, np.full(col.size, V / 2.0)


def anderson_hubbard_4x4(W: float = 1.0, seed: int = 0):
    """The Anderson-Hubbard workload of the main text's correlated example: 4 x 4 open
    lattice, N = 8 fermions taken as 4 per spin species, both species in the lowest four
    orbitals of the same disordered Hamiltonian (Eq. 5)."""
    return anderson_square(4, 4, 4, W, seed)


def haar(L: int, N: int, seed: int = 0, complex_: bool = True) -> np.ndarray:
    """Haar-random L x N orbitals: Q of the QR factorisation of an i.i.d. Gaussian matrix.
    (Column phases are irrelevant: P(x) is invariant under U -> U D with D diagonal unitary.)"""
    r = _rng(seed)
    G = r.standard_normal((L, N))
    if complex_:
        G = G + 1j * r.standard_normal((L, N))
    Q, _ = np.linalg.qr(G)
    return np.ascontiguousarray(Q)


def batch_sizes(n: int = 256, seed: int = 0, L_range=(256, 8192), N_max: int = 1024):
    """n independent (L, N) pairs: L log-uniform in L_range, N log-uniform in
    [16, min(N_max, L/4)]."""
    r = _rng(seed)
    out = []
    for _ in range(n):
        L = int(round(math.exp(r.uniform(math.log(L_range[0]), math.log(L_range[1])))))
        hi = min(N_max, L // 4)
        N = int(round(math.exp(r.uniform(math.log(16), math.log(hi)))))
        out.append((L, max(1, min(N, hi))))
    return out


def lensemble_features(L: int, D: int, seed: int = 0) -> np.ndarray:
    """L unit-norm Gaussian feature rows of dimension D (the b_i of the L-ensemble)."""
    Phi = _rng(seed).standard_normal((L, D))
    return Phi / np.linalg.norm(Phi, axis=1, keepdims=True)


def lensemble_orbitals(Phi: np.ndarray, N: int) -> np.ndarray:
    """Top-N eigenvectors of C = Phi Phi^T, taken as the left singular vectors of Phi
    (thin SVD; the L x L kernel is never formed)."""
    Uf, s, _ = np.linalg.svd(Phi, full_matrices=False)
    return np.ascontiguousarray(Uf[:, :N])


def lensemble_spectrum(Phi: np.ndarray):
    """Eigen-decomposition of C = Phi Phi^T restricted to its rank: (lambda_j, u_j),
    lambda descending, from the thin SVD of Phi."""
    Uf, s, _ = np.linalg.svd(Phi, full_matrices=False)
    return s**2, np.ascontiguousarray(Uf)


def lensemble_quality_features(L: int, D: int, alpha: float, seed: int = 0) -> np.ndarray:
    """Quality-scaled feature rows b~_i = q_i b_i of the text-summarisation L-ensemble:
    b_i unit-norm Gaussian rows of dimension D (stand-ins for sentence embeddings) and
    qualities q_i = alpha exp(z_i / 2), z_i ~ N(0, 1) (stand-ins for the log-linear quality
    model).  The kernel is C = Phi Phi^T; ``lensemble_spectrum`` gives its eigenpairs."""
    Phi = lensemble_features(L, D, seed)
    z = _rng(seed + 1).standard_normal(L)
    return Phi * (alpha * np.exp(z / 2.0))[:, None]


def double_well(L: int = 64, N: int = 4, c: float = 89.929, a: float = 4096.0, b: float = 2.0,
                t: float = math.pi**2 / 6) -> np.ndarray:
    """Lowest-N orbitals of H = -t sum (c_i^+ c_{i+1} + h.c.) + sum_i V(x_i) n_i with
    V(x) = a (x^2 - b)^2 - c x and x_i evenly spaced on [-2, 2] (supplementary
    double-well section).  The section quotes the balanced-to-imbalanced transition at
    c = 89.929; with t as the nearest-neighbour element on these points it falls at
    c = 46.645, so the default c is in the imbalanced stage."""
    xs = np.linspace(-2.0, 2.0, L)
    V = a * (xs**2 - b) ** 2 - c * xs
    H = np.diag(V) - t * (np.eye(L, k=1) + np.eye(L, k=-1))
    w, v = np.linalg.eigh(H)
    return np.ascontiguousarray(v[:, :N]), xs


# Named workloads with the sizes the tests and the bench use.
def chain_L64_N8():
    """1D open chain, L = 64, N = 8, real (the small plain FP64 workload)."""
    return open_chain(64, 8)


def lattice_64x64_N1024(seed: int = 0):
    """64 x 64 open square lattice with random U(1) hopping phases, N = 1024, complex."""
    return square_lattice(64, 64, 1024, seed)


def anderson_L16384_N2048(seed: int = 0):
    """1D Anderson chain L = 16384, w_j ~ U[-1, 1], N = 2048, real."""
    return anderson_chain(16384, 2048, 1.0, seed)


# ---------------------------------------------------------------------------------
# Device-side generators for the large multi-instance workloads (seeded torch; the
# QR / SVD are library factorisations, not sampling arithmetic).
def haar_torch(L: int, N: int, seed: int, device="cuda", complex_=True):
    """Haar-random L x N orbitals generated on the device: Q of the QR of a Gaussian."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    G = torch.randn((L, N), generator=g, device=device, dtype=torch.float64)
    if complex_:
        G = G + 1j * torch.randn((L, N), generator=g, device=device, dtype=torch.float64)
    Q, _ = torch.linalg.qr(G)
    return Q.contiguous()


def lensemble_orbitals_torch(L: int, D: int, N: int, seed: int, device="cuda"):
    """Top-N left singular vectors of L unit-norm Gaussian feature rows of dimension D."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Phi = torch.randn((L, D), generator=g, device=device, dtype=torch.float64)
    Phi = Phi / Phi.norm(dim=1, keepdim=True)
    Uf, _, _ = torch.linalg.svd(Phi, full_matrices=False)
    return Uf[:, :N].contiguous()


def serving_requests(n: int, seed: int = 0, L_range=(500, 20000), D_range=(64, 512), N_max=200,
                     samples=(1, 32)):
    """Sizes of n serving requests: L log-uniform, D uniform, N uniform in [5, min(N_max, D)],
    samples uniform; returns a list of (L, D, N, n_samples)."""
    r = _rng(seed)
    out = []
    for _ in range(n):
        L = int(round(math.exp(r.uniform(math.log(L_range[0]), math.log(L_range[1])))))
        D = int(r.integers(D_range[0], D_range[1] + 1))
        N = int(r.integers(5, min(N_max, D) + 1))
        s = int(r.integers(samples[0], samples[1] + 1))
        out.append((L, D, N, s))
    return out
