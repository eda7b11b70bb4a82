"""Pins of the oracle's pressure operator, V-cycle and PCG (Eq. 53 solver).

The matrix is assembled here, independently of the oracle, from the definition
of the 7-point operator: (A p)_c = sum_faces T_f (p_c - p_nb) + Dd_c p_c, with
per-cell high-face coefficients Tx, Ty, Tz and Dirichlet diagonal Dd; the
dense solve is numpy's LAPACK routine."""
import numpy as np
import pytest

from oracle import api


def dense_matrix(n, Tx, Ty, Tz, Dd):
    nx, ny, nz = n
    N = nx * ny * nz
    M = np.zeros((N, N))
    T = (Tx, Ty, Tz)
    stride = (1, nx, nx * ny)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                M[c, c] += Dd[c]
                for d, (q, nd) in enumerate(((i, nx), (j, ny), (k, nz))):
                    if q + 1 < nd:
                        t = T[d][c]
                        o = c + stride[d]
                        M[c, c] += t
                        M[o, o] += t
                        M[c, o] -= t
                        M[o, c] -= t
    return M


def random_coeffs(n, rng, contrast=1.0, outlet_side=1):
    nx, ny, nz = n
    N = nx * ny * nz
    T = [np.exp(contrast * rng.standard_normal(N)) for _ in range(3)]
    idx = np.arange(N)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    T[0][i == nx - 1] = 0
    T[1][j == ny - 1] = 0
    T[2][k == nz - 1] = 0
    Dd = np.zeros(N)
    if outlet_side == 1:
        Dd[i == nx - 1] = 2.0 * np.exp(rng.standard_normal((i == nx - 1).sum()))
    return T[0], T[1], T[2], Dd


def test_operator_1d_tridiagonal():
    """Uniform T = 1 in 1-D with a Dirichlet outlet: the textbook [-1 2 -1] matrix with the
    ghost-cell Dirichlet row (2 + 1) at the outlet end."""
    n = (6, 1, 1)
    Tx = np.ones(6); Tx[-1] = 0
    Dd = np.zeros(6); Dd[-1] = 2.0
    M = np.column_stack([api.apply_A(n, Tx, np.zeros(6), np.zeros(6), Dd, e) for e in np.eye(6)])
    ref = 2 * np.eye(6) - np.eye(6, k=1) - np.eye(6, k=-1)
    ref[0, 0] = 1.0
    ref[-1, -1] = 3.0
    assert np.array_equal(M, ref)


def test_operator_annihilates_linear_field_interior():
    """Constant coefficients: the discrete Laplacian of a linear field is zero away from
    the boundary."""
    n = (8, 7, 6)
    N = 8 * 7 * 6
    T = [np.ones(N) for _ in range(3)]
    Dd = np.zeros(N)
    idx = np.arange(N)
    i, j, k = idx % 8, (idx // 8) % 7, idx // 56
    x = 3.0 * i - 2.0 * j + 0.5 * k
    y = api.apply_A(n, T[0], T[1], T[2], Dd, x)
    inner = (i > 0) & (i < 7) & (j > 0) & (j < 6) & (k > 0) & (k < 5)
    assert np.max(np.abs(y[inner])) < 1e-13


@pytest.mark.parametrize("n", [(8, 8, 8), (7, 5, 6), (8, 8, 1), (5, 9, 1)])
@pytest.mark.parametrize("contrast", [0.0, 2.0])
def test_pcg_matches_dense_solve(n, contrast):
    rng = np.random.default_rng(11)
    Tx, Ty, Tz, Dd = random_coeffs(n, rng, contrast)
    N = np.prod(n)
    b = rng.standard_normal(N)
    x, it, res = api.pcg(n, Tx, Ty, Tz, Dd, b, tol=1e-13, max_it=400)
    ref = np.linalg.solve(dense_matrix(n, Tx, Ty, Tz, Dd), b)
    assert res <= 1e-13
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_operator_matches_dense_definition():
    rng = np.random.default_rng(3)
    n = (5, 4, 3)
    Tx, Ty, Tz, Dd = random_coeffs(n, rng, 1.0)
    x = rng.standard_normal(60)
    y = api.apply_A(n, Tx, Ty, Tz, Dd, x)
    assert np.allclose(y, dense_matrix(n, Tx, Ty, Tz, Dd) @ x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n", [(8, 8, 8), (12, 10, 1), (9, 6, 5)])
def test_vcycle_symmetric_positive_definite(n):
    """CG needs a symmetric positive-definite preconditioner: the V-cycle with (R,B) pre- and
    (B,R) post-smoothing and a palindromic coarsest solve is a symmetric linear map."""
    rng = np.random.default_rng(5)
    Tx, Ty, Tz, Dd = random_coeffs(n, rng, 1.5)
    N = int(np.prod(n))
    Mz = np.column_stack([api.vcycle(n, Tx, Ty, Tz, Dd, e) for e in np.eye(N)])
    assert np.max(np.abs(Mz - Mz.T)) <= 1e-12 * np.max(np.abs(Mz))
    assert np.min(np.linalg.eigvalsh(0.5 * (Mz + Mz.T))) > 0


def pc_prolongation(n, nc):
    """Piecewise-constant prolongation from the coarse grid nc to n (an axis longer
    than 4 cells is halved, rounding up): fine cell (i, j, k) takes its coarse cell's value."""
    nx, ny, nz = n
    P = np.zeros((nx * ny * nz, int(np.prod(nc))))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                q = [c // 2 if m < nf else c for c, m, nf in zip((i, j, k), nc, n)]
                P[i + nx * (j + ny * k), q[0] + nc[0] * (q[1] + nc[1] * q[2])] = 1.0
    return P


@pytest.mark.parametrize("n,nc", [((8, 8, 8), (4, 4, 4)), ((8, 6, 1), (4, 3, 1)), ((8, 1, 1), (4, 1, 1)),
                                  ((7, 8, 8), (4, 4, 4))])
def test_two_level_coarse_operator_is_half_the_galerkin_operator(n, nc):
    """With no smoothing the two-level V-cycle is P A_c^-1 P^T.  Where every axis of length > 1
    is coarsened the coarse operator is half of P^T A P (the Galerkin operator of
    piecewise-constant transfer), so the V-cycle must equal 2 P (P^T A P)^-1 P^T, formed here
    with dense linear algebra (odd length 7: the last coarse cell covers one fine cell)."""
    rng = np.random.default_rng(11)
    Tx, Ty, Tz, Dd = random_coeffs(n, rng, 2.0)
    N = int(np.prod(n))
    A = dense_matrix(n, Tx, Ty, Tz, Dd)
    P = pc_prolongation(n, nc)
    ref = 2.0 * P @ np.linalg.solve(P.T @ A @ P, P.T)
    M = np.column_stack([api.vcycle(n, Tx, Ty, Tz, Dd, e, nu1=0, nu2=0) for e in np.eye(N)])
    assert np.max(np.abs(M - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_semi_coarsened_uniform_medium_gives_the_2h_discretisation():
    """8 x 8 x 3: x and y are halved, z (3 cells) is not.  For a uniform medium the coarse
    operator must be the discretisation on cells of 2h x 2h x h: link k * area / distance
    (x, y: k 2h h / 2h; z: k 4h^2 / h) and an outlet link 2 k area / cell width on x+."""
    k, h = 1.7, 1.0
    n, nc = (8, 8, 3), (4, 4, 3)
    N = int(np.prod(n))
    idx = np.arange(N)
    i, j, kk = idx % 8, (idx // 8) % 8, idx // 64
    t = k * h * h / h
    Tx = np.where(i < 7, t, 0.0)
    Ty = np.where(j < 7, t, 0.0)
    Tz = np.where(kk < 2, t, 0.0)
    Dd = np.where(i == 7, 2 * k * h * h / h, 0.0)
    Nc = int(np.prod(nc))
    ic = np.arange(Nc)
    I, J, K = ic % 4, (ic // 4) % 4, ic // 16
    hx, hy, hz = 2 * h, 2 * h, h
    Ac = dense_matrix(nc, np.where(I < 3, k * hy * hz / hx, 0.0), np.where(J < 3, k * hx * hz / hy, 0.0),
                      np.where(K < 2, k * hx * hy / hz, 0.0), np.where(I == 3, 2 * k * hy * hz / hx, 0.0))
    P = pc_prolongation(n, nc)
    ref = P @ np.linalg.solve(Ac, P.T)
    M = np.column_stack([api.vcycle(n, Tx, Ty, Tz, Dd, e, nu1=0, nu2=0) for e in np.eye(N)])
    assert np.max(np.abs(M - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [(32, 32, 1), (16, 16, 16)])
def test_vcycle_convergence_factor_constant_coefficients(n):
    """As a stationary iteration x <- x + M(b - Ax) the V-cycle contracts the residual by a
    factor below 0.4 per cycle on the constant-coefficient problem (cell-centred coarsening
    with piecewise-constant transfer gives about 0.3-0.39)."""
    N = int(np.prod(n))
    rng = np.random.default_rng(7)
    Tx, Ty, Tz, Dd = random_coeffs(n, rng, 0.0)
    b = rng.standard_normal(N)
    x = np.zeros(N)
    norms = []
    for _ in range(8):
        r = b - api.apply_A(n, Tx, Ty, Tz, Dd, x)
        norms.append(np.linalg.norm(r))
        x = x + api.vcycle(n, Tx, Ty, Tz, Dd, r)
    factor = (norms[-1] / norms[2]) ** (1.0 / 5)
    assert factor < 0.4, norms


def cell_field_coeffs(n, K):
    """Face coefficients as harmonic means of a cell field K, Dirichlet outlet on x+."""
    nx, ny, nz = n
    Kc = K.reshape(nz, ny, nx)
    T = [np.zeros((nz, ny, nx)) for _ in range(3)]
    T[0][:, :, :-1] = 2 / (1 / Kc[:, :, :-1] + 1 / Kc[:, :, 1:])
    T[1][:, :-1, :] = 2 / (1 / Kc[:, :-1, :] + 1 / Kc[:, 1:, :])
    if nz > 1:
        T[2][:-1] = 2 / (1 / Kc[:-1] + 1 / Kc[1:])
    Dd = np.zeros((nz, ny, nx))
    Dd[:, :, -1] = 2 * Kc[:, :, -1]
    return [t.ravel() for t in T] + [Dd.ravel()]


@pytest.mark.parametrize("kind,max_it", [("lognormal1", 10), ("lognormal3", 12), ("jump1e3", 16)])
def test_pcg_iterations_bounded_under_coefficient_jumps(kind, max_it):
    """Smooth log-normal coefficient fields (sigma 1 and 3, correlation length 8 cells) and a
    1e3 jump (the water/air density ratio of the free-flow pressure coefficients).  The
    halved Galerkin coarse operator takes 7, 9 and 12 iterations to 1e-8; a coarse operator
    that combines each row's links in series (harmonic along the row) takes 7, 13 and 28,
    the unhalved Galerkin operator more than either."""
    from paper_2003_08374_gb300.workloads import gaussian_random_field
    n = (32, 32, 32)
    rng = np.random.default_rng(1)
    z = gaussian_random_field(n[::-1], 8.0, rng).ravel()
    K = {"lognormal1": np.exp(z), "lognormal3": np.exp(3 * z),
         "jump1e3": np.where(z > 0.3, 1e3, 1.0)}[kind]
    Tx, Ty, Tz, Dd = cell_field_coeffs(n, K)
    b = rng.standard_normal(z.size)
    x, it, res = api.pcg(n, Tx, Ty, Tz, Dd, b, tol=1e-8, max_it=300)
    assert res <= 1e-8 and it < max_it, it
