"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check goes through an
independent route -- values printed in the paper (tests/golden/), the dense
flattening of Eq. x1 times an explicit Khatri-Rao product, closed-form
least-squares solutions, dense brute-force norms, central finite differences,
or invariants that must hold exactly.
"""
import itertools

import numpy as np
import pytest

import oracle
from golden_io import read

# ---------------------------------------------------------------------------
# Independent dense helpers (test-local; the oracle never uses dense tensors).
# ---------------------------------------------------------------------------


def dense_from_coo(idx, val, dims):
    X = np.zeros(tuple(int(d) for d in dims), np.float64)
    X[idx[0], idx[1], idx[2]] = val
    return X


def unfold(X, n):
    """Flattening X^n of Eq. x1 (0-based): X1[i, j+kJ], X2[j, k+iK], X3[k, i+jI]."""
    I, J, K = X.shape
    if n == 0:
        out = np.zeros((I, J * K))
        for i, j, k in itertools.product(range(I), range(J), range(K)):
            out[i, j + k * J] = X[i, j, k]
    elif n == 1:
        out = np.zeros((J, K * I))
        for i, j, k in itertools.product(range(I), range(J), range(K)):
            out[j, k + i * K] = X[i, j, k]
    else:
        out = np.zeros((K, I * J))
        for i, j, k in itertools.product(range(I), range(J), range(K)):
            out[k, i + j * I] = X[i, j, k]
    return out


def khatri_rao(P, Q):
    """Column-wise Kronecker product (Appendix A, Eq. khatraodef)."""
    R = P.shape[1]
    return np.stack([np.kron(P[:, r], Q[:, r]) for r in range(R)], axis=1)


def mttkrp_dense(X, n, F):
    """X^n (F_f kr F_in) with (f, in) = (C,B), (A,C), (B,A) for n = 0, 1, 2."""
    A, B, C = F
    kr = [khatri_rao(C, B), khatri_rao(A, C), khatri_rao(B, A)][n]
    return unfold(X, n) @ kr


def kruskal_dense(dims, F, lam=None):
    A, B, C = F
    R = A.shape[1]
    lam = np.ones(R) if lam is None else lam
    return np.einsum("r,ir,jr,kr->ijk", lam, A, B, C)


def random_sparse(rng, dims, density):
    cells = int(np.prod(dims))
    nnz = max(1, int(density * cells))
    lin = rng.choice(cells, size=nnz, replace=False)
    i, rem = np.divmod(lin, dims[1] * dims[2])
    j, k = np.divmod(rem, dims[2])
    idx = np.stack([i, j, k]).astype(np.int32)
    perm = rng.permutation(nnz)
    val = rng.uniform(-1.0, 1.0, nnz).astype(np.float32)
    return oracle.Tensor(idx[:, perm], val[perm], dims)


def dense_as_coo(X):
    idx = np.array(np.nonzero(np.ones_like(X)), dtype=np.int32)
    return oracle.Tensor(idx, X[idx[0], idx[1], idx[2]].astype(np.float32), X.shape)


# ---------------------------------------------------------------------------
# Appendix A.1: the flattening convention.
# ---------------------------------------------------------------------------


def appA1_tensor():
    g = read("appA1_unfolding.txt")
    I, J, K = (int(x) for x in g["dims"][0])
    X = np.zeros((I, J, K))
    for k in range(K):
        X[:, :, k] = g["slice %d" % (k + 1)]
    return X, g


def test_appA1_flattenings_match_paper():
    X, g = appA1_tensor()
    np.testing.assert_array_equal(unfold(X, 0), g["X1"])
    np.testing.assert_array_equal(unfold(X, 1), g["X2"])
    np.testing.assert_array_equal(unfold(X, 2), g["X3"])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_appA1_oracle_csr_rows_are_transposed_flattening(mode):
    """Mode n's CSR rows are the nonzero rows of (X^{n+1})^T, in order (Sec. 3)."""
    X, g = appA1_tensor()
    t = dense_as_coo(X)
    keep = t.val != 0
    t = oracle.Tensor(t.idx[:, keep], t.val[keep], X.shape)
    st, csr = oracle.build_csr(t, mode)
    assert st == oracle.OK
    nxt = g[["X2", "X3", "X1"][mode]].T  # (X^{n+1})^T as printed
    nonzero_rows = np.flatnonzero(np.any(nxt != 0, axis=1))
    assert csr["nfib"] == len(nonzero_rows)
    o_ax, in_ax, f_ax = oracle.axes(mode)
    dim_f, dim_in = X.shape[f_ax], X.shape[in_ax]
    for fib, row in enumerate(nonzero_rows):
        o, f = divmod(row, dim_f)  # row index of (X^{n+1})^T is f + o*dim_f
        assert csr["fiber_idx"][fib] == f
        assert csr["fiber_ptr"][o] <= fib < csr["fiber_ptr"][o + 1]
        dense_row = np.zeros(dim_in)
        s, e = csr["nz_ptr"][fib], csr["nz_ptr"][fib + 1]
        assert np.all(np.diff(csr["nz_idx"][s:e]) > 0)  # ascending columns
        dense_row[csr["nz_idx"][s:e]] = csr["nz_val"][s:e]
        np.testing.assert_array_equal(dense_row, nxt[row])


# ---------------------------------------------------------------------------
# Appendix D: the MTTKRP worked example.
# ---------------------------------------------------------------------------


def appD():
    g = read("appD_example.txt")
    idx = g["S"].T.astype(np.int32)
    val = g["v"][:, 0].astype(np.float32)
    dims = [int(x) for x in g["dims"][0]]
    return oracle.Tensor(idx, val, dims), g


def test_appD_coo_listing_is_the_printed_tensor():
    t, g = appD()
    X = dense_from_coo(t.idx, t.val, t.dims)
    np.testing.assert_array_equal(unfold(X, 0), g["X1"])
    np.testing.assert_array_equal(unfold(X, 1), g["X2"])
    np.testing.assert_array_equal(unfold(X, 1).T, g["X2T"])


def test_appD_csr_bit_exact():
    t, _ = appD()
    st, csr = oracle.build_csr(t, 0)
    assert st == oracle.OK
    want = read("appD_csr_mode1.txt")
    for key in ("fiber_ptr", "fiber_idx", "nz_ptr", "nz_idx", "nz_val"):
        np.testing.assert_array_equal(csr[key], want[key].reshape(-1), err_msg=key)


def test_appD_intermediates_and_result_through_csr():
    """value(M^r) <- (Xhat^2)^T b_r, n_r <- M^r c_r (Algorithm 1) on the oracle CSR."""
    t, g = appD()
    st, csr = oracle.build_csr(t, 0)
    B, C = g["B"], g["C"]
    I, K = t.dims[0], t.dims[2]
    for r, name in enumerate(["M1", "M2"]):
        v = np.array([np.dot(csr["nz_val"][s:e], B[csr["nz_idx"][s:e], r])
                      for s, e in zip(csr["nz_ptr"][:-1], csr["nz_ptr"][1:])])
        M = np.zeros((I, K))
        for o in range(I):
            for fib in range(csr["fiber_ptr"][o], csr["fiber_ptr"][o + 1]):
                M[o, csr["fiber_idx"][fib]] = v[fib]
        np.testing.assert_array_equal(M, g[name])
        np.testing.assert_array_equal(M @ C[:, r], g["M"][:, r])


def test_appD_oracle_mttkrp_equals_printed_result():
    t, g = appD()
    A = np.ones((t.dims[0], 2))
    N = oracle.mttkrp(t, 0, [A, g["B"], g["C"]])
    np.testing.assert_array_equal(N, g["M"])


# ---------------------------------------------------------------------------
# Brute force and invariants.
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp_brute_force_khatri_rao(seed, mode):
    rng = np.random.default_rng(1000 + seed)
    dims = [int(x) for x in rng.integers(1, 8, size=3)]
    R = int(rng.integers(1, 6))
    t = random_sparse(rng, dims, density=0.35)
    F = [rng.standard_normal((d, R)) for d in dims]
    X = dense_from_coo(t.idx, t.val, dims)
    np.testing.assert_allclose(oracle.mttkrp(t, mode, F), mttkrp_dense(X, mode, F),
                               rtol=1e-12, atol=1e-12)


def test_mttkrp_rows_restriction():
    rng = np.random.default_rng(7)
    dims = [30, 20, 10]
    t = random_sparse(rng, dims, 0.05)
    F = [rng.standard_normal((d, 4)) for d in dims]
    full = oracle.mttkrp(t, 1, F)
    rows = np.array([19, 0, 7, 3])
    np.testing.assert_array_equal(oracle.mttkrp_rows(t, 1, F, rows), full[rows])


def test_cross_mode_invariant():
    """sum_i A.M1 = sum_j B.M2 = sum_k C.M3 = <X, [[A,B,C]]> (each is the
    trilinear form sum_nnz x a_ir b_jr c_kr summed over r)."""
    rng = np.random.default_rng(11)
    dims = [9, 7, 5]
    t = random_sparse(rng, dims, 0.3)
    F = [rng.standard_normal((d, 3)) for d in dims]
    X = dense_from_coo(t.idx, t.val, dims)
    want = float(np.sum(X * kruskal_dense(dims, F)))
    for mode in range(3):
        got = float(np.sum(F[mode] * oracle.mttkrp(t, mode, F)))
        assert got == pytest.approx(want, rel=1e-12)
    assert oracle.inner(t, F) == pytest.approx(want, rel=1e-12)


def test_gram_khatri_rao_identity():
    """(C kr B)^T (C kr B) = C^T C * B^T B (Eq. kr-product)."""
    rng = np.random.default_rng(3)
    B, C = rng.standard_normal((6, 4)), rng.standard_normal((5, 4))
    KR = khatri_rao(C, B)
    np.testing.assert_allclose(oracle.gram(C) * oracle.gram(B), KR.T @ KR, rtol=1e-12)
    np.testing.assert_allclose(oracle.gram(B), B.T @ B, rtol=1e-13)


def test_jacobi_eigen_and_pinv():
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((7, 4))
    S = Q @ Q.T  # rank 4, 7 x 7
    w, V = oracle.sym_eig_jacobi(S)
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(S), atol=1e-11)
    np.testing.assert_allclose(V @ np.diag(w) @ V.T, S, atol=1e-11)
    np.testing.assert_allclose(V.T @ V, np.eye(7), atol=1e-12)
    np.testing.assert_allclose(oracle.pinv_sym(S), np.linalg.pinv(S, hermitian=True),
                               atol=1e-9)


# ---------------------------------------------------------------------------
# ALS.
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("lam_reg", [0.0, 0.7])
def test_als_update_is_least_squares(mode, lam_reg):
    """One ALS update equals the textbook least-squares (ridge) solution of
    Eq. als-astep / Eq. tensorapprx-ref-sol on the dense flattening."""
    rng = np.random.default_rng(21 + mode)
    dims = [6, 5, 4]
    R = 3
    t = random_sparse(rng, dims, 0.5)
    F = [rng.standard_normal((d, R)) for d in dims]
    X = dense_from_coo(t.idx, t.val, dims)
    kr = [khatri_rao(F[2], F[1]), khatri_rao(F[0], F[2]), khatri_rao(F[1], F[0])][mode]
    Xn = unfold(X, mode)
    aug_A = np.vstack([kr, np.sqrt(lam_reg) * np.eye(R)])
    aug_b = np.vstack([Xn.T, np.zeros((R, Xn.shape[0]))])
    want = np.linalg.lstsq(aug_A, aug_b, rcond=None)[0].T
    st, F2, lam = oracle.als_mode_update(t, mode, F, lam_reg)
    assert st == oracle.OK
    np.testing.assert_allclose(F2[mode] * lam, want, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(np.linalg.norm(F2[mode], axis=0), 1.0, rtol=1e-13)
    for m in range(3):
        if m != mode:
            np.testing.assert_array_equal(F2[m], F[m])


def test_als_singular_gamma_uses_pseudo_inverse():
    """Duplicated factor columns make the Hadamard of Grams singular; the update
    must then be the minimum-norm least-squares solution (Eq. kr-pseudo)."""
    rng = np.random.default_rng(8)
    dims = [6, 5, 4]
    t = random_sparse(rng, dims, 0.6)
    b = rng.standard_normal((5, 1))
    c = rng.standard_normal((4, 1))
    F = [rng.standard_normal((6, 2)), np.hstack([b, b]), np.hstack([c, c])]
    X = dense_from_coo(t.idx, t.val, dims)
    kr = khatri_rao(F[2], F[1])
    want = unfold(X, 0) @ np.linalg.pinv(kr.T)
    st, F2, lam = oracle.als_mode_update(t, 0, F)
    assert st == oracle.ESINGULAR
    np.testing.assert_allclose(F2[0] * lam, want, rtol=1e-8, atol=1e-9)


def test_fit_matches_dense_residual():
    rng = np.random.default_rng(13)
    dims = [7, 6, 5]
    t = random_sparse(rng, dims, 0.4)
    F = [rng.standard_normal((d, 3)) for d in dims]
    lam = rng.uniform(0.5, 2.0, 3)
    X = dense_from_coo(t.idx, t.val, dims)
    want = 1.0 - np.linalg.norm(X - kruskal_dense(dims, F, lam)) / np.linalg.norm(X)
    assert oracle.fit(t, F, lam) == pytest.approx(want, abs=1e-12)
    assert oracle.model_norm2(dims, F, lam) == pytest.approx(
        float(np.sum(kruskal_dense(dims, F, lam) ** 2)), rel=1e-12)
    assert oracle.norm2(t) == pytest.approx(float(np.sum(X * X)), rel=1e-13)


def test_als_rank_one_tensor_fits_after_one_sweep():
    rng = np.random.default_rng(17)
    dims = [6, 5, 4]
    a, b, c = (rng.uniform(0.5, 1.5, (d, 1)) for d in dims)
    X = kruskal_dense(dims, [a, b, c])
    t = dense_as_coo(X)
    F0 = [rng.uniform(0.1, 1.0, (d, 1)) for d in dims]
    st, F, lam, fit = oracle.als_sweep(t, F0)
    assert st == oracle.OK
    assert fit > 1.0 - 1e-6  # fp32 storage of the values bounds the residual
    np.testing.assert_allclose(np.abs(F[0][:, 0]), (a / np.linalg.norm(a))[:, 0], rtol=1e-6)


def test_als_exact_rank_tensor_converges():
    rng = np.random.default_rng(19)
    dims = [10, 9, 8]
    R = 3
    truth = [rng.standard_normal((d, R)) for d in dims]
    t = dense_as_coo(kruskal_dense(dims, truth))
    F = [rng.standard_normal((d, R)) for d in dims]
    fit = 0.0
    for _ in range(300):
        st, F, lam, fit = oracle.als_sweep(t, F)
        if fit >= 0.99999:
            break
    assert fit >= 0.9999


def test_als_fit_is_monotone_on_sparse_data():
    """ALS never increases the least-squares objective (each update is an exact
    block minimiser), so the fit sequence is non-decreasing."""
    rng = np.random.default_rng(23)
    dims = [20, 15, 10]
    t = random_sparse(rng, dims, 0.1)
    F = [rng.standard_normal((d, 4)) for d in dims]
    fits = []
    for _ in range(8):
        st, F, lam, fit = oracle.als_sweep(t, F)
        fits.append(fit)
    assert all(b >= a - 1e-12 for a, b in zip(fits, fits[1:]))


# ---------------------------------------------------------------------------
# GD.
# ---------------------------------------------------------------------------


def dense_loss(X, F, lam_reg):
    dims = X.shape
    return 0.5 * float(np.sum((X - kruskal_dense(dims, F)) ** 2)) + 0.5 * lam_reg * sum(
        float(np.sum(f * f)) for f in F)


@pytest.mark.parametrize("lam_reg", [0.0, 0.3])
def test_loss_matches_dense(lam_reg):
    rng = np.random.default_rng(29)
    dims = [6, 5, 7]
    t = random_sparse(rng, dims, 0.3)
    F = [rng.standard_normal((d, 3)) for d in dims]
    X = dense_from_coo(t.idx, t.val, dims)
    assert oracle.loss(t, F, lam_reg) == pytest.approx(dense_loss(X, F, lam_reg), rel=1e-12)


@pytest.mark.parametrize("lam_reg", [0.0, 0.3])
def test_gradient_central_differences(lam_reg):
    """Eq. gd-A (with -N) against central differences of the dense objective."""
    rng = np.random.default_rng(31)
    dims = [5, 4, 3]
    t = random_sparse(rng, dims, 0.5)
    F = [rng.standard_normal((d, 2)) for d in dims]
    X = dense_from_coo(t.idx, t.val, dims)
    G = oracle.gd_gradient(t, F, lam_reg)
    h = 1e-6
    for m in range(3):
        fd = np.zeros_like(F[m])
        for i in range(F[m].shape[0]):
            for r in range(F[m].shape[1]):
                Fp = [f.copy() for f in F]
                Fm = [f.copy() for f in F]
                Fp[m][i, r] += h
                Fm[m][i, r] -= h
                fd[i, r] = (dense_loss(X, Fp, lam_reg) - dense_loss(X, Fm, lam_reg)) / (2 * h)
        np.testing.assert_allclose(G[m], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("seed,scale", [(37, 1.0), (38, 6.0)])
def test_gd_step_armijo_backtracking(seed, scale):
    """Each step reproduces an independent backtracking run on the dense loss:
    alpha0 = min(2 alpha_prev, 1), halve until f(theta - alpha grad) <= f(theta)
    - 1e-4 alpha ||grad||^2, then theta <- theta - alpha grad.  With scale > 1 the
    loss is steep, the accepted steps are far below 1 and alpha0 = 2 alpha_prev
    decides where the search starts."""
    rng = np.random.default_rng(seed)
    dims = [8, 7, 6]
    t = random_sparse(rng, dims, 0.3)
    t = oracle.Tensor(t.idx, t.val * scale, dims)
    X = dense_from_coo(t.idx, t.val, dims)
    F = [scale * rng.standard_normal((d, 3)) for d in dims]
    alpha = 0.0
    prev = dense_loss(X, F, 0.0)
    halvings = 0
    start_matters = 0

    def backtrack(a, F, G, f0, g2):
        n = 0
        for _ in range(100):
            if dense_loss(X, [f - a * g for f, g in zip(F, G)], 0.0) <= f0 - 1e-4 * a * g2:
                break
            a *= 0.5
            n += 1
        return a, n

    for it in range(8):
        G = oracle.gd_gradient(t, F)
        g2 = sum(float(np.sum(g * g)) for g in G)
        want, n = backtrack(1.0 if alpha <= 0 else min(2 * alpha, 1.0), F, G, prev, g2)
        halvings += n
        start_matters += backtrack(1.0, F, G, prev, g2)[0] != want
        st, F2, alpha, lo, g2o = oracle.gd_step(t, F, alpha)
        assert st == oracle.OK
        assert g2o == pytest.approx(g2, rel=1e-12)
        assert alpha == want
        assert lo <= prev - 1e-4 * alpha * g2 + 1e-12 * abs(prev)
        for m in range(3):
            np.testing.assert_allclose(F2[m], F[m] - alpha * G[m], rtol=1e-14, atol=1e-14)
        assert lo == pytest.approx(dense_loss(X, F2, 0.0), rel=1e-12)
        F, prev = F2, lo
    assert halvings > 0  # the run exercised the backtracking branch
    if scale > 1.0:
        assert start_matters > 0  # starting at 1 instead of 2 alpha_prev would differ


@pytest.mark.parametrize("seed,lam_reg", [(41, 0.0), (42, 0.4)])
def test_gd_ray_polynomial_is_the_loss_along_the_ray(seed, lam_reg):
    """The seven coefficients of phi(alpha) = f(theta - alpha grad) reproduce the
    dense loss (computed here from the dense tensor, independently of the
    oracle) at step sizes from 1e-4 to 10."""
    rng = np.random.default_rng(seed)
    dims = [8, 7, 6]
    t = random_sparse(rng, dims, 0.3)
    X = dense_from_coo(t.idx, t.val, dims)
    F = [rng.standard_normal((d, 3)) for d in dims]
    G = oracle.gd_gradient(t, F, lam_reg)
    c = oracle.gd_ray_poly(t, F, G, lam_reg)
    for a in [0.0, 1e-4, 3e-3, 0.02, 0.1, 0.7, 2.5, 10.0]:
        want = dense_loss(X, [f - a * g for f, g in zip(F, G)], lam_reg)
        assert np.polyval(c[::-1], a) == pytest.approx(want, rel=1e-10), a


@pytest.mark.parametrize("seed,lam_reg,scale", [(43, 0.0, 1.0), (44, 0.4, 1.0), (45, 0.0, 6.0)])
def test_gd_exact_step_is_the_minimiser_on_the_ray(seed, lam_reg, scale):
    """The exact step's alpha is the global minimiser of the dense loss along the
    ray: no point of a brute-force grid (log-spaced over eight decades around
    alpha and linear up to 4 alpha) is lower; the new point is theta - alpha
    grad with the loss it reports; it is at least as low as the backtracking
    step's; the loss keeps decreasing over the steps."""
    rng = np.random.default_rng(seed)
    dims = [8, 7, 6]
    t = random_sparse(rng, dims, 0.3)
    t = oracle.Tensor(t.idx, t.val * scale, dims)
    X = dense_from_coo(t.idx, t.val, dims)
    F = [scale * rng.standard_normal((d, 3)) for d in dims]
    prev = dense_loss(X, F, lam_reg)
    for it in range(4):
        G = oracle.gd_gradient(t, F, lam_reg)
        st, F2, alpha, lo, g2 = oracle.gd_step_exact(t, F, lam_reg)
        assert st == oracle.OK and alpha > 0
        for m in range(3):
            np.testing.assert_allclose(F2[m], F[m] - alpha * G[m], rtol=1e-14, atol=1e-14)
        assert lo == pytest.approx(dense_loss(X, F2, lam_reg), rel=1e-12)
        grid = np.concatenate([np.geomspace(alpha * 1e-4, alpha * 1e4, 1601),
                               np.linspace(0.0, 4 * alpha, 801)])
        best = min(dense_loss(X, [f - a * g for f, g in zip(F, G)], lam_reg) for a in grid)
        assert lo <= best + 1e-12 * abs(best)
        st_b, Fb, ab, lob, _ = oracle.gd_step(t, F, 0.0, lam_reg)
        assert lo <= lob + 1e-12 * abs(lob)
        assert lo < prev
        F, prev = F2, lo


def test_gd_line_search_failure_leaves_factors():
    """When no trial passes the test (here a NaN value makes every comparison
    false), the step reports ELSFAIL and leaves the factors and alpha as they were."""
    dims = [2, 2, 2]
    t = oracle.Tensor(np.array([[0], [0], [0]]), [np.nan], dims)
    F = [np.ones((2, 1)) for _ in range(3)]
    st, F2, alpha, lo, g2 = oracle.gd_step(t, F, 0.5)
    assert st == oracle.ELSFAIL
    for m in range(3):
        np.testing.assert_array_equal(F2[m], F[m])
    assert alpha == 0.5


# ---------------------------------------------------------------------------
# Joint matrix completion and tensor factorization (Appendix F).
# ---------------------------------------------------------------------------


def joint_problem(seed, dims=(7, 6, 5), R=3, density=0.35, ny=20):
    rng = np.random.default_rng(seed)
    t = random_sparse(rng, list(dims), density)
    lin = rng.choice(dims[0] * dims[1], size=ny, replace=False)
    yi, yj = np.divmod(lin, dims[1])
    y = oracle.Ratings(np.stack([yi, yj]), rng.uniform(0.0, 5.0, ny))
    F = [rng.standard_normal((d, R)) for d in dims]
    return rng, t, y, F


def dense_joint_loss(X, Ymask, Y, F, mu, lam):
    """Eq. joint-obj-fn from dense arrays: the observed ratings (Ymask), every
    cell of X, and the ridge."""
    A, B, C = F
    fy = 0.5 * float(np.sum(Ymask * (Y - A @ B.T) ** 2))
    return fy + mu * dense_loss(X, F, 0.0) + 0.5 * lam * sum(float(np.sum(f * f)) for f in F)


def dense_ratings(y, dims):
    Ymask = np.zeros((dims[0], dims[1]))
    Y = np.zeros((dims[0], dims[1]))
    Ymask[y.idx[0], y.idx[1]] = 1.0
    Y[y.idx[0], y.idx[1]] = y.val
    return Ymask, Y


@pytest.mark.parametrize("mu,lam", [(1.0, 0.0), (0.3, 0.5), (0.0, 0.2)])
def test_joint_loss_and_gradient(mu, lam):
    """The joint objective equals its dense definition, and its gradient (Eq.
    grad-joint-A for every row of A, B and C) equals central finite differences
    of the dense objective."""
    rng, t, y, F = joint_problem(51)
    dims = list(t.dims)
    X = dense_from_coo(t.idx, t.val, dims)
    Ymask, Y = dense_ratings(y, dims)
    assert oracle.joint_loss(y, t, F, mu, lam) == pytest.approx(
        dense_joint_loss(X, Ymask, Y, F, mu, lam), rel=1e-12)
    G = oracle.joint_gradient(y, t, F, mu, lam)
    h = 1e-6
    for m in range(3):
        fd = np.zeros_like(F[m])
        for i in range(F[m].shape[0]):
            for r in range(F[m].shape[1]):
                Fp = [f.copy() for f in F]
                Fm = [f.copy() for f in F]
                Fp[m][i, r] += h
                Fm[m][i, r] -= h
                fd[i, r] = (dense_joint_loss(X, Ymask, Y, Fp, mu, lam)
                            - dense_joint_loss(X, Ymask, Y, Fm, mu, lam)) / (2 * h)
        np.testing.assert_allclose(G[m], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("mu,lam", [(1.0, 0.1), (0.05, 1.0)])
def test_joint_als_rows_are_ridge_least_squares(mu, lam):
    """Each row update of the joint ALS sweep (A, then B with the new A, then C
    with the new A and B) is the minimiser of the joint objective over that row:
    a ridge least-squares problem whose design stacks the row's ratings, every
    cell of the tensor's matching slice (weight sqrt(mu)) and sqrt(lambda) I,
    solved here by numpy's lstsq."""
    rng, t, y, F = joint_problem(52)
    dims = list(t.dims)
    R = F[0].shape[1]
    X = dense_from_coo(t.idx, t.val, dims)
    Ymask, Y = dense_ratings(y, dims)
    st, Fs = oracle.joint_als_sweep(y, t, F, mu, lam)
    assert st == oracle.OK
    cur = [f.copy() for f in F]
    for side in range(3):
        want = np.zeros_like(F[side])
        for row in range(dims[side]):
            rows, rhs = [], []
            if side < 2:
                other = cur[1 - side]
                obs = np.nonzero(Ymask[row] if side == 0 else Ymask[:, row])[0]
                for o in obs:
                    rows.append(other[o])
                    rhs.append(Y[row, o] if side == 0 else Y[o, row])
            # tensor slice: x[row, :, :] against the Khatri-Rao rows of the other two
            o1, o2 = [m for m in range(3) if m != side]
            sl = np.take(X, row, axis=side)  # dims[o1] x dims[o2]
            for p in range(dims[o1]):
                for q in range(dims[o2]):
                    rows.append(np.sqrt(mu) * cur[o1][p] * cur[o2][q])
                    rhs.append(np.sqrt(mu) * sl[p, q])
            for r in range(R):
                e = np.zeros(R)
                e[r] = np.sqrt(lam)
                rows.append(e)
                rhs.append(0.0)
            want[row] = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
        np.testing.assert_allclose(Fs[side], want, rtol=1e-9, atol=1e-10)
        cur[side] = want


def test_joint_als_sweeps_decrease_the_objective():
    """Every block update minimises the objective exactly, so the joint
    objective never increases over ALS sweeps."""
    rng, t, y, F = joint_problem(53, dims=(9, 8, 6), density=0.3, ny=30)
    prev = oracle.joint_loss(y, t, F, 0.7, 0.2)
    for _ in range(6):
        st, F = oracle.joint_als_sweep(y, t, F, 0.7, 0.2)
        assert st == oracle.OK
        cur = oracle.joint_loss(y, t, F, 0.7, 0.2)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_joint_gd_step_is_backtracking_on_the_joint_objective():
    """Each joint GD step reproduces an independent backtracking run on the
    dense joint objective (the rule of the tensor GD step)."""
    rng, t, y, F = joint_problem(54)
    dims = list(t.dims)
    X = dense_from_coo(t.idx, t.val, dims)
    Ymask, Y = dense_ratings(y, dims)
    mu, lam = 0.5, 0.1
    alpha = 0.0
    prev = dense_joint_loss(X, Ymask, Y, F, mu, lam)
    for it in range(6):
        G = oracle.joint_gradient(y, t, F, mu, lam)
        g2 = sum(float(np.sum(g * g)) for g in G)
        a = 1.0 if alpha <= 0 else min(2 * alpha, 1.0)
        for _ in range(100):
            if dense_joint_loss(X, Ymask, Y, [f - a * g for f, g in zip(F, G)], mu, lam) <= prev - 1e-4 * a * g2:
                break
            a *= 0.5
        st, F2, alpha, lo, g2o = oracle.joint_gd_step(y, t, F, mu, lam, alpha)
        assert st == oracle.OK
        assert alpha == a
        assert g2o == pytest.approx(g2, rel=1e-12)
        for m in range(3):
            np.testing.assert_allclose(F2[m], F[m] - alpha * G[m], rtol=1e-14, atol=1e-14)
        assert lo == pytest.approx(dense_joint_loss(X, Ymask, Y, F2, mu, lam), rel=1e-12)
        F, prev = F2, lo


# ---------------------------------------------------------------------------
# Error paths.
# ---------------------------------------------------------------------------


def test_out_of_range_and_duplicates():
    dims = [3, 3, 3]
    bad = oracle.Tensor(np.array([[0, 3], [0, 0], [0, 0]]), [1, 2], dims)
    assert oracle.check_coo(bad) == oracle.ERANGE
    assert oracle.build_csr(bad, 0)[0] == oracle.ERANGE
    neg = oracle.Tensor(np.array([[0, 1], [0, -1], [0, 0]]), [1, 2], dims)
    assert oracle.build_csr(neg, 1)[0] == oracle.ERANGE
    dup = oracle.Tensor(np.array([[1, 2, 1], [0, 0, 0], [2, 2, 2]]), [1, 2, 3], dims)
    for mode in range(3):
        assert oracle.build_csr(dup, mode)[0] == oracle.EDUP


def test_empty_tensor():
    t = oracle.Tensor(np.zeros((3, 0), np.int32), np.zeros(0, np.float32), [4, 3, 2])
    for mode in range(3):
        st, csr = oracle.build_csr(t, mode)
        assert st == oracle.OK and csr["nfib"] == 0
        np.testing.assert_array_equal(csr["fiber_ptr"], np.zeros(t.dims[mode] + 1))
        np.testing.assert_array_equal(csr["nz_ptr"], [0])
        F = [np.ones((d, 2)) for d in t.dims]
        np.testing.assert_array_equal(oracle.mttkrp(t, mode, F), 0.0)
