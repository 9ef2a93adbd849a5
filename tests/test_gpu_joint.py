"""Joint matrix completion and tensor factorization (Appendix F) on the GPU,
through the C ABI, against the FP64 oracle: the ratings CSR copies bit for
bit, ALS sweeps and GD steps step-wise (the oracle repeats each step from the
factors the GPU held before it), the objective, and the error paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_4519_gb300 import dfacto, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def host(t):
    return t.detach().double().cpu().numpy()


def problem(users=300, items=200, words=150, n_ratings=3000, wpr=4, R=8, seed=61, lam=0.1, mu=0.5,
            dtype=dfacto.F32, line_search=0):
    yidx, yval, idx, val = synth.joint_ratings_reviews(users, items, words, n_ratings, wpr, R,
                                                       seed=seed, device="cuda")
    dims = [users, items, words]
    F = synth.normal_factors(dims, R, seed=seed + 1, device="cuda")
    F = [f * 0.3 for f in F]
    t = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam, factor_dtype=dtype,
                      line_search=line_search)
    t.set_factors(F)
    t.set_ratings(yidx, yval, mu)
    ot = oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), dims)
    oy = oracle.Ratings(yidx.cpu().numpy(), yval.cpu().numpy())
    return t, ot, oy, dims, yidx, yval


def objective_tolerance(oy, ot, F, mu, lam, eps=2e-6):
    """Rounding bound of the objective from FP32 accumulation: eps times the
    magnitudes of its terms (ratings residuals, tensor terms, ridge)."""
    A, B, C = F
    fy = 0.0
    pred = np.einsum("tr,tr->t", A[oy.idx[0]], B[oy.idx[1]])
    fy = float(np.sum(np.abs(oy.val.astype(np.float64)) ** 2 + pred ** 2))
    nx2 = oracle.norm2(ot)
    ip = abs(oracle.inner(ot, F))
    nm2 = oracle.model_norm2(ot.dims, F)
    ridge = lam * sum(float(np.sum(f * f)) for f in F)
    return eps * (fy + mu * (nx2 + 2 * ip + nm2) + ridge) + 1e-9


@pytest.mark.parametrize("side", [0, 1])
def test_ratings_csr_bit_exact(side):
    """Both CSR copies of the ratings equal a lexicographic sort by (row, col)
    of the input, values bit for bit."""
    t, ot, oy, dims, yidx, yval = problem(seed=62)
    v = dfacto.ratings_to_tensors(dfacto.dfacto_get_ratings_csr(t.h, side))
    rows = oy.idx[side].astype(np.int64)
    cols = oy.idx[1 - side].astype(np.int64)
    order = np.lexsort((cols, rows))
    ptr = np.searchsorted(rows[order], np.arange(dims[side] + 1), side="left")
    np.testing.assert_array_equal(v["ptr"].cpu().numpy(), ptr)
    np.testing.assert_array_equal(v["col"].cpu().numpy(), cols[order].astype(np.int32))
    np.testing.assert_array_equal(v["val"].cpu().numpy().view(np.uint32),
                                  oy.val[order].view(np.uint32))


def test_ratings_errors():
    dims = [20, 10, 5]
    idx, val = synth.uniform_tensor(dims, 200, seed=63, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=4, lambda_reg=0.1)
    good = torch.tensor([[0, 1, 2], [0, 0, 3]], dtype=torch.int32, device="cuda")
    y = torch.ones(3, device="cuda")
    bad = torch.tensor([[0, 20, 2], [0, 0, 3]], dtype=torch.int32, device="cuda")
    with pytest.raises(dfacto.DfactoError) as e:
        t.set_ratings(bad, y, 1.0)
    assert e.value.status == dfacto.ERANGE
    dup = torch.tensor([[0, 1, 0], [3, 0, 3]], dtype=torch.int32, device="cuda")
    with pytest.raises(dfacto.DfactoError) as e:
        t.set_ratings(dup, y, 1.0)
    assert e.value.status == dfacto.EDUP
    with pytest.raises(dfacto.DfactoError) as e:
        t.set_ratings(good, y, -1.0)
    assert e.value.status == dfacto.EINVAL
    t.set_ratings(good, y, 1.0)  # valid ratings after refused ones
    t0 = dfacto.Tensor(idx, val, dims, rank=4)  # lambda_reg = 0: ALS refused
    t0.set_ratings(good, y, 1.0)
    with pytest.raises(dfacto.DfactoError) as e:
        t0.joint_als_iter()
    assert e.value.status == dfacto.EINVAL
    big = dfacto.Tensor(idx, val, dims, rank=36)
    with pytest.raises(dfacto.DfactoError) as e:
        big.set_ratings(good, y, 1.0)
    assert e.value.status == dfacto.EINVAL


@pytest.mark.parametrize("R,mu,lam", [(8, 0.5, 0.1), (10, 2.0, 1.0), (32, 0.05, 0.3)])
def test_joint_als_stepwise(R, mu, lam):
    """Three joint ALS sweeps, each against the oracle's sweep from the GPU's
    factors: factors to 1e-4 normwise (FP32 accumulation amplified by the R x R
    solves), the objective within its rounding bound, and the objective never
    rises."""
    t, ot, oy, dims, _, _ = problem(R=R, mu=mu, lam=lam, seed=64 + R)
    prev = None
    for it in range(3):
        before = [host(f) for f in t.factors()]
        obj = t.joint_als_iter()
        st_o, Fo = oracle.joint_als_sweep(oy, ot, before, mu, lam)
        assert st_o == oracle.OK
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-4, (it, m, rel(after[m], Fo[m]))
        want = oracle.joint_loss(oy, ot, Fo, mu, lam)
        assert abs(obj - want) <= objective_tolerance(oy, ot, Fo, mu, lam), (it, obj, want)
        if prev is not None:
            assert obj <= prev * (1 + 1e-6)
        prev = obj


def test_joint_objective_matches_oracle():
    t, ot, oy, dims, _, _ = problem(seed=70)
    F = [host(f) for f in t.factors()]
    got = t.joint_objective()
    want = oracle.joint_loss(oy, ot, F, 0.5, 0.1)
    assert abs(got - want) <= objective_tolerance(oy, ot, F, 0.5, 0.1), (got, want)


@pytest.mark.parametrize("R,mu,lam", [(8, 0.5, 0.1), (12, 3.0, 0.0)])
def test_joint_gd_stepwise(R, mu, lam):
    """Joint GD steps from the GPU's state against the oracle's (Eq.
    grad-joint-A gradients, backtracking on Eq. joint-obj-fn): the accepted
    step is the same, the objective within its rounding bound, the factors to
    1e-5 normwise."""
    t, ot, oy, dims, _, _ = problem(R=R, mu=mu, lam=lam, seed=80 + R)
    alpha_prev = 0.0
    for it in range(4):
        before = [host(f) for f in t.factors()]
        st, obj, alpha = t.joint_gd_iter()
        st_o, Fo, alpha_o, loss_o, g2 = oracle.joint_gd_step(oy, ot, before, mu, lam, alpha_prev)
        assert st == dfacto.OK and st_o == oracle.OK
        assert alpha == alpha_o, (it, alpha, alpha_o)
        assert abs(obj - loss_o) <= objective_tolerance(oy, ot, Fo, mu, lam), (it, obj, loss_o)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-5, (it, m)
        alpha_prev = alpha


def test_joint_gd_exact_line_search_beats_backtracking():
    """With the exact line search each joint GD step lowers the objective at
    least as much as the oracle's backtracking step from the same point (up to
    rounding), and the step it takes reproduces the oracle's objective there."""
    mu, lam = 0.5, 0.1
    t, ot, oy, dims, _, _ = problem(R=8, mu=mu, lam=lam, seed=90, line_search=dfacto.EXACT)
    prev = t.joint_objective()
    for it in range(4):
        before = [host(f) for f in t.factors()]
        st, obj, alpha = t.joint_gd_iter()
        assert st == dfacto.OK and alpha > 0
        G = oracle.joint_gradient(oy, ot, before, mu, lam)
        stepped = [before[m] - alpha * G[m] for m in range(3)]
        want = oracle.joint_loss(oy, ot, stepped, mu, lam)
        tol = objective_tolerance(oy, ot, stepped, mu, lam)
        assert abs(obj - want) <= tol, (it, obj, want)
        st_b, Fb, ab, lb, _ = oracle.joint_gd_step(oy, ot, before, mu, lam, 0.0)
        assert obj <= lb + tol
        assert obj < prev
        prev = obj


def test_joint_als_bf16_factors_within_bar():
    """BF16 factor storage: one joint ALS sweep within 1e-2 normwise of the
    oracle's FP64 sweep from the same (BF16-rounded) start."""
    mu, lam = 0.5, 0.1
    t, ot, oy, dims, _, _ = problem(R=16, mu=mu, lam=lam, seed=95, dtype=dfacto.BF16)
    before = [host(f) for f in t.factors()]
    t.joint_als_iter()
    st_o, Fo = oracle.joint_als_sweep(oy, ot, before, mu, lam)
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-2, m
