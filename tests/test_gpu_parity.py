"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (written per test): CSR arrays bit-exact; FP32 MTTKRP within 1e-5
normwise relative error; BF16-factor MTTKRP within 1e-2 of the oracle fed the
FP32 factors and within 1e-5 of the oracle fed the BF16-rounded factors; ALS and
GD step-wise (the oracle starts from the GPU's state) within the tolerances
derived in the test docstrings.
"""
import numpy as np
import pytest
import torch

import oracle
from golden_io import read
from paper_1406_4519_gb300 import dfacto, synth

pytestmark = pytest.mark.gpu

MTTKRP_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def host(t):
    return t.detach().double().cpu().numpy()


def as_oracle(idx, val, dims):
    return oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), dims)


def make(dims, nnz, R, seed, dtype=dfacto.F32, seg=0, vec=0, zipf=None, values="uniform", walk=0):
    if zipf is None:
        idx, val = synth.uniform_tensor(dims, nnz, seed=seed, device="cuda")
    else:
        idx, val = synth.zipf_tensor(dims, nnz, zipf, seed=seed, device="cuda", values=values)
    F = synth.normal_factors(dims, R, seed=seed + 1, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=R, factor_dtype=dtype, seg_nnz=seg, vec=vec, walk=walk)
    t.set_factors(F)
    return t, idx, val, F


# ---------------------------------------------------------------------------
# CSR construction (bit-exact).
# ---------------------------------------------------------------------------


def check_csr(t, idx, val, dims):
    ot = as_oracle(idx, val, dims)
    for mode in range(3):
        st, want = oracle.build_csr(ot, mode)
        assert st == oracle.OK
        got = t.csr(mode)
        assert got["nfib"] == want["nfib"], mode
        for key in ("fiber_ptr", "fiber_idx", "nz_ptr", "nz_idx"):
            np.testing.assert_array_equal(got[key].cpu().numpy(), want[key], err_msg="%s %d" % (key, mode))
        # values are moved, never changed: compare the bits
        np.testing.assert_array_equal(got["nz_val"].cpu().numpy().view(np.uint32),
                                      want["nz_val"].view(np.uint32))


def test_csr_appendix_d_bit_exact():
    g = read("appD_example.txt")
    idx = torch.tensor(g["S"].T.astype(np.int32)).contiguous()
    val = torch.tensor(g["v"][:, 0].astype(np.float32))
    dims = [int(x) for x in g["dims"][0]]
    t = dfacto.Tensor(idx.cuda(), val.cuda(), dims, rank=2)
    want = read("appD_csr_mode1.txt")
    got = t.csr(0)
    for key in ("fiber_ptr", "fiber_idx", "nz_ptr", "nz_idx", "nz_val"):
        np.testing.assert_array_equal(got[key].cpu().numpy(), want[key].reshape(-1), err_msg=key)
    check_csr(t, idx, val, dims)


@pytest.mark.parametrize("dims,nnz,seed", [([200, 150, 100], 10000, 1),
                                           ([37, 1, 53], 1200, 2),
                                           ([1, 1, 1], 1, 3),
                                           ([5000, 3, 7], 20000, 4),
                                           ([3, 5000, 7], 20000, 8),
                                           ([7, 3, 5000], 20000, 9)])
def test_csr_uniform_bit_exact(dims, nnz, seed):
    """The chain of sorts starts at the mode whose later modes need the
    fewest digit passes: the three 5000-long cases start it at each mode."""
    idx, val = synth.uniform_tensor(dims, nnz, seed=seed, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=4)
    check_csr(t, idx, val, dims)


def test_csr_zipf_bit_exact():
    dims = [3000, 2000, 1000]
    idx, val = synth.zipf_tensor(dims, 200000, [1.2, 1.2, 1.2], seed=5, device="cuda",
                                 values="lognormal")
    t = dfacto.Tensor(idx, val, dims, rank=4)
    check_csr(t, idx, val, dims)


def test_csr_64_bit_keys_bit_exact():
    """21 + 21 + 22 = 64 key bits: the widest keys of the one-run sort, whose
    chained modes rotate all 64 bits."""
    dims = [2 ** 21, 2 ** 21, 2 ** 22]
    idx, val = synth.zipf_tensor(dims, 50000, [1.2, 1.1, 1.3], seed=7, device="cuda",
                                 values="lognormal")
    t = dfacto.Tensor(idx, val, dims, rank=2)
    check_csr(t, idx, val, dims)


def test_csr_wide_keys_bit_exact():
    """Coordinates needing more than 64 key bits take the two-run sort."""
    dims = [2 ** 23, 2 ** 22, 2 ** 21]  # 23 + 22 + 21 = 66 bits
    idx, val = synth.zipf_tensor(dims, 50000, [1.1, 1.3, 1.2], seed=6, device="cuda",
                                 values="lognormal")
    t = dfacto.Tensor(idx, val, dims, rank=2)
    check_csr(t, idx, val, dims)


# ---------------------------------------------------------------------------
# MTTKRP.
# ---------------------------------------------------------------------------


def test_mttkrp_appendix_d_exact():
    g = read("appD_example.txt")
    idx = torch.tensor(g["S"].T.astype(np.int32)).contiguous().cuda()
    val = torch.tensor(g["v"][:, 0].astype(np.float32)).cuda()
    t = dfacto.Tensor(idx, val, [2, 3, 3], rank=2)
    t.set_factors([torch.ones(2, 2).cuda(), torch.tensor(g["B"], dtype=torch.float32).cuda(),
                   torch.tensor(g["C"], dtype=torch.float32).cuda()])
    np.testing.assert_array_equal(t.mttkrp(0).cpu().numpy(), g["M"])


@pytest.mark.parametrize("walk", [1, 2])
@pytest.mark.parametrize("R", [1, 3, 8, 10, 16, 32, 64])
@pytest.mark.parametrize("seg", [32, 256])
def test_mttkrp_uniform(R, seg, walk):
    dims = [50, 40, 30]
    t, idx, val, F = make(dims, 20000, R, seed=100 + R, seg=seg, walk=walk)
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    for mode in range(3):
        err = rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, Fh))
        assert err <= MTTKRP_TOL, (mode, err)


@pytest.mark.parametrize("walk", [1, 2])
@pytest.mark.parametrize("vec", [1, 2, 4, 8])
def test_mttkrp_lane_layouts(vec, walk):
    dims = [300, 200, 100]
    t, idx, val, F = make(dims, 30000, 32, seed=200 + vec, seg=64, vec=vec, walk=walk)
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    for mode in range(3):
        assert rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, Fh)) <= MTTKRP_TOL


@pytest.mark.parametrize("walk", [1, 2])
@pytest.mark.parametrize("seg", [32, 128, 1024])
def test_mttkrp_power_law_rows_span_many_ctas(seg, walk):
    """Zipf heads put ~10% of all nonzeros in one row and long fibers across
    many segments and CTAs: the carry merge must still be exact in order."""
    dims = [2000, 1000, 500]
    t, idx, val, F = make(dims, 300000, 16, seed=300, seg=seg, zipf=[1.2, 1.2, 1.2],
                          values="cp", walk=walk)
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    for mode in range(3):
        assert rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, Fh)) <= MTTKRP_TOL


@pytest.mark.parametrize("dims,nnz", [([2000, 2000, 2000], 100000), ([20000, 20000, 20000], 40000)])
def test_preferential_attachment_csr_mttkrp_and_sweep(dims, nnz):
    """The paper's synthetic sets (Sec. 5): dense-ish (50 nonzeros per index,
    rich-get-richer heads) and sparse (nnz = 2I, singleton fibers) draws; CSR
    bit-exact, MTTKRP within the FP32 bar and one ALS sweep step-wise."""
    idx, val = synth.preferential_attachment_tensor(dims, nnz, seed=17, device="cuda")
    F = synth.normal_factors(dims, 10, seed=18, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=10)
    t.set_factors(F)
    check_csr(t, idx, val, dims)
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    for mode in range(3):
        assert rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, Fh)) <= MTTKRP_TOL, mode
    st, fit = t.als_iter()
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, Fh)
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
    assert abs(fit - fit_o) <= 1e-5


def test_mttkrp_single_row_and_single_fiber():
    """All nonzeros in one output row (mode 0) and in one fiber (i, k fixed)."""
    J = 5000
    idx = torch.stack([torch.zeros(J, dtype=torch.int32), torch.arange(J, dtype=torch.int32),
                       torch.full((J,), 3, dtype=torch.int32)]).cuda()
    val = torch.rand(J, generator=torch.Generator().manual_seed(1)).cuda()
    dims = [4, J, 5]
    F = synth.normal_factors(dims, 8, seed=9, device="cuda")
    for seg, walk in ((32, 1), (256, 1), (32, 2), (256, 2)):
        t = dfacto.Tensor(idx, val, dims, rank=8, seg_nnz=seg, walk=walk)
        t.set_factors(F)
        ot = as_oracle(idx, val, dims)
        for mode in range(3):
            assert rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, [host(f) for f in F])) <= MTTKRP_TOL


def test_mttkrp_empty_tensor_and_empty_rows():
    dims = [7, 6, 5]
    t = dfacto.Tensor(torch.zeros(3, 0, dtype=torch.int32).cuda(), torch.zeros(0).cuda(), dims, rank=4)
    t.set_factors(synth.normal_factors(dims, 4, seed=1, device="cuda"))
    for mode in range(3):
        out = torch.full((dims[mode], 4), 7.0, device="cuda")
        assert torch.all(t.mttkrp(mode, out) == 0)
    # sparse rows: most output rows have no nonzeros and must come back as 0
    idx = torch.tensor([[0, 999], [1, 2], [3, 4]], dtype=torch.int32).cuda()
    val = torch.tensor([2.0, 3.0]).cuda()
    dims = [1000, 10, 10]
    t = dfacto.Tensor(idx, val, dims, rank=4)
    F = synth.normal_factors(dims, 4, seed=2, device="cuda")
    t.set_factors(F)
    out = torch.full((1000, 4), float("nan"), device="cuda")
    got = host(t.mttkrp(0, out))
    want = oracle.mttkrp(as_oracle(idx, val, dims), 0, [host(f) for f in F])
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("R", [32, 10])
def test_mttkrp_is_bitwise_deterministic(R):
    """Repeated calls give the same bits, and so do the two walks (at R = 10
    both run on the padded copies)."""
    dims = [2000, 1000, 500]
    t, idx, val, F = make(dims, 200000, R, seed=400, seg=32, zipf=[1.2, 1.2, 1.2], walk=1)
    t2 = dfacto.Tensor(idx, val, dims, rank=R, seg_nnz=32, walk=2)
    t2.set_factors(F)
    for mode in range(3):
        a = t.mttkrp(mode).clone()
        b = t.mttkrp(mode).clone()
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
        # both walks add the same terms in the same order
        c2 = t2.mttkrp(mode).clone()
        assert torch.equal(a.view(torch.int32), c2.view(torch.int32))


@pytest.mark.parametrize("walk", [1, 2])
@pytest.mark.parametrize("R", [8, 10, 16, 32])
def test_mttkrp_bf16_factors(R, walk):
    dims = [400, 300, 200]
    idx, val = synth.zipf_tensor(dims, 60000, [1.2, 1.2, 1.2], seed=500 + R, device="cuda",
                                 values="uniform")
    F = synth.normal_factors(dims, R, seed=R, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=R, factor_dtype=dfacto.BF16, walk=walk)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    F32 = [host(f) for f in F]
    Fbf = [host(f.to(torch.bfloat16)) for f in F]  # the values the GPU actually holds
    for mode in range(3):
        got = host(t.mttkrp(mode))
        assert rel(got, oracle.mttkrp(ot, mode, F32)) <= 1e-2
        assert rel(got, oracle.mttkrp(ot, mode, Fbf)) <= MTTKRP_TOL


@pytest.mark.parametrize("dtype", [dfacto.F32, dfacto.BF16])
def test_mttkrp_padded_ranks(dtype):
    """Ranks that are not a multiple of four walk zero-padded FP32 copies of the
    factors at the rank rounded up (the default lane width); the result, copied
    back to R columns, is the oracle's within the MTTKRP bar for every such rank
    from 3 to 31, on power-law rows that span many CTAs (small segments), and
    so is the unpadded walk that an explicit lane width keeps."""
    dims = [900, 700, 500]
    idx, val = synth.zipf_tensor(dims, 80000, [1.2, 1.1, 1.3], seed=77, device="cuda",
                                 values="uniform")
    ot = as_oracle(idx, val, dims)
    for R in (3, 5, 6, 7, 9, 10, 11, 13, 14, 15, 18, 22, 31):
        F = synth.normal_factors(dims, R, seed=100 + R, device="cuda")
        Fh = [host(f.to(torch.bfloat16)) if dtype == dfacto.BF16 else host(f) for f in F]
        for vec in (0, 1):
            t = dfacto.Tensor(idx, val, dims, rank=R, factor_dtype=dtype, seg_nnz=64, vec=vec)
            t.set_factors(F)
            # the lane width in use: four columns of the padded copies, or the one asked for
            assert list(t.info().vec) == [4 if vec == 0 else 1] * 3, (R, vec)
            for mode in range(3):
                got = host(t.mttkrp(mode))
                assert got.shape == (dims[mode], R)
                assert rel(got, oracle.mttkrp(ot, mode, Fh)) <= MTTKRP_TOL, (R, vec, mode)


# ---------------------------------------------------------------------------
# ALS, fit and GD (step-wise: the oracle starts from the GPU's state).
# ---------------------------------------------------------------------------


def test_als_stepwise_c1_config():
    """200 x 150 x 100, 10,000 uniform nonzeros, U(0,1) values, R = 10, five
    sweeps from seeded N(0,1) factors.  Each sweep: the oracle repeats it from the
    factors the GPU held before it.  Factors agree to 1e-4 normwise (FP32 MTTKRP
    error 1e-6 amplified by the R x R solves), lambda to 1e-4 relative, and the fit
    to 1e-5 absolute."""
    dims = [200, 150, 100]
    R = 10
    t, idx, val, F = make(dims, 10000, R, seed=14064520)
    ot = as_oracle(idx, val, dims)
    for it in range(5):
        before = [host(f) for f in t.factors()]
        st, fit = t.als_iter()
        assert st == dfacto.OK
        st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, before)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-4, (it, m)
        np.testing.assert_allclose(t.lam(), lam_o, rtol=1e-4)
        assert abs(fit - fit_o) <= 1e-5, (it, fit, fit_o)


def test_als_exact_rank_tensor_reaches_fit():
    """A tensor that is exactly rank 3 on every cell (dense, as COO): ALS from a
    random start reaches fit >= 0.9999 (the invariant the oracle is pinned to)."""
    rng = np.random.default_rng(19)
    dims = [20, 18, 16]
    truth = [rng.standard_normal((d, 3)) for d in dims]
    X = np.einsum("ir,jr,kr->ijk", *truth)
    idx = torch.tensor(np.array(np.nonzero(np.ones_like(X)), dtype=np.int32)).cuda()
    val = torch.tensor(X.reshape(-1).astype(np.float32)).cuda()
    t = dfacto.Tensor(idx, val, dims, rank=3)
    t.set_factors([torch.tensor(rng.standard_normal((d, 3)), dtype=torch.float32).cuda() for d in dims])
    fit = 0.0
    for _ in range(300):
        st, fit = t.als_iter()
        if fit >= 0.99999:
            break
    assert fit >= 0.9999


def test_fit_matches_oracle():
    dims = [120, 90, 60]
    t, idx, val, F = make(dims, 8000, 6, seed=600)
    lam = [0.5 + 0.1 * r for r in range(6)]
    dfacto.dfacto_set_lambda(t.h, lam)
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    lam = np.array(lam)
    want = oracle.fit(ot, Fh, lam)
    assert abs(t.fit() - want) <= fit_tolerance(ot, Fh, lam)


def fit_tolerance(ot, Fh, lam, eps=1e-6):
    """|d fit| from relative errors eps in the FP32-accumulated <X, Xhat> and
    ||Xhat||^2: fit = 1 - res/||X||, res^2 = ||X||^2 - 2<X,Xhat> + ||Xhat||^2, so
    d fit ~ eps (||Xhat||^2 + 2 |<X,Xhat>|) / (2 res ||X||)."""
    nx2 = oracle.norm2(ot)
    ip = oracle.inner(ot, Fh, lam)
    nm2 = oracle.model_norm2(ot.dims, Fh, lam)
    res = np.sqrt(max(nx2 - 2 * ip + nm2, 1e-300))
    return eps * (nm2 + 2 * abs(ip)) / (2 * res * np.sqrt(nx2)) + 1e-9


def test_als_singular_gamma_reports_and_matches_pinv():
    """Duplicated factor columns make every Gamma of the sweep exactly singular
    (Eq. kr-pseudo): the status is ESINGULAR, and the factors, lambda and fit
    after the sweep equal the oracle's sweep, which takes the pseudo-inverse
    (minimum-norm) solution of each mode in FP64."""
    dims = [30, 20, 10]
    idx, val = synth.uniform_tensor(dims, 3000, seed=7, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(30, 2, device="cuda", generator=g)
    b = torch.randn(20, 1, device="cuda", generator=g)
    c = torch.randn(10, 1, device="cuda", generator=g)
    F = [A, torch.cat([b, b], 1), torch.cat([c, c], 1)]
    t = dfacto.Tensor(idx, val, dims, rank=2)
    t.set_factors(F)
    st, fit = t.als_iter()
    assert st == dfacto.ESINGULAR
    ot = as_oracle(idx, val, dims)
    Fh = [host(f) for f in F]
    st_m, _, _ = oracle.als_mode_update(ot, 0, Fh)
    assert st_m == oracle.ESINGULAR
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, Fh)
    assert st_o == oracle.ESINGULAR
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
        # the minimum-norm solution keeps the duplicated columns equal
        np.testing.assert_allclose(after[m][:, 0], after[m][:, 1], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(t.lam(), lam_o, rtol=1e-4)
    assert abs(fit - fit_o) <= fit_tolerance(ot, Fo, lam_o), (fit, fit_o)


@pytest.mark.parametrize("R", [4, 8])
def test_als_singular_gamma_rank_deficient_start_stepwise(R):
    """A start whose factors have rank R/2 (each column repeated): Gamma is
    singular in every mode of the first sweep; three sweeps step-wise against
    the oracle's pseudo-inverse path (factors and lambda to 1e-4)."""
    dims = [60, 40, 30]
    idx, val = synth.zipf_tensor(dims, 5000, [1.2, 1.1, 1.3], seed=77, device="cuda", values="cp",
                                 R_true=4)
    g = torch.Generator(device="cuda").manual_seed(78)
    F = [torch.randn(d, R // 2, device="cuda", generator=g).repeat(1, 2) for d in dims]
    t = dfacto.Tensor(idx, val, dims, rank=R)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    for it in range(3):
        before = [host(f) for f in t.factors()]
        st, fit = t.als_iter()
        st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, before)
        assert st == (dfacto.ESINGULAR if st_o == oracle.ESINGULAR else dfacto.OK), (it, st, st_o)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-4, (it, m)
        np.testing.assert_allclose(t.lam(), lam_o, rtol=1e-4, atol=1e-12)
        assert abs(fit - fit_o) <= fit_tolerance(ot, Fo, lam_o), (it, fit, fit_o)


@pytest.mark.parametrize("lam_reg,R", [(0.1, 8), (3.0, 10), (0.5, 32)])
def test_als_regularized_stepwise(lam_reg, R):
    """Regularized ALS (Appendix B, Eq. tensorapprx-ref-sol: F = N (Gamma +
    lambda_reg I)^-1): four sweeps step-wise against the oracle's regularized
    sweep from the factors the GPU held before each one."""
    dims = [150, 120, 90]
    t, idx, val, F = make(dims, 9000, R, seed=900 + R, zipf=[1.2, 1.2, 1.2], values="cp")
    t = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam_reg)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    for it in range(4):
        before = [host(f) for f in t.factors()]
        st, fit = t.als_iter()
        assert st == dfacto.OK
        st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, before, lam_reg)
        assert st_o == oracle.OK
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-4, (it, m)
        np.testing.assert_allclose(t.lam(), lam_o, rtol=1e-4)
        assert abs(fit - fit_o) <= fit_tolerance(ot, Fo, lam_o), (it, fit, fit_o)


def test_als_regularized_singular_gamma_needs_no_pinv():
    """The duplicated-column start that makes Gamma singular: with lambda_reg > 0
    Gamma + lambda_reg I is positive definite, so the sweep takes the Cholesky
    path (status OK) and equals the oracle's regularized sweep."""
    dims = [30, 20, 10]
    idx, val = synth.uniform_tensor(dims, 3000, seed=7, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(30, 2, device="cuda", generator=g)
    b = torch.randn(20, 1, device="cuda", generator=g)
    c = torch.randn(10, 1, device="cuda", generator=g)
    F = [A, torch.cat([b, b], 1), torch.cat([c, c], 1)]
    t = dfacto.Tensor(idx, val, dims, rank=2, lambda_reg=0.25)
    t.set_factors(F)
    st, fit = t.als_iter()
    assert st == dfacto.OK
    ot = as_oracle(idx, val, dims)
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, [host(f) for f in F], 0.25)
    assert st_o == oracle.OK
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
    np.testing.assert_allclose(t.lam(), lam_o, rtol=1e-4)


def ray_tolerance(ot, F, G, alpha, lam_reg, eps=2e-6):
    """Rounding bound of f(alpha) = 1/2 (||X||^2 - 2 P(alpha) + Q(alpha)) (+ ridge)
    evaluated, as the line search does, from terms taken at the starting point:
    P(alpha) = sum_S (-alpha)^|S| T_S with T_S = <X, [[F or G per mode]]>, and
    Q(alpha) = sum_rs prod_n (M_n)_rs with M_n = F^T F - alpha (F^T G + G^T F)
    + alpha^2 G^T G.  Each term carries a relative error eps from FP32
    accumulation, so |d f| <= eps (2 sum_S alpha^|S| |T_S| + Q_abs) / 2 with Q_abs
    the same sum over absolute values."""
    import itertools
    T = 0.0
    for S in itertools.product([0, 1], repeat=3):
        T += alpha ** sum(S) * abs(oracle.inner(ot, [G[m] if S[m] else F[m] for m in range(3)]))
    M = [np.abs(F[m].T @ F[m]) + alpha * np.abs(F[m].T @ G[m] + G[m].T @ F[m])
         + alpha ** 2 * np.abs(G[m].T @ G[m]) for m in range(3)]
    Qabs = float(np.sum(M[0] * M[1] * M[2]))
    ridge = lam_reg * sum(float(np.sum(np.abs(f) ** 2)) + alpha ** 2 * float(np.sum(g * g))
                          for f, g in zip(F, G))
    return eps * (2 * T + Qabs + ridge) / 2 + 1e-9


def ray_slope_tolerance(ot, F, G, alpha, lam_reg, eps=2e-6):
    """Rounding bound of f'(alpha) formed from the same FP32-accumulated terms
    as ray_tolerance: the derivative of each term's magnitude along the ray,
    times eps."""
    import itertools
    T = 0.0
    for S in itertools.product([0, 1], repeat=3):
        k = sum(S)
        if k:
            T += k * alpha ** (k - 1) * abs(oracle.inner(ot, [G[m] if S[m] else F[m] for m in range(3)]))
    a0 = [np.abs(F[m].T @ F[m]) for m in range(3)]
    a1 = [np.abs(F[m].T @ G[m] + G[m].T @ F[m]) for m in range(3)]
    a2 = [np.abs(G[m].T @ G[m]) for m in range(3)]
    M = [a0[m] + alpha * a1[m] + alpha ** 2 * a2[m] for m in range(3)]
    dM = [a1[m] + 2 * alpha * a2[m] for m in range(3)]
    dQ = float(np.sum(dM[0] * M[1] * M[2] + M[0] * dM[1] * M[2] + M[0] * M[1] * dM[2]))
    ridge = lam_reg * sum(2 * float(np.sum(np.abs(f * g))) + 2 * alpha * float(np.sum(g * g))
                          for f, g in zip(F, G))
    return eps * (2 * T + dQ + ridge) / 2


@pytest.mark.parametrize("R", [8, 10, 32])
@pytest.mark.parametrize("lam_reg", [0.0, 0.5])
def test_gd_exact_line_search_stepwise(lam_reg, R):
    """GD with the exact line search (line_search = 1), each step from the GPU's
    state against the oracle's exact step (the global minimiser of the degree-6
    polynomial f(theta - alpha grad), evaluated from the definition): alpha agrees
    within the bound a rounding error of f' moves a minimum (|d f'| / f''), the
    objective within ray_tolerance, the factors to 1e-5 normwise plus what the
    alpha difference moves them.  Every step lowers the objective, by at least
    as much as the backtracking step would from the same point."""
    dims = [120, 90, 60]
    t, idx, val, F = make(dims, 8000, R, seed=800 + R, zipf=[1.2, 1.1, 1.3], values="cp")
    t = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam_reg, line_search=dfacto.EXACT)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    prev = oracle.loss(ot, [host(f) for f in F], lam_reg)
    for it in range(4):
        before = [host(f) for f in t.factors()]
        st, loss, alpha = t.gd_iter()
        st_o, Fo, alpha_o, loss_o, g2 = oracle.gd_step_exact(ot, before, lam_reg)
        assert st == dfacto.OK and st_o == oracle.OK
        G = oracle.gd_gradient(ot, before, lam_reg)
        c = oracle.gd_ray_poly(ot, before, G, lam_reg)
        curv = sum(k * (k - 1) * c[k] * alpha_o ** (k - 2) for k in range(2, 7))
        assert curv > 0
        tol_a = 2 * ray_slope_tolerance(ot, before, G, alpha_o, lam_reg) / curv + 1e-12 * alpha_o
        assert abs(alpha - alpha_o) <= tol_a, (it, alpha, alpha_o, tol_a)
        tol = ray_tolerance(ot, before, G, alpha_o, lam_reg) + 0.5 * curv * tol_a ** 2
        assert abs(loss - loss_o) <= tol, (it, loss, loss_o, tol)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            shift = tol_a * np.linalg.norm(G[m]) / max(np.linalg.norm(Fo[m]), 1e-300)
            assert rel(after[m], Fo[m]) <= 1e-5 + shift, (it, m)
        st_b, Fb, alpha_b, loss_b, _ = oracle.gd_step(ot, before, 0.0, lam_reg)
        assert loss_o <= loss_b + 1e-12 * abs(loss_b)
        assert loss_o < prev
        prev = loss_o


@pytest.mark.parametrize("R", [8, 10, 12])
@pytest.mark.parametrize("lam_reg", [0.0, 0.5])
def test_gd_stepwise(lam_reg, R):
    """Each GD step from the GPU's state: the accepted alpha is the oracle's (the
    Armijo decisions coincide unless a trial sits within rounding of the
    threshold), the objective agrees within ray_tolerance and the new factors
    to 1e-5 normwise."""
    dims = [120, 90, 60]
    t, idx, val, F = make(dims, 8000, R, seed=700 + R)
    t = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam_reg)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    alpha_prev = 0.0
    for it in range(4):
        before = [host(f) for f in t.factors()]
        st, loss, alpha = t.gd_iter()
        st_o, Fo, alpha_o, loss_o, g2 = oracle.gd_step(ot, before, alpha_prev, lam_reg)
        assert st == dfacto.OK and st_o == oracle.OK
        assert alpha == alpha_o, (it, alpha, alpha_o)
        G = oracle.gd_gradient(ot, before, lam_reg)
        tol = ray_tolerance(ot, before, G, alpha_o, lam_reg)
        assert abs(loss - loss_o) <= tol, (it, loss, loss_o, tol)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-5
        alpha_prev = alpha


@pytest.mark.parametrize("R", [36, 128])
def test_large_ranks_mttkrp_als_gd(R):
    """Ranks above 32 (up to the largest accepted, 128) take the generic row
    solve and store, four columns per lane in the merges and the fix-up, and an
    R x R Gamma of up to 128 x 128: the MTTKRP of every mode is the oracle's
    within the MTTKRP bar, a regularized ALS sweep from the GPU's state agrees
    with the oracle's to 1e-4 normwise, and two GD steps agree as in the
    step-wise GD test (same accepted alpha, objective within ray_tolerance,
    factors to 1e-5)."""
    dims = [300, 250, 200]
    lam = 1.0
    idx, val = synth.zipf_tensor(dims, 20000, [1.2, 1.1, 1.3], seed=900 + R, device="cuda",
                                 values="uniform")
    F = synth.normal_factors(dims, R, seed=901 + R, device="cuda")
    ot = as_oracle(idx, val, dims)
    t = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam)
    t.set_factors(F)
    Fh = [host(f) for f in F]
    for mode in range(3):
        assert rel(host(t.mttkrp(mode)), oracle.mttkrp(ot, mode, Fh)) <= MTTKRP_TOL, mode
    before = [host(f) for f in t.factors()]
    st, fit = t.als_iter()
    assert st in (dfacto.OK, dfacto.ESINGULAR)
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, before, lam)
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
    g = dfacto.Tensor(idx, val, dims, rank=R, lambda_reg=lam)
    g.set_factors(F)
    alpha_prev = 0.0
    for it in range(2):
        before = [host(f) for f in g.factors()]
        st, loss, alpha = g.gd_iter()
        st_o, Fo, alpha_o, loss_o, g2 = oracle.gd_step(ot, before, alpha_prev, lam)
        assert st == dfacto.OK and st_o == oracle.OK
        assert alpha == alpha_o, (it, alpha, alpha_o)
        G = oracle.gd_gradient(ot, before, lam)
        assert abs(loss - loss_o) <= ray_tolerance(ot, before, G, alpha_o, lam), (it, loss, loss_o)
        after = [host(f) for f in g.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-5, (it, m)
        alpha_prev = alpha


# ---------------------------------------------------------------------------
# Error paths on the device.
# ---------------------------------------------------------------------------


def test_out_of_range_and_duplicate_coordinates():
    dims = [4, 4, 4]
    idx = torch.tensor([[0, 4], [0, 0], [0, 0]], dtype=torch.int32).cuda()
    with pytest.raises(dfacto.DfactoError) as e:
        dfacto.Tensor(idx, torch.ones(2).cuda(), dims, rank=2)
    assert e.value.status == dfacto.ERANGE
    idx = torch.tensor([[1, 2, 1], [0, 0, 0], [3, 3, 3]], dtype=torch.int32).cuda()
    with pytest.raises(dfacto.DfactoError) as e:
        dfacto.Tensor(idx, torch.ones(3).cuda(), dims, rank=2)
    assert e.value.status == dfacto.EDUP


def test_build_out_of_device_memory_is_enomem_and_the_device_stays_usable():
    """A tensor whose dense arrays need ~1 TiB (a 2^31 - 1 long mode at
    R = 128): the build's allocation is refused, dfacto_build returns ENOMEM
    after releasing what it had allocated, and the device keeps working: a
    small tensor built afterwards sweeps like the oracle, and the same huge
    request is refused the same way a second time."""
    huge = [2 ** 31 - 1, 2, 2]
    idx = torch.zeros(3, 1, dtype=torch.int32, device="cuda")
    val = torch.ones(1, device="cuda")
    for _ in range(2):
        with pytest.raises(dfacto.DfactoError) as e:
            dfacto.Tensor(idx, val, huge, rank=128)
        assert e.value.status == dfacto.ENOMEM
        torch.cuda.synchronize()  # no error left on the context
        dims = [40, 30, 20]
        sidx, sval = synth.uniform_tensor(dims, 2000, seed=12, device="cuda")
        F = synth.normal_factors(dims, 4, seed=13, device="cuda")
        t = dfacto.Tensor(sidx, sval, dims, rank=4)
        t.set_factors(F)
        st, fit = t.als_iter()
        assert st in (dfacto.OK, dfacto.ESINGULAR)
        ot = as_oracle(sidx, sval, dims)
        st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, [f.double().cpu().numpy() for f in F])
        got = [f.double().cpu().numpy() for f in t.factors()]
        for m in range(3):
            assert np.linalg.norm(got[m] - Fo[m]) <= 1e-4 * np.linalg.norm(Fo[m]), m


def test_host_inputs_give_the_same_csr():
    dims = [60, 50, 40]
    idx, val = synth.uniform_tensor(dims, 5000, seed=11, device="cpu")
    t_host = dfacto.Tensor(idx, val, dims, rank=4)
    t_dev = dfacto.Tensor(idx.cuda(), val.cuda(), dims, rank=4)
    for mode in range(3):
        a, b = t_host.csr(mode), t_dev.csr(mode)
        for key in ("fiber_ptr", "fiber_idx", "nz_ptr", "nz_idx", "nz_val"):
            assert torch.equal(a[key], b[key])


@pytest.mark.parametrize("case", ["uniform10k", "zipf1M"])
def test_bf16_als_fit_within_1e4_of_fp64_run(case):
    """BF16 factor storage (FP32 accumulation, FP64 R x R solve and fit): five
    ALS sweeps from the same start as the FP64 oracle's five sweeps; after
    every sweep the fits differ by at most 1e-4 (the BF16 target)."""
    if case == "uniform10k":
        dims, R = [200, 150, 100], 10
        idx, val = synth.uniform_tensor(dims, 10000, seed=14064520, device="cuda")
    else:
        dims, R = [20000, 10000, 5000], 16
        idx, val = synth.zipf_tensor(dims, 1_000_000, [1.2, 1.2, 1.2], seed=61, device="cuda",
                                     values="cp", R_true=R)
    F = synth.normal_factors(dims, R, seed=62, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=R, factor_dtype=dfacto.BF16)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    Fo = [host(f) for f in F]
    for it in range(5):
        st, fit = t.als_iter()
        assert st == dfacto.OK
        st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, Fo)
        assert abs(fit - fit_o) <= 1e-4, (case, it, fit, fit_o)


def test_gd_step_with_large_gradients():
    """Factors scaled by 64 make the gradients ~1e13-1e14, so <X, [[GA, GB, GC]]>
    (three gradient factors per nonzero) exceeds the FP32 range unless the
    gradients are rescaled: the step still matches the oracle (alpha identical,
    objective within ray_tolerance, factors 1e-5) and everything stays finite."""
    dims = [100, 80, 60]
    R = 8
    idx, val = synth.uniform_tensor(dims, 5000, seed=711, device="cuda")
    F = [64.0 * f for f in synth.normal_factors(dims, R, seed=712, device="cuda")]
    t = dfacto.Tensor(idx, val, dims, rank=R)
    t.set_factors(F)
    ot = as_oracle(idx, val, dims)
    before = [host(f) for f in t.factors()]
    G = oracle.gd_gradient(ot, before)
    assert max(np.abs(g).max() for g in G) > 1e13
    st, loss, alpha = t.gd_iter()
    st_o, Fo, alpha_o, loss_o, g2 = oracle.gd_step(ot, before, 0.0)
    assert st == dfacto.OK and st_o == oracle.OK
    assert np.isfinite(loss) and alpha == alpha_o, (loss, alpha, alpha_o)
    tol = ray_tolerance(ot, before, G, alpha_o, 0.0)
    assert abs(loss - loss_o) <= tol, (loss, loss_o, tol)
    after = [host(f) for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-5


def test_gd_stepwise_bf16_factors():
    """GD with BF16 factor storage, step-wise from the GPU's (BF16) state: the
    accepted alpha is the oracle's and the new factors (rounded to BF16 on the
    GPU) are within the BF16 bar, 1e-2 normwise, of the oracle's FP64 step."""
    dims = [120, 90, 60]
    R = 8
    t, idx, val, F = make(dims, 8000, R, seed=730, dtype=dfacto.BF16)
    ot = as_oracle(idx, val, dims)
    alpha_prev = 0.0
    for it in range(3):
        before = [host(f) for f in t.factors()]
        st, loss, alpha = t.gd_iter()
        st_o, Fo, alpha_o, loss_o, g2 = oracle.gd_step(ot, before, alpha_prev)
        assert st == dfacto.OK and st_o == oracle.OK
        assert alpha == alpha_o, (it, alpha, alpha_o)
        after = [host(f) for f in t.factors()]
        for m in range(3):
            assert rel(after[m], Fo[m]) <= 1e-2, (it, m)
        alpha_prev = alpha
