"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot redo a whole MTTKRP of these tensors in seconds, so each
check is one the oracle computes exactly at any size:

  * sampled rows: 10,000 seeded output rows of every mode plus the three
    heaviest rows (most nonzeros; on the Zipf workloads these hold millions of
    nonzeros and cross many segments, warps and CTAs), computed by the oracle
    with the per-nonzero sum restricted to those rows (FP64), against the
    kernel's rows: normwise 1e-5 for FP32 factors;
  * the cross-mode invariant sum_{o,r} N_n[o,r] F_n[o,r] = <X, [[A,B,C]]> for
    every mode n (all rows), against the oracle's FP64 inner product, within
    the bound 1e-5 ||N_n|| ||F_n|| that the normwise bar implies;
  * BF16 factors (the 1.2B-nonzero workload):
    within 1e-5 of the oracle fed the BF16-rounded factors and within 1e-2 of
    the oracle fed the FP32 ones;
  * one full ALS sweep of the 50M-nonzero workload against the oracle's sweep
    from the same factors (factors 1e-4 normwise, fit within the propagated
    FP32 bound).
"""
import gc

import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1406_4519_gb300 import dfacto, synth

pytestmark = pytest.mark.gpu

SAMPLE = 10_000


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def generate(name):
    wl = bench.WORKLOADS[name]
    dims = wl["dims"]
    if wl["zipf"]:
        idx, val = synth.zipf_tensor(dims, wl["nnz"], wl["zipf"], seed=wl["seed"], device="cuda",
                                     values=wl["values"], R_true=wl["R"])
    else:
        idx, val = synth.uniform_tensor(dims, wl["nnz"], seed=wl["seed"], device="cuda")
    F = synth.normal_factors(dims, wl["R"], seed=wl["seed"] + 1, device="cuda")
    return wl, dims, idx, val, F


def sample_rows(idx_h, mode, dim, seed):
    rng = np.random.default_rng(seed + mode)
    counts = np.bincount(idx_h[mode], minlength=dim)
    heavy = np.argsort(counts)[-3:]
    rows = np.unique(np.concatenate([rng.choice(dim, size=min(SAMPLE, dim), replace=False), heavy]))
    return rows, heavy, counts[heavy]


def check_mttkrp(t, ot, dims, F_ref, idx_h, seed, tol, F_ref2=None, tol2=None):
    inner = oracle.inner(ot, F_ref)
    for mode in range(3):
        N = t.mttkrp(mode)
        torch.cuda.synchronize()
        rows, heavy, heavy_nnz = sample_rows(idx_h, mode, dims[mode], seed)
        got = N[torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        want = oracle.mttkrp_rows(ot, mode, F_ref, rows)
        assert rel(got, want) <= tol, (mode, rel(got, want))
        pos = np.searchsorted(rows, heavy)
        for k, p in enumerate(pos):
            assert rel(got[p], want[p]) <= tol, ("heavy row", mode, int(heavy[k]), int(heavy_nnz[k]))
        if F_ref2 is not None:
            want2 = oracle.mttkrp_rows(ot, mode, F_ref2, rows)
            assert rel(got, want2) <= tol2, (mode, rel(got, want2))
        # cross-mode invariant over all rows
        Fm = torch.as_tensor(F_ref[mode], device="cuda")
        ip = float((N.double() * Fm).sum())
        bound = tol * float(torch.linalg.norm(N.double())) * float(torch.linalg.norm(Fm))
        assert abs(ip - inner) <= bound, (mode, ip, inner, bound)
        del N


def test_zipf50m_mttkrp_sampled_rows_invariant_and_als_sweep():
    wl, dims, idx, val, F = generate("zipf50M")
    idx_h = idx.cpu().numpy()
    val_h = val.cpu().numpy()
    ot = oracle.Tensor(idx_h, val_h, dims)
    F64 = [f.double().cpu().numpy() for f in F]
    t = dfacto.Tensor(idx, val, dims, rank=wl["R"])
    del idx, val
    t.set_factors(F)
    check_mttkrp(t, ot, dims, F64, idx_h, wl["seed"], 1e-5)
    # one ALS sweep, step-wise against the oracle
    st, fit = t.als_iter()
    assert st == dfacto.OK
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, F64)
    after = [f.double().cpu().numpy() for f in t.factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
    nx2 = oracle.norm2(ot)
    ip = oracle.inner(ot, Fo, lam_o)
    nm2 = oracle.model_norm2(dims, Fo, lam_o)
    res = np.sqrt(max(nx2 - 2 * ip + nm2, 1e-300))
    tol_fit = 1e-6 * (nm2 + 2 * abs(ip)) / (2 * res * np.sqrt(nx2)) + 1e-9
    assert abs(fit - fit_o) <= tol_fit, (fit, fit_o, tol_fit)
    del t
    gc.collect()
    torch.cuda.empty_cache()


def test_zipf1200m_mttkrp_fp32_and_bf16_sampled_rows_and_invariant():
    """The 1.2B-nonzero workload (66-bit (o, f, in) keys: the two-run chained
    build) in the launch configuration bench.py times, FP32 and BF16 factors.
    Several minutes: 1.2B-nonzero generation, 19 GB of host copies and the
    oracle's FP64 passes over every nonzero."""
    wl, dims, idx, val, F = generate("zipf1200M")
    idx_h = idx.cpu().numpy()
    val_h = val.cpu().numpy()
    ot = oracle.Tensor(idx_h, val_h, dims)
    F64 = [f.double().cpu().numpy() for f in F]
    t = dfacto.Tensor(idx, val, dims, rank=wl["R"])
    del idx, val
    gc.collect()
    torch.cuda.empty_cache()
    t.set_factors(F)
    check_mttkrp(t, ot, dims, F64, idx_h, wl["seed"], 1e-5)
    del t
    gc.collect()
    torch.cuda.empty_cache()
    # BF16 factors, built from the host copy of the COO
    tb = dfacto.Tensor(torch.from_numpy(idx_h), torch.from_numpy(val_h), dims, rank=wl["R"],
                       factor_dtype=dfacto.BF16)
    tb.set_factors(F)
    Fb = [f.bfloat16().double().cpu().numpy() for f in F]
    check_mttkrp(tb, ot, dims, Fb, idx_h, wl["seed"], 1e-5, F_ref2=F64, tol2=1e-2)
    del tb
    gc.collect()
    torch.cuda.empty_cache()
