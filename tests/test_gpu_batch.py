"""Batches (dfacto_batch_*): many independent jobs advanced together.

A batch must give every job what the job gives alone: its MTTKRPs equal the
single-tensor MTTKRP and the FP64 oracle within the FP32 bar (1e-5 normwise;
the summation splits differ, so not bitwise), and its ALS sweeps follow the
oracle step by step (factors 1e-4 normwise, lambda 1e-4, fit 1e-5: the bars of
the single-tensor step-wise test).  A graph replay must equal the same sweep
issued launch by launch bitwise (same kernels, same order).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_4519_gb300 import dfacto, synth

pytestmark = pytest.mark.gpu

MTTKRP_TOL = 1e-5

# Jobs of mixed rank, factor type, size and skew: ranks 8/16/32 share three
# rank classes of the batched kernel, R = 10 and R = 40 take their own walk
# launch, R = 40 and 64 the row passes for R > 32, three jobs are BF16, one has
# an empty mode-0 majority and one has a single nonzero.
JOB_SPECS = [
    dict(dims=[300, 200, 100], nnz=20000, R=8, seed=101),
    dict(dims=[1200, 90, 400], nnz=30000, R=16, seed=102, zipf=[1.2, 1.1, 1.3]),
    dict(dims=[500, 500, 500], nnz=60000, R=32, seed=103, zipf=[1.2, 1.2, 1.2]),
    dict(dims=[80, 60, 40], nnz=5000, R=10, seed=104),
    dict(dims=[4000, 50, 30], nnz=8000, R=16, seed=105),
    dict(dims=[700, 300, 200], nnz=40000, R=32, seed=106, dtype=dfacto.BF16),
    dict(dims=[250, 250, 250], nnz=15000, R=8, seed=107, dtype=dfacto.BF16, zipf=[1.1, 1.1, 1.1]),
    dict(dims=[20, 30, 10], nnz=1, R=8, seed=108, twin_only=True),
    dict(dims=[900, 400, 300], nnz=45000, R=32, seed=109),
    # R > 32: the row passes of the tiled kernels through the N Gamma^-1 buffer
    dict(dims=[600, 300, 200], nnz=30000, R=40, seed=110),
    dict(dims=[400, 350, 300], nnz=25000, R=64, seed=111, dtype=dfacto.BF16),
]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def host(t):
    return t.detach().double().cpu().numpy()


def make_job(spec):
    dims = spec["dims"]
    if spec.get("zipf"):
        idx, val = synth.zipf_tensor(dims, spec["nnz"], spec["zipf"], seed=spec["seed"], device="cuda")
    else:
        idx, val = synth.uniform_tensor(dims, spec["nnz"], seed=spec["seed"], device="cuda")
    F = synth.normal_factors(dims, spec["R"], seed=spec["seed"] + 7, device="cuda")
    dtype = spec.get("dtype", dfacto.F32)

    def build():
        t = dfacto.Tensor(idx, val, dims, rank=spec["R"], factor_dtype=dtype)
        t.set_factors(F)
        return t

    return build, idx, val, F


@pytest.fixture(scope="module")
def jobs():
    return [make_job(s) for s in JOB_SPECS]


def test_batch_mttkrp_matches_single_and_oracle(jobs):
    tensors = [build() for build, _, _, _ in jobs]
    twins = [build() for build, _, _, _ in jobs]
    b = dfacto.Batch(tensors)
    classes = b.classes()
    assert sum(c.n_jobs for c in classes) == len(JOB_SPECS)
    for mode in range(3):
        got = b.mttkrp(mode)
        b.sync()
        for j, (spec, (_, idx, val, F)) in enumerate(zip(JOB_SPECS, jobs)):
            want = twins[j].mttkrp(mode)
            torch.cuda.synchronize()
            assert torch.isfinite(got[j]).all()
            assert rel(host(got[j]), host(want)) <= MTTKRP_TOL, (j, mode)
            if spec.get("dtype", dfacto.F32) == dfacto.F32:
                ot = oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), spec["dims"])
                ref = oracle.mttkrp(ot, mode, [host(f) for f in F])
                assert rel(host(got[j]), ref) <= MTTKRP_TOL, (j, mode)
    b.close()


def test_batch_als_stepwise_against_oracle(jobs):
    """Three sweeps (the first issued launch by launch, the second captured and
    replayed, the third replayed): each FP32 job follows the oracle from the
    factors it held before the sweep; each BF16 job follows its twin run alone
    (factors 1e-3: both round to BF16 from FP32 values that differ by ~1e-6),
    and so does the one-nonzero job, whose rank-1 factors make Gamma singular
    (both sides take the same pseudo-inverse path)."""
    tensors = [build() for build, _, _, _ in jobs]
    twins = [build() for build, _, _, _ in jobs]
    b = dfacto.Batch(tensors)
    ots = [oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), s["dims"])
           for s, (_, idx, val, _) in zip(JOB_SPECS, jobs)]
    for it in range(3):
        before = [[host(f) for f in t.factors()] for t in tensors]
        st, fits = b.als_iter()
        assert st in (dfacto.OK, dfacto.ESINGULAR)
        for j, spec in enumerate(JOB_SPECS):
            after = [host(f) for f in tensors[j].factors()]
            if spec.get("dtype", dfacto.F32) == dfacto.F32 and not spec.get("twin_only"):
                st_o, Fo, lam_o, fit_o = oracle.als_sweep(ots[j], before[j])
                for m in range(3):
                    assert rel(after[m], Fo[m]) <= 1e-4, (it, j, m)
                np.testing.assert_allclose(tensors[j].lam(), lam_o, rtol=1e-4, atol=1e-12)
                assert abs(fits[j] - fit_o) <= 1e-5, (it, j, fits[j], fit_o)
            else:
                st_t, fit_t = twins[j].als_iter()
                tw = [host(f) for f in twins[j].factors()]
                for m in range(3):
                    assert rel(after[m], tw[m]) <= 1e-3, (it, j, m)
                assert abs(fits[j] - fit_t) <= 1e-4, (it, j)
                # restart the twin from the batch's state (step-wise, no drift)
                twins[j].set_factors([torch.tensor(x, dtype=torch.float32, device="cuda") for x in after])
    b.close()


def _run(build_jobs, use_graph, sweeps=4):
    tensors = [build() for build, _, _, _ in build_jobs]
    b = dfacto.Batch(tensors, use_graph=use_graph, autotune=False)
    fits = None
    for _ in range(sweeps):
        st, fits = b.als_iter()
        assert st in (dfacto.OK, dfacto.ESINGULAR)
    out = [[host(f) for f in t.factors()] for t in tensors]
    lams = [t.lam() for t in tensors]
    b.close()
    return out, lams, fits


def test_graph_replay_equals_eager_bitwise(jobs):
    eager, lam_e, fit_e = _run(jobs, use_graph=False)
    graph, lam_g, fit_g = _run(jobs, use_graph=True)
    for j in range(len(JOB_SPECS)):
        for m in range(3):
            np.testing.assert_array_equal(eager[j][m], graph[j][m], err_msg="job %d mode %d" % (j, m))
        np.testing.assert_array_equal(lam_e[j], lam_g[j])
    np.testing.assert_array_equal(fit_e, fit_g)


def test_set_factors_after_capture_takes_effect(jobs):
    """Changing one job's factors between sweeps: the next sweep starts from
    them (the captured graph is dropped and the sweep re-issued)."""
    sub = jobs[:3]
    tensors = [build() for build, _, _, _ in sub]
    b = dfacto.Batch(tensors)
    for _ in range(3):
        b.als_iter()
    fresh = synth.normal_factors(JOB_SPECS[1]["dims"], JOB_SPECS[1]["R"], seed=5, device="cuda")
    tensors[1].set_factors(fresh)
    before = [host(f) for f in tensors[1].factors()]
    st, fits = b.als_iter()
    idx, val = sub[1][1], sub[1][2]
    ot = oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), JOB_SPECS[1]["dims"])
    st_o, Fo, lam_o, fit_o = oracle.als_sweep(ot, before)
    after = [host(f) for f in tensors[1].factors()]
    for m in range(3):
        assert rel(after[m], Fo[m]) <= 1e-4, m
    assert abs(fits[1] - fit_o) <= 1e-5
    b.close()


def test_destroy_hands_factors_back(jobs):
    tensors = [build() for build, _, _, _ in jobs[:4]]
    b = dfacto.Batch(tensors)
    b.als_iter()
    inside = [[host(f) for f in t.factors()] for t in tensors]
    b.close()
    for j, t in enumerate(tensors):
        for m, f in enumerate(t.factors()):
            np.testing.assert_array_equal(host(f), inside[j][m])
        st, fit = t.als_iter()  # the job keeps working alone
        assert st in (dfacto.OK, dfacto.ESINGULAR) and np.isfinite(fit)


def test_job_destroyed_first_makes_batch_refuse(jobs):
    tensors = [build() for build, _, _, _ in jobs[:3]]
    b = dfacto.Batch(tensors)
    dfacto.dfacto_destroy(tensors[0].h)
    tensors[0].h = None
    with pytest.raises(dfacto.DfactoError) as e:
        b.als_iter()
    assert e.value.status == dfacto.EINVAL
    b.close()


def test_handle_in_two_batches_is_refused(jobs):
    tensors = [build() for build, _, _, _ in jobs[:2]]
    b = dfacto.Batch(tensors)
    with pytest.raises(dfacto.DfactoError) as e:
        dfacto.Batch(tensors[1:])
    assert e.value.status == dfacto.EINVAL
    b.close()


def test_autotuner_picks_a_candidate(jobs):
    tensors = [build() for build, _, _, _ in jobs]
    b = dfacto.Batch(tensors, autotune=True)
    for c in b.classes():
        assert c.seg_nnz % 32 == 0 and c.vec * c.lanes >= c.rank
        if c.rank in (8, 16, 32) and c.nnz > 0:
            assert c.tuned_ms > 0 and c.vec in (4, 8) and c.seg_nnz in (64, 128, 256)
    b.close()
