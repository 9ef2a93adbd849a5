"""dfacto_mttkrp_noalloc: the MTTKRP for callers that may not allocate device
memory (their memory belongs to another allocator, or allocating at that point
could block or fail).  It must give what dfacto_mttkrp gives, call after call,
while keeping its scratch in the library's fixed device array.

This file is collected last on purpose: the entry point's first call on a
device looks up the array's address, and the test must pass both in a fresh
process and after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1406_4519_gb300 import dfacto, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the normwise bar of every FP32 MTTKRP test


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("kind,R", [("zipf", 32), ("zipf", 10), ("uniform", 16)])
def test_noalloc_matches_mttkrp_twice(kind, R):
    if kind == "zipf":
        dims = [3000, 2000, 1000]
        idx, val = synth.zipf_tensor(dims, 400000, [1.2, 1.2, 1.2], seed=41 + R, device="cuda",
                                     values="cp", R_true=8)
    else:
        dims = [4000, 50, 30]  # most mode-0 rows are empty
        idx, val = synth.uniform_tensor(dims, 20000, seed=43, device="cuda")
    F = synth.normal_factors(dims, R, seed=7, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=R)
    t.set_factors(F)
    ot = oracle.Tensor(idx.cpu().numpy(), val.cpu().numpy(), dims)
    Fh = [f.double().cpu().numpy() for f in F]
    for mode in range(3):
        want = t.mttkrp(mode)
        exact = torch.from_numpy(oracle.mttkrp(ot, mode, Fh))  # FP64 definition
        csr = dfacto.dfacto_get_csr(t.h, mode)
        F_in, F_f = F[(mode + 1) % 3], F[(mode + 2) % 3]
        for call in range(2):  # the second call reuses the scratch the first left behind
            out = torch.full((dims[mode], R), float("nan"), device="cuda")
            dfacto.dfacto_mttkrp_noalloc(csr, F_in, F_f, R, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel(out, want) <= TOL, (mode, call)
            assert rel(out, exact) <= TOL, (mode, call)


def test_noalloc_rejects_problems_beyond_its_scratch():
    """The size check happens on the host before any launch: a view claiming
    the largest accepted nonzero count (2^31 - 2^16) needs far more than
    16 MiB and is refused with ENOMEM; one nonzero more is not a valid view."""
    dims = [50, 40, 30]
    idx, val = synth.uniform_tensor(dims, 2000, seed=3, device="cuda")
    t = dfacto.Tensor(idx, val, dims, rank=8)
    csr = dfacto.dfacto_get_csr(t.h, 0)
    big = dfacto.dfacto_csr_view()
    ctypes.pointer(big)[0] = csr
    big.nnz = 2 ** 31 - 2 ** 16
    F = synth.normal_factors(dims, 8, seed=1, device="cuda")
    out = torch.zeros(dims[0], 8, device="cuda")
    with pytest.raises(dfacto.DfactoError) as e:
        dfacto.dfacto_mttkrp_noalloc(big, F[1], F[2], 8, out)
    assert e.value.status == dfacto.ENOMEM
    big.nnz = 2 ** 31 - 2 ** 16 + 1
    with pytest.raises(dfacto.DfactoError) as e:
        dfacto.dfacto_mttkrp_noalloc(big, F[1], F[2], 8, out)
    assert e.value.status == dfacto.EINVAL
