"""The preferential-attachment generator (the paper's synthetic sets, Sec. 5).

Each axis is a Polya urn: index i is drawn with probability proportional to
1 + its earlier draws.  For two indices the count of index 0 after T draws is
then uniform on {0, ..., T} (the Beta(1,1)-binomial law of a Polya urn started
with one ball of each colour), which pins the rule; the tensor itself must
have exactly nnz distinct in-range coordinates and be reproducible."""
import numpy as np
import torch

from paper_1406_4519_gb300 import synth


def test_two_index_urn_count_is_uniform():
    T, runs = 12, 3000
    counts = np.zeros(T + 1)
    for r in range(runs):
        axis = synth._AttachmentAxis(2, synth.generator(1000 + r, "cpu"), "cpu")
        drawn = axis.extend(T)
        counts[int((drawn == 0).sum())] += 1
    expected = runs / (T + 1)
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    # 12 degrees of freedom: P(chi2 > 32.9) = 0.001
    assert chi2 < 32.9, (chi2, counts)


def test_extend_continues_the_process():
    """A second extension continues the first (its copies may point into the
    first piece): indices stay in range and the history is kept in order."""
    axis = synth._AttachmentAxis(5, synth.generator(7, "cpu"), "cpu")
    a = axis.extend(50)
    b = axis.extend(50)
    assert a.min() >= 0 and a.max() < 5 and b.min() >= 0 and b.max() < 5
    assert torch.equal(axis.drawn, torch.cat([a, b]))


def test_tensor_unique_in_range_and_seeded():
    dims = [300, 200, 100]
    idx, val = synth.preferential_attachment_tensor(dims, 20000, seed=3)
    assert idx.dtype == torch.int32 and val.dtype == torch.float32
    assert idx.shape == (3, 20000) and val.shape == (20000,)
    for m in range(3):
        assert int(idx[m].min()) >= 0 and int(idx[m].max()) < dims[m]
    key = (idx[0].long() * dims[1] + idx[1].long()) * dims[2] + idx[2].long()
    assert key.unique().numel() == 20000
    assert float(val.min()) >= 0.0 and float(val.max()) < 1.0
    idx2, val2 = synth.preferential_attachment_tensor(dims, 20000, seed=3)
    assert torch.equal(idx, idx2) and torch.equal(val, val2)


def test_rich_get_richer():
    """With 100 nonzeros per index on average the busiest index holds several
    times the mean (uniform coordinates stay within ~1.5x); with far more
    indices than nonzeros nearly every (o, f) fiber holds one nonzero, as the
    paper observes for these sets."""
    d, nnz = 1000, 100000
    idx, _ = synth.preferential_attachment_tensor([d, d, d], nnz, seed=4)
    top = int(torch.bincount(idx[0].long(), minlength=d).max())
    uidx, _ = synth.uniform_tensor([d, d, d], nnz, seed=4)
    utop = int(torch.bincount(uidx[0].long(), minlength=d).max())
    assert top > 4 * nnz / d and utop < 1.5 * nnz / d
    d2 = 100000
    idx, _ = synth.preferential_attachment_tensor([d2, d2, d2], 2 * d2, seed=5)
    fibers = (idx[0].long() * d2 + idx[2].long()).unique().numel()
    assert fibers > 0.99 * 2 * d2
