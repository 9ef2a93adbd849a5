"""Seeded synthetic sparse 3-way tensors and factor initialisations.

This module only draws inputs: coordinates, values and starting factors.  It
contains none of the factorization's arithmetic and imports nothing else from
this package, so both the CUDA library's tests and the CPU oracle can be fed
from it.  Everything runs in plain PyTorch on the device it is asked for
(``cpu`` or ``cuda``); a given (recipe, seed, device) always yields the same
tensor.

Recipes (the shapes and distributions of the workloads this library is
measured on; the paper's real datasets are not available, these stand in):

* ``uniform_tensor``  -- unique coordinates drawn uniformly, values U(0,1).
* ``zipf_tensor``     -- per-mode Zipf(s) coordinates (index 0 the most
  frequent), deduplicated to exactly ``nnz`` unique coordinates by redrawing;
  values either a planted CP model plus Gaussian noise, lognormal(0,1) or U(0,1).
* ``preferential_attachment_tensor`` -- coordinates drawn one nonzero after
  another, each axis index with probability proportional to (1 + the number of
  nonzeros already at that index), values U(0,1).
* ``normal_factors``  -- N(0,1) starting factors.
* ``joint_ratings_reviews`` -- the joint model's inputs (Appendix F): a users x
  items ratings matrix and a users x items x words review tensor on the rated
  pairs, from planted factors.

Coordinates are returned as int32 [3, nnz] (rows i, j, k), values as float32,
in a seeded random order (never pre-sorted).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import torch

__all__ = [
    "generator", "zipf_cdf", "draw_zipf", "unique_coords", "uniform_tensor",
    "zipf_tensor", "preferential_attachment_tensor", "normal_factors", "batch_job_specs",
    "poisson_arrivals", "joint_ratings_reviews",
]


def generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    return g


def zipf_cdf(n: int, s: float) -> torch.Tensor:
    """CDF table of Zipf(s) truncated to ranks 1..n, as float64 on the CPU.

    Rank r has probability proportional to r**-s; rank r maps to index r-1.
    """
    w = torch.arange(1, n + 1, dtype=torch.float64).pow_(-float(s))
    c = torch.cumsum(w, 0)
    c /= c[-1].clone()
    c[-1] = 1.0
    return c


def draw_zipf(m: int, cdf: torch.Tensor, g: torch.Generator, device) -> torch.Tensor:
    u = torch.rand(m, dtype=torch.float64, generator=g, device=device)
    idx = torch.searchsorted(cdf, u, right=True)
    return idx.clamp_(max=cdf.numel() - 1)


def _first_occurrences(cols: List[torch.Tensor]) -> torch.Tensor:
    """Positions (ascending) of the first occurrence of each distinct tuple.

    ``cols`` are int64 key columns, most significant first; the tuple order is
    found with stable sorts from the least significant column up.
    """
    n = cols[0].numel()
    order = torch.arange(n, device=cols[0].device)
    for c in reversed(cols):
        order = order[torch.argsort(c[order], stable=True)]
    first = torch.ones(n, dtype=torch.bool, device=cols[0].device)
    if n > 1:
        diff = torch.zeros(n - 1, dtype=torch.bool, device=cols[0].device)
        for c in cols:
            sc = c[order]
            diff |= sc[1:] != sc[:-1]
        first[1:] = diff
    return torch.sort(order[first]).values


def _key_columns(ijk: torch.Tensor, dims: Sequence[int]) -> List[torch.Tensor]:
    I, J, K = (int(d) for d in dims)
    if I * J * K < (1 << 62):
        return [(ijk[0] * J + ijk[1]) * K + ijk[2]]
    return [ijk[0], ijk[1] * K + ijk[2]]


def unique_coords(dims: Sequence[int], nnz: int, sampler, g: torch.Generator, device,
                  max_rounds: int = 400) -> torch.Tensor:
    """Draw coordinates with ``sampler(m) -> int64 [3, m]`` until ``nnz`` are unique.

    Duplicates are redrawn from the same distribution; the first ``nnz`` distinct
    coordinates in draw order are kept.  Returns int64 [3, nnz].
    """
    cap = int(dims[0]) * int(dims[1]) * int(dims[2])
    if nnz > cap:
        raise ValueError("nnz %d exceeds the %d cells of the tensor" % (nnz, cap))
    pool = torch.empty((3, 0), dtype=torch.int64, device=device)
    for _ in range(max_rounds):
        need = nnz - pool.shape[1]
        if need <= 0:
            break
        m = int(need * 1.05) + 64
        pool = torch.cat([pool, sampler(m)], dim=1)
        keep = _first_occurrences(_key_columns(pool, dims))
        pool = pool[:, keep]
    if pool.shape[1] < nnz:
        raise RuntimeError("could not draw %d unique coordinates" % nnz)
    return pool[:, :nnz]


def _shuffle(ijk: torch.Tensor, g: torch.Generator, device) -> torch.Tensor:
    perm = torch.randperm(ijk.shape[1], generator=g, device=device)
    return ijk[:, perm]


def uniform_tensor(dims: Sequence[int], nnz: int, seed: int, device="cpu"
                   ) -> Tuple[torch.Tensor, torch.Tensor]:
    """Unique uniform coordinates, values U(0,1)."""
    device = torch.device(device)
    g = generator(seed, device)

    def sampler(m):
        return torch.stack([torch.randint(0, int(d), (m,), generator=g, device=device)
                            for d in dims])

    ijk = _shuffle(unique_coords(dims, nnz, sampler, g, device), g, device)
    val = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    return ijk.to(torch.int32).contiguous(), val.contiguous()


def normal_factors(dims: Sequence[int], R: int, seed: int, device="cpu",
                   dtype=torch.float32) -> List[torch.Tensor]:
    """Three N(0,1) factor matrices dims[m] x R (row-major)."""
    device = torch.device(device)
    g = generator(seed, device)
    return [torch.randn(int(d), R, generator=g, device=device, dtype=torch.float64)
            .to(dtype).contiguous() for d in dims]


def zipf_tensor(dims: Sequence[int], nnz: int, exponents: Sequence[float], seed: int,
                device="cpu", values: str = "cp", R_true: int = 32,
                noise: float = 0.01, chunk: int = 1 << 22
                ) -> Tuple[torch.Tensor, torch.Tensor]:
    """Per-mode Zipf coordinates, exactly ``nnz`` unique.

    values = "cp":        x = sum_r a_ir b_jr c_kr over planted N(0,1) factors of
                          rank ``R_true``, plus N(0, (noise * rms(x))^2);
             "lognormal": x = exp(N(0,1));
             "uniform":   x ~ U(0,1).
    """
    device = torch.device(device)
    g = generator(seed, device)
    cdfs = [zipf_cdf(int(d), s).to(device) for d, s in zip(dims, exponents)]

    def sampler(m):
        return torch.stack([draw_zipf(m, c, g, device) for c in cdfs])

    ijk = _shuffle(unique_coords(dims, nnz, sampler, g, device), g, device)
    if values == "cp":
        gp = generator(seed + 7919, device)
        planted = [torch.randn(int(d), R_true, generator=gp, device=device,
                               dtype=torch.float64) for d in dims]
        x = torch.empty(nnz, dtype=torch.float64, device=device)
        for s0 in range(0, nnz, chunk):
            s1 = min(nnz, s0 + chunk)
            x[s0:s1] = (planted[0][ijk[0, s0:s1]] * planted[1][ijk[1, s0:s1]]
                        * planted[2][ijk[2, s0:s1]]).sum(1)
        rms = float(torch.sqrt(torch.mean(x * x))) if nnz else 0.0
        x += noise * rms * torch.randn(nnz, generator=g, device=device, dtype=torch.float64)
        val = x.to(torch.float32)
    elif values == "lognormal":
        val = torch.exp(torch.randn(nnz, generator=g, device=device, dtype=torch.float64)
                        ).to(torch.float32)
    elif values == "uniform":
        val = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    else:
        raise ValueError(values)
    return ijk.to(torch.int32).contiguous(), val.contiguous()


class _AttachmentAxis:
    """One axis of the preferential-attachment process.

    Draw t (0-based) takes index i with probability (c_i + 1) / (t + d), c_i
    being the number of earlier draws at i: with probability d / (t + d) a
    uniform index, otherwise the index of a uniformly chosen earlier draw (an
    index with c_i earlier draws is copied with probability c_i / (t + d)).
    ``extend(m)`` continues the process by m draws and returns their indices.
    """

    def __init__(self, d: int, g: torch.Generator, device):
        self.d, self.g, self.device = int(d), g, device
        self.drawn = torch.empty(0, dtype=torch.int64, device=device)

    def extend(self, m: int) -> torch.Tensor:
        t0 = self.drawn.numel()
        t = torch.arange(t0, t0 + m, device=self.device, dtype=torch.int64)
        u = torch.rand(m, generator=self.g, device=self.device, dtype=torch.float64)
        fresh = u * (t + self.d).to(torch.float64) < self.d
        uni = torch.randint(0, self.d, (m,), generator=self.g, device=self.device)
        src = (torch.rand(m, generator=self.g, device=self.device, dtype=torch.float64)
               * t.to(torch.float64)).to(torch.int64)
        src = torch.minimum(src, (t - 1).clamp(min=0))
        # a copy points at an earlier draw: earlier batches are resolved, draws
        # of this batch are followed until they reach a uniform one
        old = ~fresh & (src < t0)
        val = torch.where(fresh, uni, torch.zeros_like(uni))
        if t0 > 0:
            val = torch.where(old, self.drawn[src.clamp(max=t0 - 1)], val)
        local = torch.where(fresh | old, t, src) - t0
        while True:
            nxt = local[local]
            if torch.equal(nxt, local):
                break
            local = nxt
        out = val[local]
        self.drawn = torch.cat([self.drawn, out])
        return out


def preferential_attachment_tensor(dims: Sequence[int], nnz: int, seed: int, device="cpu"
                                   ) -> Tuple[torch.Tensor, torch.Tensor]:
    """Skewed coordinates from a preferential-attachment process, values U(0,1).

    Nonzeros are added one after another and the axes draw independently, so
    the probability of (i, j, k) is the product of per-axis probabilities, each
    proportional to 1 + the number of nonzeros already at that index (the +1
    lets unused indices start).  Draws continue until ``nnz`` distinct
    coordinates exist; repeated coordinates still count.  Returns (int32
    [3, nnz] in a seeded random order, float32 [nnz]).
    """
    device = torch.device(device)
    g = generator(seed, device)
    axes = [_AttachmentAxis(int(d), g, device) for d in dims]

    def sampler(m):
        return torch.stack([a.extend(m) for a in axes])

    ijk = _shuffle(unique_coords(dims, nnz, sampler, g, device), g, device)
    val = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    return ijk.to(torch.int32).contiguous(), val.contiguous()


def batch_job_specs(n_jobs: int, seed: int, dim_lo: int = 1000, dim_hi: int = 200000,
                    nnz_median: float = 5e5, nnz_sigma: float = 1.0, nnz_lo: int = 10000,
                    nnz_hi: int = 5000000, ranks: Sequence[int] = (8, 16, 32)):
    """Shapes of independent jobs: dims log-uniform in [dim_lo, dim_hi], nnz
    lognormal with the given median and sigma clipped to [nnz_lo, nnz_hi], R
    uniform over ``ranks``.  Returns a list of dicts (dims, nnz, R, seed)."""
    g = generator(seed, "cpu")
    specs = []
    for t in range(n_jobs):
        u = torch.rand(3, generator=g, dtype=torch.float64)
        dims = [int(round(math.exp(math.log(dim_lo) + float(x) *
                                   (math.log(dim_hi) - math.log(dim_lo))))) for x in u]
        z = float(torch.randn(1, generator=g, dtype=torch.float64))
        nnz = int(min(max(math.exp(math.log(nnz_median) + nnz_sigma * z), nnz_lo), nnz_hi))
        nnz = min(nnz, dims[0] * dims[1] * dims[2] // 2)
        R = int(ranks[int(torch.randint(0, len(ranks), (1,), generator=g))])
        specs.append(dict(dims=dims, nnz=nnz, R=R, seed=int(seed * 1000003 + t)))
    return specs


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> List[float]:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    g = generator(seed, "cpu")
    u = torch.rand(n, generator=g, dtype=torch.float64).clamp_(min=1e-300)
    gaps = -torch.log(u) / float(rate_per_s)
    return torch.cumsum(gaps, 0).tolist()


def joint_ratings_reviews(users: int, items: int, words: int, n_ratings: int, words_per_review: int,
                          R: int, seed: int, device="cpu", noise: float = 0.1):
    """Inputs of the joint matrix completion + tensor factorization model: the
    real review data is not available, so ratings and reviews come from planted
    factors A (users x R), B (items x R), C (words x R) with N(0, 1/R) entries.

    Rated (user, item) pairs: ``n_ratings`` unique pairs, users and items each
    Zipf(1.1) (a few users rate a lot, a few items are rated a lot); rating
    y = 3 + 5 a_i . b_j + N(0, noise^2).  Each rated pair carries a review of
    ``words_per_review`` words drawn Zipf(1.2) over the vocabulary (repeats
    dropped), with value x = sum_r a_ir b_jr c_kr + N(0, noise^2).

    Returns (yidx int32 [2, n], yval float32 [n], idx int32 [3, nnz],
    val float32 [nnz]); pairs and nonzeros in seeded random order.
    """
    device = torch.device(device)
    g = generator(seed, device)
    s = 1.0 / math.sqrt(R)
    A = torch.randn(users, R, generator=g, device=device) * s
    B = torch.randn(items, R, generator=g, device=device) * s
    C = torch.randn(words, R, generator=g, device=device) * s
    cu, ci = zipf_cdf(users, 1.1).to(device), zipf_cdf(items, 1.1).to(device)

    def pair_sampler(m):
        return torch.stack([draw_zipf(m, cu, g, device), draw_zipf(m, ci, g, device),
                            torch.zeros(m, dtype=torch.int64, device=device)])

    pairs = unique_coords([users, items, 1], n_ratings, pair_sampler, g, device)[:2]
    pairs = pairs[:, torch.randperm(pairs.shape[1], generator=g, device=device)]
    yval = 3.0 + 5.0 * (A[pairs[0]] * B[pairs[1]]).sum(1)
    yval = yval + noise * torch.randn(yval.shape[0], generator=g, device=device)
    cw = zipf_cdf(words, 1.2).to(device)
    rep_i = pairs[0].repeat_interleave(words_per_review)
    rep_j = pairs[1].repeat_interleave(words_per_review)
    wk = draw_zipf(rep_i.shape[0], cw, g, device)
    ijk = torch.stack([rep_i, rep_j, wk])
    keep = _first_occurrences(_key_columns(ijk, [users, items, words]))
    ijk = _shuffle(ijk[:, keep], g, device)
    val = (A[ijk[0]] * B[ijk[1]] * C[ijk[2]]).sum(1)
    val = val + noise * torch.randn(val.shape[0], generator=g, device=device)
    return (pairs.to(torch.int32).contiguous(), yval.to(torch.float32).contiguous(),
            ijk.to(torch.int32).contiguous(), val.to(torch.float32).contiguous())

