"""Seeded synthetic inputs for set-similarity self-joins.

This module holds random-number plumbing only: it draws collections of
integer token sets in CSR form (``offsets`` int64[N+1], ``tokens`` int32[]),
probe queries, arrival times and batched-job specifications.  It contains
none of the join's arithmetic (no similarity, no bitmap, no filter), so the
CPU oracle and the CUDA path can both consume it without sharing method code.

Shapes follow the paper's experimental collections (Section 5, Table 5):
token frequencies are Zipf-like (Section 5, Fig. 4) and collections range
from 1e5 to 1e7 sets.  Tokens inside a set are distinct and strictly
increasing, because a set has no repeated elements (Section 2.1).

Sampling recipe (fixed so that every run with the same seed is identical):
* set sizes: ``uniform(lo, hi)`` inclusive, or ``lognormal(mu, sigma)``
  rounded to the nearest integer and clipped to ``[lo, hi]``; sizes are
  also capped at the universe size;
* tokens: token id = Zipf rank - 1, ranks drawn from the finite Zipf law
  ``P(k) ~ k^-s`` over ``1..U`` by inverse CDF; each set keeps drawing until
  it holds ``size`` distinct tokens (the first ``size`` distinct ones in draw
  order), then is sorted ascending;
* planted near-duplicates (optional): a fraction of the sets is replaced by
  a copy of a random earlier set with ``k`` in ``[0, max_edits]`` random
  token edits (delete / insert / substitute), so that joins at high
  thresholds have non-empty results.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


# ----------------------------------------------------------------------------
# Collection specification
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class CollectionSpec:
    n_sets: int
    universe: int
    zipf_s: float
    size_dist: tuple  # ("uniform", lo, hi) or ("lognormal", mu, sigma, lo, hi)
    seed: int = 0
    planted_frac: float = 0.0
    planted_max_edits: int = 3

    def describe(self) -> str:
        d = self.size_dist
        if d[0] == "uniform":
            sz = f"sizes U[{d[1]},{d[2]}]"
        else:
            sz = f"sizes lognormal(mu={d[1]},sigma={d[2]}) clip [{d[3]},{d[4]}]"
        s = (f"N={self.n_sets}, Zipf(s={self.zipf_s}) over {self.universe} tokens, "
             f"{sz}, seed {self.seed}")
        if self.planted_frac > 0:
            s += (f", {self.planted_frac:.0%} planted near-duplicates "
                  f"(0..{self.planted_max_edits} edits)")
        return s


# The paper-shaped workloads (sizes of the experiments, synthetic content).
def spec_small(planted: bool = False) -> CollectionSpec:
    """10,000 sets, Zipf(1.0) over 5,000 tokens, sizes U[5,50], seed 0."""
    return CollectionSpec(10_000, 5_000, 1.0, ("uniform", 5, 50), seed=0,
                          planted_frac=0.05 if planted else 0.0)


def spec_1m(seed: int = 0, planted: bool = False) -> CollectionSpec:
    """1,000,000 sets, Zipf(1.1) over 200,000, sizes lognormal(2.3,0.6) in [1,500]."""
    return CollectionSpec(1_000_000, 200_000, 1.1, ("lognormal", 2.3, 0.6, 1, 500),
                          seed=seed, planted_frac=0.05 if planted else 0.0)


def spec_10m(seed: int = 0) -> CollectionSpec:
    """10,000,000 sets, Zipf(1.0) over 1,000,000, sizes lognormal(2.0,0.8) in [1,1000]."""
    return CollectionSpec(10_000_000, 1_000_000, 1.0, ("lognormal", 2.0, 0.8, 1, 1000),
                          seed=seed)


def spec_resident_2m(seed: int = 0) -> CollectionSpec:
    """2,000,000 sets, Zipf(1.1) over 300,000, sizes lognormal(2.3,0.6) in [1,500]."""
    return CollectionSpec(2_000_000, 300_000, 1.1, ("lognormal", 2.3, 0.6, 1, 500),
                          seed=seed)


# ----------------------------------------------------------------------------
# Samplers
# ----------------------------------------------------------------------------
def _zipf_cdf(universe: int, s: float) -> np.ndarray:
    k = np.arange(1, universe + 1, dtype=np.float64)
    w = k ** (-float(s))
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


_GUIDE_CACHE: dict = {}


def _guide(cdf: np.ndarray) -> np.ndarray:
    """Guide table: g[k] = first index with cdf > k/M (Chen & Asau)."""
    key = (id(cdf), len(cdf))
    g = _GUIDE_CACHE.get(key)
    if g is None or g[0] is not cdf:
        M = 4 * len(cdf)
        table = np.searchsorted(cdf, np.arange(M, dtype=np.float64) / M, side="right")
        g = (cdf, table)
        _GUIDE_CACHE.clear()
        _GUIDE_CACHE[key] = g
    return g[1]


def _draw_tokens(rng: np.random.Generator, cdf: np.ndarray, n: int) -> np.ndarray:
    """Inverse-CDF draws: the first index with cdf > u, u ~ U[0,1)."""
    u = rng.random(n)
    table = _guide(cdf)
    M = len(table)
    t = table[np.minimum((u * M).astype(np.int64), M - 1)]
    np.minimum(t, len(cdf) - 1, out=t)
    idx = np.nonzero(cdf[t] <= u)[0]
    while len(idx):
        t[idx] += 1
        np.minimum(t, len(cdf) - 1, out=t)
        sub = cdf[t[idx]] <= u[idx]
        sub &= t[idx] < len(cdf) - 1
        idx = idx[sub]
    return t.astype(np.int64)


def _draw_sizes(rng: np.random.Generator, spec: CollectionSpec) -> np.ndarray:
    d = spec.size_dist
    n = spec.n_sets
    if d[0] == "uniform":
        sizes = rng.integers(d[1], d[2] + 1, size=n, dtype=np.int64)
    elif d[0] == "lognormal":
        x = np.rint(np.exp(rng.normal(d[1], d[2], size=n)))
        sizes = np.clip(x, d[3], d[4]).astype(np.int64)
    else:
        raise ValueError(f"unknown size distribution {d[0]!r}")
    return np.minimum(sizes, spec.universe)


def _rank_in_run(s: np.ndarray) -> np.ndarray:
    """For a sorted array, each element's index within its run of equal values."""
    if len(s) == 0:
        return np.zeros(0, np.int64)
    change = np.ones(len(s), bool)
    change[1:] = s[1:] != s[:-1]
    heads = np.flatnonzero(change)
    lens = np.diff(np.append(heads, len(s)))
    return np.arange(len(s), dtype=np.int64) - np.repeat(heads, lens)


def _distinct_sets(rng, sizes: np.ndarray, cdf: np.ndarray):
    """Per set, the first ``sizes[i]`` distinct tokens of an i.i.d. Zipf stream.

    Returns CSR (offsets, tokens) with each set sorted ascending.
    """
    n = len(sizes)
    U = len(cdf)
    tbits = max(1, int(U - 1).bit_length())
    sbits = max(1, int(n).bit_length())
    # Entries of sets still short of their size: (set id, per-set draw index,
    # token).  Completed sets move to ``done`` as packed (set, token) keys.
    acc_set = np.zeros(0, np.int64)
    acc_seq = np.zeros(0, np.int64)
    acc_tok = np.zeros(0, np.int64)
    done = []
    have = np.zeros(n, np.int64)
    drawn = np.zeros(n, np.int64)
    todo = np.nonzero(sizes > 0)[0]
    rounds = 0
    while len(todo):
        rounds += 1
        if rounds > 200:
            raise RuntimeError("token sampling did not converge")
        want = sizes[todo] - have[todo]
        if rounds > 1:
            want = want + (want + 3) // 4
        new_set = np.repeat(todo, want)
        starts = np.repeat(np.cumsum(want) - want, want)
        new_seq = drawn[new_set] + (np.arange(len(new_set), dtype=np.int64) - starts)
        drawn[todo] += want
        new_tok = _draw_tokens(rng, cdf, len(new_set))
        s_ = np.concatenate([acc_set, new_set])
        q_ = np.concatenate([acc_seq, new_seq])
        t_ = np.concatenate([acc_tok, new_tok])
        qbits = max(1, int(drawn.max()).bit_length())
        if sbits + tbits + qbits > 63:
            raise ValueError("collection too large for 64-bit sampling keys")
        # Sort by (set, token, draw index): the earliest draw of each
        # duplicated token comes first.
        key = (((s_ << tbits) | t_) << qbits) | q_
        key.sort()
        st = key >> qbits
        first = np.ones(len(key), bool)
        first[1:] = st[1:] != st[:-1]
        key = key[first]
        s_ = key >> (qbits + tbits)
        t_ = (key >> qbits) & ((1 << tbits) - 1)
        q_ = key & ((1 << qbits) - 1)
        # Sort by (set, draw index) and keep the earliest ``sizes`` per set.
        key = (((s_ << qbits) | q_) << tbits) | t_
        key.sort()
        s_ = key >> (qbits + tbits)
        q_ = (key >> tbits) & ((1 << qbits) - 1)
        t_ = key & ((1 << tbits) - 1)
        ok = _rank_in_run(s_) < sizes[s_]
        s_, q_, t_ = s_[ok], q_[ok], t_[ok]
        have[todo] = 0
        cnt_sets, cnt = np.unique(s_, return_counts=True)
        have[cnt_sets] = cnt
        complete = have[s_] == sizes[s_]
        done.append((s_[complete] << tbits) | t_[complete])
        acc_set, acc_seq, acc_tok = s_[~complete], q_[~complete], t_[~complete]
        todo = np.unique(acc_set)
        # Sets whose every draw so far was a duplicate have no entry left.
        short = np.nonzero(have < sizes)[0]
        if len(short) != len(todo):
            todo = short
    key = np.concatenate(done) if done else np.zeros(0, np.int64)
    key.sort()
    tokens = (key & ((1 << tbits) - 1)).astype(np.int32)
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return offsets, tokens


def _plant(rng, spec: CollectionSpec, offsets, tokens, cdf):
    """Replace ``planted_frac`` of the sets by edited copies of earlier sets."""
    n = spec.n_sets
    n_plant = int(round(spec.planted_frac * n))
    if n_plant == 0 or n < 2:
        return offsets, tokens
    targets = np.sort(rng.choice(np.arange(1, n), size=min(n_plant, n - 1), replace=False))
    sets = [tokens[offsets[i]:offsets[i + 1]] for i in range(n)]
    for t in targets:
        src = int(rng.integers(0, t))
        cur = set(int(x) for x in sets[src])
        k = int(rng.integers(0, spec.planted_max_edits + 1))
        for _ in range(k):
            op = int(rng.integers(0, 3))
            if op == 0 and len(cur) > 1:  # delete
                victim = sorted(cur)[int(rng.integers(0, len(cur)))]
                cur.discard(victim)
            else:
                if op == 2 and len(cur) > 1:  # substitute = delete + insert
                    victim = sorted(cur)[int(rng.integers(0, len(cur)))]
                    cur.discard(victim)
                if len(cur) < spec.universe:
                    for _try in range(64):
                        tok = int(_draw_tokens(rng, cdf, 1)[0])
                        if tok not in cur:
                            cur.add(tok)
                            break
        sets[t] = np.array(sorted(cur), dtype=np.int32)
    sizes = np.array([len(s) for s in sets], np.int64)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(sizes, out=offs[1:])
    toks = np.concatenate(sets).astype(np.int32) if n else np.zeros(0, np.int32)
    return offs, toks


def gen_collection(spec: CollectionSpec):
    """Draw a CSR collection (offsets int64[N+1], tokens int32[]) for ``spec``."""
    rng = np.random.default_rng(spec.seed)
    cdf = _zipf_cdf(spec.universe, spec.zipf_s)
    sizes = _draw_sizes(rng, spec)
    offsets, tokens = _distinct_sets(rng, sizes, cdf)
    if spec.planted_frac > 0:
        offsets, tokens = _plant(rng, spec, offsets, tokens, cdf)
    return offsets, tokens


def random_collection(n_sets: int, universe: int, lo: int, hi: int, seed: int,
                      zipf_s: float = 1.0, planted_frac: float = 0.0):
    """Small helper for tests: uniform sizes in [lo, hi]."""
    spec = CollectionSpec(n_sets, universe, zipf_s, ("uniform", lo, hi), seed=seed,
                          planted_frac=planted_frac)
    return gen_collection(spec)


# ----------------------------------------------------------------------------
# Batched joins and served queries
# ----------------------------------------------------------------------------
THRESHOLDS_BATCH = ((1, 2), (7, 10), (4, 5), (9, 10))
THRESHOLDS_SERVE = ((1, 2), (3, 4), (9, 10))


@dataclass
class BatchSpec:
    n_jobs: int = 512
    min_sets: int = 1_000
    max_sets: int = 200_000
    universe: int = 50_000
    zipf_s: float = 1.0
    size_lo: int = 3
    size_hi: int = 100
    seed: int = 0


def gen_batch(spec: BatchSpec):
    """Independent collections with log-uniform set counts and per-job thresholds.

    Returns a list of (offsets, tokens, p, q).
    """
    rng = np.random.default_rng(spec.seed)
    logn = rng.uniform(np.log(spec.min_sets), np.log(spec.max_sets), size=spec.n_jobs)
    ns = np.rint(np.exp(logn)).astype(np.int64)
    th = rng.integers(0, len(THRESHOLDS_BATCH), size=spec.n_jobs)
    seeds = rng.integers(0, 2**31 - 1, size=spec.n_jobs)
    jobs = []
    for k in range(spec.n_jobs):
        cs = CollectionSpec(int(ns[k]), spec.universe, spec.zipf_s,
                            ("uniform", spec.size_lo, spec.size_hi), seed=int(seeds[k]))
        off, tok = gen_collection(cs)
        p, q = THRESHOLDS_BATCH[int(th[k])]
        jobs.append((off, tok, p, q))
    return jobs


@dataclass
class QuerySpec:
    n_queries: int = 20_000
    rate_qps: float = 20_000.0
    size_lo: int = 2
    size_hi: int = 300
    perturbed_frac: float = 0.5
    max_edits: int = 3
    seed: int = 1


def gen_queries(spec: QuerySpec, coll_spec: CollectionSpec, offsets, tokens):
    """Probe sets with Poisson arrival times.

    Half of the probes (``perturbed_frac``) are copies of random resident sets
    with up to ``max_edits`` token edits, so results are non-empty; the rest
    draw a uniform size in [size_lo, size_hi] and Zipf tokens like the
    collection.  Returns (arrival_s float64[Q], offsets int64[Q+1],
    tokens int32[], p uint32[Q], q uint32[Q]).
    """
    rng = np.random.default_rng(spec.seed)
    cdf = _zipf_cdf(coll_spec.universe, coll_spec.zipf_s)
    Q = spec.n_queries
    gaps = rng.exponential(1.0 / spec.rate_qps, size=Q)
    arrival = np.cumsum(gaps) - gaps[0]
    th = rng.integers(0, len(THRESHOLDS_SERVE), size=Q)
    p = np.array([THRESHOLDS_SERVE[t][0] for t in th], np.uint32)
    q = np.array([THRESHOLDS_SERVE[t][1] for t in th], np.uint32)
    n_res = len(offsets) - 1
    probes = []
    for k in range(Q):
        if rng.random() < spec.perturbed_frac and n_res > 0:
            src = int(rng.integers(0, n_res))
            cur = set(int(x) for x in tokens[offsets[src]:offsets[src + 1]])
            for _ in range(int(rng.integers(0, spec.max_edits + 1))):
                if rng.random() < 0.5 and len(cur) > 1:
                    cur.discard(sorted(cur)[int(rng.integers(0, len(cur)))])
                else:
                    for _try in range(64):
                        tok = int(_draw_tokens(rng, cdf, 1)[0])
                        if tok not in cur:
                            cur.add(tok)
                            break
            probes.append(np.array(sorted(cur), np.int32))
        else:
            size = int(min(rng.integers(spec.size_lo, spec.size_hi + 1), coll_spec.universe))
            seen: set = set()
            while len(seen) < size:
                for x in _draw_tokens(rng, cdf, size - len(seen) + 4):
                    seen.add(int(x))
                    if len(seen) == size:
                        break
            probes.append(np.array(sorted(seen), np.int32))
    sizes = np.array([len(x) for x in probes], np.int64)
    poff = np.zeros(Q + 1, np.int64)
    np.cumsum(sizes, out=poff[1:])
    ptok = np.concatenate(probes).astype(np.int32) if Q else np.zeros(0, np.int32)
    return arrival, poff, ptok, p, q


# ----------------------------------------------------------------------------
# Device-side sampler for large workloads
# ----------------------------------------------------------------------------
def _rank_in_run_t(torch, s):
    if s.numel() == 0:
        return torch.zeros(0, dtype=torch.int64, device=s.device)
    change = torch.ones(s.numel(), dtype=torch.bool, device=s.device)
    change[1:] = s[1:] != s[:-1]
    heads = torch.nonzero(change).flatten()
    lens = torch.diff(torch.cat([heads, torch.tensor([s.numel()], device=s.device)]))
    return torch.arange(s.numel(), device=s.device) - torch.repeat_interleave(heads, lens)


def gen_collection_device(spec: CollectionSpec, device="cuda"):
    """The recipe of gen_collection drawn with torch's generator on a CUDA device.

    Same size law, Zipf law and first-distinct-draws rule as the host
    sampler, for workloads whose 1e8-1e9 tokens make the host sampler slow;
    the random stream differs, so the sets differ from gen_collection's.
    Planted near-duplicates are not supported here.  Returns device tensors
    (offsets int64[N+1], tokens int32[]).
    """
    import torch
    if spec.planted_frac:
        raise ValueError("planted near-duplicates are host-sampler only")
    g = torch.Generator(device=device)
    g.manual_seed(int(spec.seed))
    n, U = spec.n_sets, spec.universe
    d = spec.size_dist
    if d[0] == "uniform":
        sizes = torch.randint(d[1], d[2] + 1, (n,), generator=g, device=device, dtype=torch.int64)
    else:
        x = torch.normal(float(d[1]), float(d[2]), (n,), generator=g, device=device,
                         dtype=torch.float64)
        sizes = torch.clamp(torch.round(torch.exp(x)), d[3], d[4]).to(torch.int64)
    sizes = torch.clamp(sizes, max=U)
    cdf = torch.from_numpy(_zipf_cdf(U, spec.zipf_s)).to(device)
    tbits = max(1, int(U - 1).bit_length())
    sbits = max(1, int(n).bit_length())
    tmask = (1 << tbits) - 1
    acc_s = torch.zeros(0, dtype=torch.int64, device=device)
    acc_q = torch.zeros(0, dtype=torch.int64, device=device)
    acc_t = torch.zeros(0, dtype=torch.int64, device=device)
    have = torch.zeros(n, dtype=torch.int64, device=device)
    drawn = torch.zeros(n, dtype=torch.int64, device=device)
    done = []
    todo = torch.nonzero(sizes > 0).flatten()
    rounds = 0
    while todo.numel():
        rounds += 1
        if rounds > 200:
            raise RuntimeError("token sampling did not converge")
        want = sizes[todo] - have[todo]
        if rounds > 1:
            want = want + (want + 3) // 4
        new_s = torch.repeat_interleave(todo, want)
        starts = torch.repeat_interleave(torch.cumsum(want, 0) - want, want)
        new_q = drawn[new_s] + (torch.arange(new_s.numel(), device=device) - starts)
        drawn[todo] += want
        u = torch.rand(new_s.numel(), generator=g, device=device, dtype=torch.float64)
        new_t = torch.clamp(torch.searchsorted(cdf, u, right=True), max=U - 1)
        s_ = torch.cat([acc_s, new_s])
        q_ = torch.cat([acc_q, new_q])
        t_ = torch.cat([acc_t, new_t])
        del new_s, new_q, new_t, starts, u
        qbits = max(1, int(drawn.max().item()).bit_length())
        if sbits + tbits + qbits > 63:
            raise ValueError("collection too large for 64-bit sampling keys")
        key, _ = torch.sort((((s_ << tbits) | t_) << qbits) | q_)
        st = key >> qbits
        first = torch.ones(key.numel(), dtype=torch.bool, device=device)
        first[1:] = st[1:] != st[:-1]
        key = key[first]
        del st, first
        s_ = key >> (qbits + tbits)
        t_ = (key >> qbits) & tmask
        q_ = key & ((1 << qbits) - 1)
        key, _ = torch.sort((((s_ << qbits) | q_) << tbits) | t_)
        s_ = key >> (qbits + tbits)
        q_ = (key >> tbits) & ((1 << qbits) - 1)
        t_ = key & tmask
        del key
        ok = _rank_in_run_t(torch, s_) < sizes[s_]
        s_, q_, t_ = s_[ok], q_[ok], t_[ok]
        have[todo] = 0
        have.index_add_(0, s_, torch.ones_like(s_))
        complete = have[s_] == sizes[s_]
        done.append((s_[complete] << tbits) | t_[complete])
        keep = ~complete
        acc_s, acc_q, acc_t = s_[keep], q_[keep], t_[keep]
        todo = torch.nonzero(have < sizes).flatten()
    key = torch.cat(done) if done else torch.zeros(0, dtype=torch.int64, device=device)
    key, _ = torch.sort(key)
    tokens = (key & tmask).to(torch.int32)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    offsets[1:] = torch.cumsum(sizes, 0)
    return offsets, tokens


def gen_batch_device(spec: BatchSpec, device="cuda"):
    """The batched workload drawn on the device: job sizes log-uniform in
    [min_sets, max_sets], thresholds uniform over THRESHOLDS_BATCH; all jobs'
    sets come from one collection (sizes U[size_lo, size_hi], Zipf tokens) cut
    into consecutive jobs.  Returns (offsets, tokens) device tensors and
    numpy job_sets int64[n_jobs+1], p, q uint32[n_jobs]."""
    rng = np.random.default_rng(spec.seed)
    logn = rng.uniform(np.log(spec.min_sets), np.log(spec.max_sets), size=spec.n_jobs)
    ns = np.rint(np.exp(logn)).astype(np.int64)
    th = rng.integers(0, len(THRESHOLDS_BATCH), size=spec.n_jobs)
    job_sets = np.zeros(spec.n_jobs + 1, np.int64)
    np.cumsum(ns, out=job_sets[1:])
    cs = CollectionSpec(int(job_sets[-1]), spec.universe, spec.zipf_s,
                        ("uniform", spec.size_lo, spec.size_hi), seed=spec.seed)
    off, tok = gen_collection_device(cs, device)
    p = np.array([THRESHOLDS_BATCH[t][0] for t in th], np.uint32)
    q = np.array([THRESHOLDS_BATCH[t][1] for t in th], np.uint32)
    return off, tok, job_sets, p, q
