"""Seeded synthetic workloads for guided (banded, Z-drop) extension alignment.

This module only draws random inputs: reads, their mutated reference
counterparts and the scoring parameters of each workload.  It holds none of
the alignment arithmetic, so both the CUDA path and the CPU oracle can be fed
from it without sharing any of the method's code.

The paper evaluates on GIAB HiFi / CLR / ONT reads after minimap2's chaining
step (Section 5.1).  Those datasets are not available here, so each workload
below is a seeded stand-in with the length distribution and error profile of
one read technology:

* ``small``   - 256 pairs of 1,000 bp, 5% sub / 2.5% ins / 2.5% del.
* ``ont``     - 20,000 pairs, log-normal length (median 5 kbp, sigma 0.8,
  clipped to [500, 50k]), 12% errors (5% sub / 4% del / 3% ins), 10% of the
  pairs continue into unrelated sequence from a uniform position.
* ``hifi``    - 20,000 pairs, Normal(15 kbp, 3 kbp) length (min 2 kbp), 1%
  errors, 2% divergent tails, HiFi scoring.
* ``skewed``  - 100,000 pairs, Pareto(alpha=1.5, min 500 bp, cap 100 kbp)
  length, 8% errors (4% sub / 2% ins / 2% del), 20% divergent tails.

Bases are integer codes A=0, C=1, G=2, T=3.  The query is uniform random; the
target (reference) is the query after substitutions, insertions and deletions
(indel length geometric with mean 2; an indel event starts at a base with
probability rate / mean length), optionally followed by a divergent tail.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional

import numpy as np

SEED_BASE = 2403_06478

ALPHABET = "ACGT"


@dataclass(frozen=True)
class Scoring:
    """Scoring and guiding parameters (minimap2 naming).

    A gap of length l costs min(q + l*e, q2 + l*e2).  ``w`` is the band
    half-width (|t - q| <= w), ``zdrop`` the Z-drop threshold (negative: off).
    """
    a: int = 2
    b: int = 4
    q: int = 4
    e: int = 2
    q2: int = 24
    e2: int = 1
    w: int = 100
    zdrop: int = 400
    end_bonus: int = 0

    def as_tuple(self):
        return (self.a, self.b, self.q, self.e, self.q2, self.e2, self.w,
                self.zdrop, self.end_bonus)


@dataclass
class Batch:
    """A batch of read/reference pairs stored as concatenated code arrays."""
    name: str
    q_codes: np.ndarray          # uint8, all queries back to back
    t_codes: np.ndarray          # uint8, all targets back to back
    q_off: np.ndarray            # int64, start of pair i in q_codes
    t_off: np.ndarray            # int64
    q_len: np.ndarray            # int32
    t_len: np.ndarray            # int32
    scoring: Scoring
    meta: Dict = field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return int(self.q_len.shape[0])

    def query(self, i: int) -> np.ndarray:
        o = int(self.q_off[i])
        return self.q_codes[o:o + int(self.q_len[i])]

    def target(self, i: int) -> np.ndarray:
        o = int(self.t_off[i])
        return self.t_codes[o:o + int(self.t_len[i])]

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        qs = [self.query(int(i)) for i in idx]
        ts = [self.target(int(i)) for i in idx]
        return from_pairs(qs, ts, self.scoring, name=f"{self.name}[subset]")

    def with_scoring(self, **kw) -> "Batch":
        return replace(self, scoring=replace(self.scoring, **kw))

    def total_bases(self) -> int:
        return int(self.q_len.sum()) + int(self.t_len.sum())


def from_pairs(queries: List[np.ndarray], targets: List[np.ndarray],
               scoring: Scoring, name: str = "pairs") -> Batch:
    """Build a batch from per-pair code arrays (or ACGT strings)."""
    qs = [_as_codes(x) for x in queries]
    ts = [_as_codes(x) for x in targets]
    q_len = np.array([len(x) for x in qs], dtype=np.int32)
    t_len = np.array([len(x) for x in ts], dtype=np.int32)
    q_off = np.zeros(len(qs), dtype=np.int64)
    t_off = np.zeros(len(ts), dtype=np.int64)
    if len(qs):
        q_off[1:] = np.cumsum(q_len[:-1], dtype=np.int64)
        t_off[1:] = np.cumsum(t_len[:-1], dtype=np.int64)
    q_codes = np.concatenate(qs).astype(np.uint8) if qs else np.zeros(0, np.uint8)
    t_codes = np.concatenate(ts).astype(np.uint8) if ts else np.zeros(0, np.uint8)
    return Batch(name, q_codes, t_codes, q_off, t_off, q_len, t_len, scoring)


def _as_codes(x) -> np.ndarray:
    if isinstance(x, str):
        lut = np.full(256, 255, dtype=np.uint8)
        for i, ch in enumerate(ALPHABET):
            lut[ord(ch)] = i
            lut[ord(ch.lower())] = i
        arr = lut[np.frombuffer(x.encode("ascii"), dtype=np.uint8)]
        if (arr == 255).any():
            raise ValueError("only A, C, G, T are supported")
        return arr
    return np.asarray(x, dtype=np.uint8)


def codes_to_str(codes: np.ndarray) -> str:
    return "".join(ALPHABET[int(c)] for c in codes)


# --------------------------------------------------------------------------
# Mutation model
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class ErrorModel:
    sub: float
    ins: float
    dele: float
    tail_frac: float = 0.0       # fraction of pairs with a divergent tail
    indel_mean: float = 2.0


def _mutate_chunk(rng: np.random.Generator, q: np.ndarray, q_len: np.ndarray,
                  em: ErrorModel):
    """Mutate a chunk of concatenated queries; returns (targets, t_len)."""
    n = q.shape[0]
    n_pairs = q_len.shape[0]
    pair_end = np.repeat(np.cumsum(q_len, dtype=np.int64), q_len)
    pos = np.arange(n, dtype=np.int64)
    u = rng.random(n)
    p_del = em.dele / em.indel_mean
    p_ins = em.ins / em.indel_mean
    is_sub = u < em.sub
    is_del = (u >= em.sub) & (u < em.sub + p_del)
    is_ins = (u >= em.sub + p_del) & (u < em.sub + p_del + p_ins)
    p_geo = 1.0 / em.indel_mean
    # deletions: base i starts a run of L deleted query bases (clipped to the pair)
    del_at = np.flatnonzero(is_del)
    del_end = np.zeros(n, dtype=np.int64)
    del_end[del_at] = np.minimum(del_at + rng.geometric(p_geo, del_at.size),
                                 pair_end[del_at])
    run_end = np.maximum.accumulate(del_end)
    deleted = run_end > pos
    # insertions: L random bases are emitted before base i
    ins_at = np.flatnonzero(is_ins)
    ins_len = np.zeros(n, dtype=np.int64)
    ins_len[ins_at] = rng.geometric(p_geo, ins_at.size)
    # substitutions: a different base, uniformly among the other three
    base = q.copy()
    sub_at = np.flatnonzero(is_sub)
    base[sub_at] = (q[sub_at] + rng.integers(1, 4, sub_at.size, dtype=np.uint8)) & 3
    keep = (~deleted).astype(np.int64)
    counts = ins_len + keep
    total = int(counts.sum())
    src = np.repeat(pos, counts)
    out = base[src]
    # the inserted bases are the first ins_len[i] slots of each group
    first = np.cumsum(counts) - counts
    ins_groups = np.flatnonzero(ins_len)
    if ins_groups.size:
        lens = ins_len[ins_groups]
        starts = np.repeat(first[ins_groups], lens)
        within = np.arange(int(lens.sum()), dtype=np.int64) - np.repeat(np.cumsum(lens) - lens, lens)
        out[starts + within] = rng.integers(0, 4, starts.size, dtype=np.uint8)
    pair_id = np.repeat(np.arange(n_pairs, dtype=np.int64), q_len)
    t_len = np.bincount(pair_id, weights=counts, minlength=n_pairs).astype(np.int64)
    # divergent tails: from a uniform position on, the target is fresh sequence
    if em.tail_frac > 0 and n_pairs:
        has_tail = rng.random(n_pairs) < em.tail_frac
        cut = np.floor(rng.random(n_pairs) * t_len).astype(np.int64)
        t_start = np.cumsum(t_len) - t_len
        pid_out = np.repeat(np.arange(n_pairs, dtype=np.int64), t_len)
        within = np.arange(total, dtype=np.int64) - t_start[pid_out]
        replace_mask = has_tail[pid_out] & (within >= cut[pid_out])
        rep = np.flatnonzero(replace_mask)
        out[rep] = rng.integers(0, 4, rep.size, dtype=np.uint8)
    return out, t_len.astype(np.int32)


def _build(name: str, rng: np.random.Generator, q_len: np.ndarray,
           em: ErrorModel, scoring: Scoring, chunk_bases: int = 1 << 24) -> Batch:
    q_len = q_len.astype(np.int32)
    n_pairs = q_len.shape[0]
    q_parts, t_parts, t_lens = [], [], []
    i = 0
    while i < n_pairs:
        j = i
        acc = 0
        while j < n_pairs and (acc == 0 or acc + int(q_len[j]) <= chunk_bases):
            acc += int(q_len[j])
            j += 1
        ql = q_len[i:j]
        q = rng.integers(0, 4, int(ql.sum()), dtype=np.uint8)
        t, tl = _mutate_chunk(rng, q, ql, em)
        q_parts.append(q)
        t_parts.append(t)
        t_lens.append(tl)
        i = j
    q_codes = np.concatenate(q_parts) if q_parts else np.zeros(0, np.uint8)
    t_codes = np.concatenate(t_parts) if t_parts else np.zeros(0, np.uint8)
    t_len = np.concatenate(t_lens) if t_lens else np.zeros(0, np.int32)
    q_off = np.zeros(n_pairs, np.int64)
    t_off = np.zeros(n_pairs, np.int64)
    if n_pairs:
        q_off[1:] = np.cumsum(q_len[:-1], dtype=np.int64)
        t_off[1:] = np.cumsum(t_len[:-1], dtype=np.int64)
    return Batch(name, q_codes, t_codes, q_off, t_off, q_len, t_len.astype(np.int32),
                 scoring)


ONT_SCORING = Scoring(a=2, b=4, q=4, e=2, q2=24, e2=1, w=500, zdrop=400, end_bonus=0)
HIFI_SCORING = Scoring(a=1, b=4, q=6, e=2, q2=26, e2=1, w=500, zdrop=200, end_bonus=0)
SMALL_SCORING = Scoring(a=2, b=4, q=4, e=2, q2=24, e2=1, w=100, zdrop=400, end_bonus=0)
SKEWED_SCORING = Scoring(a=2, b=4, q=4, e=2, q2=24, e2=1, w=750, zdrop=400, end_bonus=0)

CONFIG_NAMES = ("small", "ont", "hifi", "skewed")

# BWA-MEM's default extension parameters (match 1, mismatch 4, gap open 6,
# extend 1, band 100, Z-drop 100, end bonus 5): single-piece gaps, so the
# second piece repeats the first and collapses.  Used with this method's own
# extension rules (the paper applies its kernel to BWA-MEM, Section 5.9, but
# states no other rule of BWA's).
BWA_SCORING = Scoring(a=1, b=4, q=6, e=1, q2=6, e2=1, w=100, zdrop=100, end_bonus=5)


def ont_lengths(rng: np.random.Generator, n: int) -> np.ndarray:
    x = rng.lognormal(mean=np.log(5000.0), sigma=0.8, size=n)
    return np.clip(np.rint(x), 500, 50_000).astype(np.int32)


def make_small(n_pairs: int = 256, seed: Optional[int] = None) -> Batch:
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    ql = np.full(n_pairs, 1000, dtype=np.int32)
    em = ErrorModel(sub=0.05, ins=0.025, dele=0.025)
    return _build("small", rng, ql, em, SMALL_SCORING)


def make_ont(n_pairs: int = 20_000, seed: Optional[int] = None) -> Batch:
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    ql = ont_lengths(rng, n_pairs)
    em = ErrorModel(sub=0.05, ins=0.03, dele=0.04, tail_frac=0.10)
    return _build("ont", rng, ql, em, ONT_SCORING)


def make_hifi(n_pairs: int = 20_000, seed: Optional[int] = None) -> Batch:
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    ql = np.maximum(np.rint(rng.normal(15_000.0, 3_000.0, n_pairs)), 2000).astype(np.int32)
    em = ErrorModel(sub=0.005, ins=0.0025, dele=0.0025, tail_frac=0.02)
    return _build("hifi", rng, ql, em, HIFI_SCORING)


def make_skewed(n_pairs: int = 100_000, seed: Optional[int] = None) -> Batch:
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    x = (rng.pareto(1.5, n_pairs) + 1.0) * 500.0
    ql = np.minimum(np.rint(x), 100_000).astype(np.int32)
    em = ErrorModel(sub=0.04, ins=0.02, dele=0.02, tail_frac=0.20)
    return _build("skewed", rng, ql, em, SKEWED_SCORING)


def make_short(n_pairs: int = 200_000, seed: Optional[int] = None) -> Batch:
    """Short-read extensions with BWA-MEM's default parameters: 150 bp
    queries, 1% errors (0.8 sub / 0.1 ins / 0.1 del), 5% divergent tails."""
    rng = np.random.default_rng(SEED_BASE + 7 if seed is None else seed)
    ql = np.full(n_pairs, 150, dtype=np.int32)
    em = ErrorModel(sub=0.008, ins=0.001, dele=0.001, tail_frac=0.05)
    return _build("short", rng, ql, em, BWA_SCORING)


def seed_scores(n_pairs: int, seed: Optional[int] = None, lo: int = 19, hi: int = 60) -> np.ndarray:
    """Initial scores for the local extension (the BWA-MEM variant): the score
    of the seed each extension continues.  BWA-MEM seeds are maximal exact
    matches of at least 19 bases scored +1 per base, so uniform in [lo, hi]."""
    rng = np.random.default_rng(SEED_BASE + 8 if seed is None else seed)
    return rng.integers(lo, hi + 1, n_pairs).astype(np.int32)


def make_long_ratio(long_frac: float, n_pairs: int = 20_000, long_len: int = 4096,
                    short_len: int = 128, seed: Optional[int] = None) -> Batch:
    """Two-length mix for the load-balancing study (the paper's synthetic
    4096 bp / 128 bp experiment, Section 5.6): a fraction `long_frac` of the
    pairs are long, shuffled among the short ones; small-config errors and
    ONT-like scoring."""
    rng = np.random.default_rng(SEED_BASE + 6 if seed is None else seed)
    n_long = int(round(long_frac * n_pairs))
    ql = np.full(n_pairs, short_len, dtype=np.int32)
    ql[:n_long] = long_len
    rng.shuffle(ql)
    em = ErrorModel(sub=0.05, ins=0.025, dele=0.025)
    return _build(f"long_ratio_{long_frac:g}", rng, ql, em, ONT_SCORING)


def make_config(name: str, n_pairs: Optional[int] = None,
                seed: Optional[int] = None) -> Batch:
    """Workload by name; ``n_pairs`` shrinks it (same distribution)."""
    makers = {"small": make_small, "ont": make_ont, "hifi": make_hifi,
              "skewed": make_skewed, "short": make_short}
    if name not in makers:
        raise KeyError(f"unknown workload {name!r}; have {sorted(makers)}")
    if n_pairs is None:
        return makers[name](seed=seed)
    return makers[name](n_pairs=n_pairs, seed=seed)


def random_pairs(rng: np.random.Generator, n: int, max_len: int,
                 scoring: Scoring, min_len: int = 0, related: float = 0.5) -> Batch:
    """Short random pairs for edge-case tests (lengths uniform in [min_len, max_len])."""
    qs, ts = [], []
    for _ in range(n):
        ql = int(rng.integers(min_len, max_len + 1))
        q = rng.integers(0, 4, ql, dtype=np.uint8)
        if rng.random() < related and ql > 0:
            t, _ = _mutate_chunk(rng, q, np.array([ql], np.int32),
                                 ErrorModel(sub=0.1, ins=0.05, dele=0.05))
            t = t[:max_len] if len(t) > max_len else t
        else:
            tl = int(rng.integers(min_len, max_len + 1))
            t = rng.integers(0, 4, tl, dtype=np.uint8)
        qs.append(q)
        ts.append(t)
    return from_pairs(qs, ts, scoring, name="random")


# --------------------------------------------------------------------------
# Serving workload: Poisson request stream drawn from the ONT-like mix
# --------------------------------------------------------------------------

@dataclass
class Request:
    arrival_s: float
    pair_idx: np.ndarray   # indices into the backing batch


def poisson_requests(rng: np.random.Generator, rate_hz: float, n_requests: int,
                     pool_pairs: int, max_pairs: int = 512) -> List[Request]:
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        k = int(rng.integers(1, max_pairs + 1))
        out.append(Request(float(t[i]), rng.integers(0, pool_pairs, k, dtype=np.int64)))
    return out
