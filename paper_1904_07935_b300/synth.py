"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module only *makes inputs*: matrices with the shapes and value
distributions of the paper's workloads (sparse term-document matrices shaped
like its text datasets, dense non-negative matrices shaped like its image
datasets, Table 4) and the random non-negative initial factors of Alg. 1
(first step).  It performs none of the factorisation arithmetic.

Two kinds of randomness:

* Workload matrices come from ``numpy.random.Generator(Philox(seed))``; the
  GPU path never regenerates them, it receives the arrays.
* Initial factors use a counter-based SplitMix64 stream (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014): output i of
  a generator seeded with ``s`` is ``mix64(s + (i + 1) * 0x9E3779B97F4A7C15)``.
  The CUDA library implements the same published definition independently so
  that ``nmf_init`` with no explicit initial factors draws the same values.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags for the two initial factors (xor-ed into the user seed).
TAG_W = np.uint64(0x5757575757575757)
TAG_H = np.uint64(0x4848484848484848)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix_uniform(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64(seed) as float32 in [0, 1).

    Each output keeps its top 24 bits: u = (x >> 40) * 2**-24, which is exact
    in float32.
    """
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + i * GOLDEN_GAMMA
    x = mix64(state)
    return ((x >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)).astype(np.float32)


def init_factors(seed: int, V: int, D: int, K: int) -> tuple[np.ndarray, np.ndarray]:
    """Random non-negative W (V x K) and H (K x D), U[0,1), float32, row-major.

    Alg. 1, first step: "Initialize W and H with random non-negative numbers".
    W is drawn from stream ``seed ^ TAG_W`` and H from ``seed ^ TAG_H``; entry
    (r, c) is output number r * cols + c of its stream.  The column
    normalisation of W that both sides apply afterwards is part of the method
    and is not done here.
    """
    sw = int(np.uint64(seed) ^ TAG_W)
    sh = int(np.uint64(seed) ^ TAG_H)
    W = splitmix_uniform(sw, V * K).reshape(V, K)
    H = splitmix_uniform(sh, K * D).reshape(K, D)
    return W, H


# ---------------------------------------------------------------------------
# Dense planted workloads (image-like, dense A)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class DenseProblem:
    A: np.ndarray          # V x D float32, row-major
    W0: np.ndarray         # planted V x K0 (float64)
    H0: np.ndarray         # planted K0 x D (float64)

    @property
    def shape(self):
        return self.A.shape


def planted_dense(V: int, D: int, K0: int, seed: int, noise: float = 0.01) -> DenseProblem:
    """A = W0 H0 + |N(0, noise^2)| with W0, H0 i.i.d. U[0,1).

    Stored as float32.  The planted product is formed in float64 and rounded
    once.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    W0 = rng.random((V, K0))
    H0 = rng.random((K0, D))
    A = W0 @ H0
    A += np.abs(rng.normal(0.0, noise, size=(V, D)))
    return DenseProblem(A=A.astype(np.float32), W0=W0, H0=H0)


# ---------------------------------------------------------------------------
# Sparse term-document workloads (text-like)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CsrMatrix:
    """Compressed sparse rows: int32 indices, float32 values, sorted columns."""

    n_rows: int
    n_cols: int
    row_ptr: np.ndarray    # int32, n_rows + 1
    col_idx: np.ndarray    # int32, nnz
    val: np.ndarray        # float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n_rows, self.n_cols), dtype=np.float32)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        out[rows, self.col_idx] = self.val
        return out

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr),
                             shape=(self.n_rows, self.n_cols))


def _coo_to_csr(rows, cols, vals, n_rows, n_cols) -> CsrMatrix:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n_rows)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 indexing")
    return CsrMatrix(n_rows, n_cols, row_ptr.astype(np.int32),
                     cols.astype(np.int32), vals.astype(np.float32))


@dataclasses.dataclass
class SparseProblem:
    A: CsrMatrix           # V x D (rows = words, columns = documents)
    At: CsrMatrix          # D x V (rows = documents)
    doc_terms: np.ndarray  # distinct terms per document (int64, D)

    @property
    def shape(self):
        return (self.A.n_rows, self.A.n_cols)


def zipf_cdf(V: int, s: float) -> np.ndarray:
    p = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(p)
    return c / c[-1]


def _draw_document(rng, cdf: np.ndarray, L: int):
    """Tokens i.i.d. Zipf until L distinct terms are seen; returns (ids, counts)."""
    V = cdf.shape[0]
    chunk = max(64, 3 * L)
    toks = np.empty(0, dtype=np.int64)
    while True:
        new = np.searchsorted(cdf, rng.random(chunk), side="right")
        np.minimum(new, V - 1, out=new)
        toks = np.concatenate([toks, new])
        uniq, first = np.unique(toks, return_index=True)
        if uniq.shape[0] >= L:
            cut = np.sort(first)[L - 1] + 1      # prefix that contains exactly L distinct
            ids, counts = np.unique(toks[:cut], return_counts=True)
            return ids, counts
        chunk *= 2


def sparse_termdoc(V: int, D: int, seed: int, mean_terms: float = 100.0,
                   sigma: float = 1.0, zipf_s: float = 1.1,
                   max_terms: int | None = None) -> SparseProblem:
    """Synthetic tf-idf term-document matrix shaped like the paper's text data.

    * distinct terms per document L_d ~ LogNormal(ln(mean) - sigma^2/2, sigma),
      rounded, clipped to [1, min(V, max_terms)];
    * tokens i.i.d. Zipf(s) over word ranks 1..V (rank r -> word id r-1) until
      L_d distinct words are seen; the term count is the multiplicity;
    * weight = count * (ln(D / df) + 1), then every document column is scaled
      to unit L2 norm (so ||A||_F^2 = D).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    cdf = zipf_cdf(V, zipf_s)
    mu = math.log(mean_terms) - 0.5 * sigma * sigma
    L = np.rint(rng.lognormal(mu, sigma, size=D)).astype(np.int64)
    cap = V if max_terms is None else min(V, max_terms)
    np.clip(L, 1, cap, out=L)
    rows, cols, cnts = [], [], []
    for d in range(D):
        ids, counts = _draw_document(rng, cdf, int(L[d]))
        rows.append(ids)
        cols.append(np.full(ids.shape[0], d, dtype=np.int64))
        cnts.append(counts)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    cnts = np.concatenate(cnts).astype(np.float64)
    df = np.bincount(rows, minlength=V).astype(np.float64)
    idf = np.log(D / np.maximum(df, 1.0)) + 1.0
    w = cnts * idf[rows]
    colnorm = np.sqrt(np.bincount(cols, weights=w * w, minlength=D))
    w = w / colnorm[cols]
    A = _coo_to_csr(rows, cols, w, V, D)
    At = _coo_to_csr(cols, rows, w, D, V)
    return SparseProblem(A=A, At=At, doc_terms=L)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

SEED_DENSE_SMALL = 0xC1
SEED_TEXT = 0xC2
SEED_DENSE_LARGE = 0xC3
SEED_BATCH = 0xC4
SEED_WARM_TRAIN = 0xC5
SEED_WARM_EVAL = 0xC5E


def dense_small() -> DenseProblem:
    """512 x 384 planted rank-16 dense matrix (factorised at K=16)."""
    return planted_dense(512, 384, 16, SEED_DENSE_SMALL)


def dense_large() -> DenseProblem:
    """8192 x 8192 planted rank-256 dense matrix (factorised at K=256)."""
    return planted_dense(8192, 8192, 256, SEED_DENSE_LARGE)


SEED_FACES = 0xF4


def faces_like(kind: str, seed: int = SEED_FACES) -> DenseProblem:
    """Face-image-shaped dense matrices with the shapes of the paper's AT&T
    (400 x 10,304: 400 images of 112 x 92 pixels) and PIE (11,554 x 4,096:
    64 x 64 pixels) datasets; synthetic contents only.  Each of r basis
    images (200 / 256: poses, lighting and expressions as well as subjects)
    is non-negative and smooth (three Gaussian blobs of
    random position and width over a gentle gradient); a row of A mixes the r
    bases with U[0,1) weights; |N(0, 0.01^2)| noise; A scaled to max 1 like
    pixel intensities.  W0 (images x r) and H0 (r x pixels) are the planted
    factors (scaled with A)."""
    if kind == "att":
        n_img, h, w, r = 400, 112, 92, 200
    elif kind == "pie":
        n_img, h, w, r = 11554, 64, 64, 256
    else:
        raise ValueError(kind)
    rng = np.random.Generator(np.random.Philox(seed + (0 if kind == "att" else 1)))
    yy, xx = np.meshgrid(np.arange(h) / h, np.arange(w) / w, indexing="ij")
    H0 = np.empty((r, h * w))
    for k in range(r):
        img = 0.2 * (1.0 + rng.uniform(-1, 1) * (yy - 0.5) + rng.uniform(-1, 1) * (xx - 0.5))
        for _ in range(3):
            cy, cx = rng.uniform(0.15, 0.85, size=2)
            sy, sx = rng.uniform(0.05, 0.25, size=2)
            img += rng.uniform(0.5, 1.0) * np.exp(-0.5 * (((yy - cy) / sy) ** 2 + ((xx - cx) / sx) ** 2))
        H0[k] = img.ravel()
    W0 = rng.random((n_img, r))
    A = W0 @ H0
    A += np.abs(rng.normal(0.0, 0.01, size=A.shape))
    scale = 1.0 / A.max()
    return DenseProblem(A=(A * scale).astype(np.float32), W0=W0 * scale, H0=H0)


def text_20ng_like(seed: int = SEED_TEXT) -> SparseProblem:
    """26,214 words x 11,314 documents, about 1.1M non-zeros (20NG-shaped)."""
    return sparse_termdoc(26214, 11314, seed)


def batch_instances(n: int = 64, seed: int = SEED_BATCH):
    """Uneven sparse instances: V~U{1000..20000}, D~U{500..8000},
    density~U[0.1%, 1%], K from {16, 32, 64, 128}."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(n):
        V = int(rng.integers(1000, 20001))
        D = int(rng.integers(500, 8001))
        dens = float(rng.uniform(0.001, 0.01))
        K = int(rng.choice([16, 32, 64, 128]))
        prob = sparse_termdoc(V, D, seed + 1000 + i, mean_terms=max(2.0, dens * V))
        out.append((prob, K))
    return out
