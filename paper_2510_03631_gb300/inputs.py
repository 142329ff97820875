"""Seeded synthetic inputs for the LWE-PIR path (numpy only).

This module holds the random draws the scheme consumes and nothing of its
arithmetic: database digits, the public matrix A when it is wanted as an
explicit array, secrets s, noise e and target columns.  Both the CPU oracle
and the CUDA path are fed from here, so parity never depends on a generator
being re-implemented twice.

Workload shapes follow the spectrum-database PIR of QPADL (arxiv 2510.03631):
the paper's server answers a query vector against an r x b database matrix
(Sec. 5.2, "Parallel Chor-PIR"; Def. 1).  The paper's SQLite spectrum tables
are not available, so the digits are uniform over Z_p, which is also the
worst case for the delta compression of Sec. 5.3.

Every stream is counter based: output i of stream `tag` under `seed` is the
SplitMix64 finaliser applied to key + (i + 1) * golden_gamma, with
key = finaliser(seed ^ tag * stream_gamma).  Any slice of any stream can be
regenerated independently, which is what the sampled full-size parity tests
rely on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_STREAM_GAMMA = np.uint64(0xD1B54A32D192ED03)

# stream tags, one per kind of draw
TAG_DB = 1
TAG_A = 2
TAG_S = 3
TAG_E = 4
TAG_COL = 5
TAG_ARRIVAL = 6
TAG_MISC = 7


def _fin(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = z.astype(np.uint64, copy=True)
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the (seed, tag) stream as uint64."""
    with np.errstate(over="ignore"):
        key = _fin(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                             ^ (np.uint64(tag) * _STREAM_GAMMA)], dtype=np.uint64))[0]
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _fin(key + idx * _GOLDEN_GAMMA)


def db_digits(rows: int, cols: int, p: int = 256, seed: int = 1,
              row_start: int = 0, row_count: int | None = None) -> np.ndarray:
    """Database D in Z_p^{rows x cols}, row-major uint8, uniform digits.

    `row_start`/`row_count` regenerate a band of rows of the same matrix
    without building the rest (used to sample full-size databases).
    p must be a power of two in [2, 256].
    """
    if p < 2 or p > 256 or (p & (p - 1)):
        raise ValueError("p must be a power of two in [2, 256]")
    if row_count is None:
        row_count = rows - row_start
    band = max(1, (64 << 20) // max(cols, 1))
    if row_count > band:
        # generate in 64 MiB bands to bound host memory
        out = np.empty((row_count, cols), dtype=np.uint8)
        for r in range(0, row_count, band):
            k = min(band, row_count - r)
            out[r:r + k] = db_digits(rows, cols, p, seed, row_start + r, k)
        return out
    total = row_count * cols
    first = row_start * cols
    # eight digits per 64-bit output; regenerate the covering range of outputs
    w0 = first // 8
    w1 = (first + total + 7) // 8
    words = stream_u64(seed, TAG_DB, w0, w1 - w0)
    b = words.view(np.uint8)[first - 8 * w0: first - 8 * w0 + total]
    if p != 256:
        b = b & np.uint8(p - 1)
    return np.ascontiguousarray(b.reshape(row_count, cols))


def uniform_u32(count: int, seed: int, tag: int, start: int = 0) -> np.ndarray:
    """Uniform words of Z_{2^32} (upper halves of the stream outputs)."""
    return (stream_u64(seed, tag, start, count) >> np.uint64(32)).astype(np.uint32)


def public_matrix(cols: int, n: int, seed: int) -> np.ndarray:
    """A uniform C x n matrix over Z_{2^32} drawn from the input streams.

    This is an explicit-array A for tests that want one; the scheme's own
    Setup derives A from its seed with a SplitMix64 counter (see the oracle
    and the CUDA Setup kernel).
    """
    return uniform_u32(cols * n, seed, TAG_A).reshape(cols, n)


def secrets(batch: int, n: int, seed: int) -> np.ndarray:
    """Client secrets s, one row of Z_{2^32}^n per query (uniform)."""
    return uniform_u32(batch * n, seed, TAG_S).reshape(batch, n)


@dataclass(frozen=True)
class NoiseTable:
    """Cumulative table of a rounded Gaussian, tail-cut at +-bound."""
    sigma: float
    bound: int
    values: np.ndarray      # int32, -bound .. bound
    cdf: np.ndarray         # uint64 thresholds scaled to 2^63


def noise_table(sigma: float = 6.4, bound: int | None = None) -> NoiseTable:
    """P(e = k) = Phi((k + 1/2)/sigma) - Phi((k - 1/2)/sigma), |k| <= bound.

    The bound defaults to 10 sigma; the table is renormalised after the cut.
    """
    if bound is None:
        bound = int(math.ceil(10 * sigma))
    ks = np.arange(-bound, bound + 1)
    phi = lambda x: 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))
    pk = np.array([phi((k + 0.5) / sigma) - phi((k - 0.5) / sigma) for k in ks])
    pk = pk / pk.sum()
    cdf = np.cumsum(pk)
    cdf[-1] = 1.0
    scaled = np.minimum(np.floor(cdf * 2.0 ** 63), 2.0 ** 63).astype(np.float64)
    thr = np.array([int(v) for v in scaled], dtype=np.uint64)
    thr[-1] = np.uint64(1 << 63)
    return NoiseTable(sigma, bound, ks.astype(np.int32), thr)


def noise(count: int, seed: int, sigma: float = 6.4, start: int = 0,
          table: NoiseTable | None = None) -> np.ndarray:
    """Rounded-Gaussian noise e (int32) by inversion of the cumulative table."""
    t = table if table is not None else noise_table(sigma)
    u = stream_u64(seed, TAG_E, start, count) >> np.uint64(1)   # 63-bit uniform
    idx = np.searchsorted(t.cdf, u, side="right")
    return t.values[np.minimum(idx, len(t.values) - 1)]


def noise_batch(batch: int, cols: int, seed: int, sigma: float = 6.4) -> np.ndarray:
    return noise(batch * cols, seed, sigma).reshape(batch, cols)


def target_columns(batch: int, cols: int, seed: int) -> np.ndarray:
    """Uniform target record indices in [0, cols) (int64)."""
    u = stream_u64(seed, TAG_COL, 0, batch)
    return ((u >> np.uint64(32)) * np.uint64(cols) >> np.uint64(32)).astype(np.int64)


def poisson_arrivals(rate_qps: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    u = (stream_u64(seed, TAG_ARRIVAL, 0, count) >> np.uint64(11)).astype(np.float64)
    u = (u + 0.5) / float(1 << 53)
    return np.cumsum(-np.log(u) / rate_qps)


def skewed_choice(count: int, weights, seed: int) -> np.ndarray:
    """Indices drawn with the given weights (e.g. 60/25/10/5 across databases)."""
    w = np.asarray(weights, dtype=np.float64)
    c = np.cumsum(w / w.sum())
    u = (stream_u64(seed, TAG_MISC, 0, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return np.minimum(np.searchsorted(c, u, side="right"), len(w) - 1).astype(np.int64)


# Named workloads: sizes of the spectrum-database configurations measured here.
def chor_db(rows: int, bits: int, seed: int) -> np.ndarray:
    """Chor database: rows x bits uniform bits, packed rows x (bits / 32) uint32 words."""
    if bits % 32:
        raise ValueError("bits must be a multiple of 32")
    return uniform_u32(rows * (bits // 32), seed, TAG_DB).reshape(rows, bits // 32)


def chor_queries(batch: int, rows: int, seed: int) -> np.ndarray:
    """Uniformly random rows-bit query vectors (what each server sees), packed
    batch x ceil(rows / 32) words, bits at positions >= rows cleared."""
    qw = (rows + 31) // 32
    Q = uniform_u32(batch * qw, seed, TAG_MISC).reshape(batch, qw)
    if rows % 32:
        Q[:, -1] &= np.uint32((1 << (rows % 32)) - 1)
    return Q


def sorted_entries(n: int, seed: int, max_gap: int) -> np.ndarray:
    """n sorted 32-bit entries (uint32): a seeded start plus cumulative gaps uniform in
    [0, max_gap], the shape of sorted spectrum records (frequencies, times) whose
    neighbours are close.  The sums wrap mod 2^32 only if n * max_gap exceeds it."""
    u = stream_u64(seed, TAG_MISC, 0, n + 1)
    gaps = (u[1:] >> np.uint64(32)) * np.uint64(max_gap + 1) >> np.uint64(32)
    start = u[0] >> np.uint64(40)   # below 2^24
    return ((start + np.cumsum(gaps, dtype=np.uint64)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


WORKLOADS = {
    "tiny": dict(rows=1024, cols=1024, n=512, p=256, sigma=6.4),
    "single_1gib": dict(rows=32768, cols=32768, n=1024, p=256, sigma=6.4),
    "batched_1gib": dict(rows=32768, cols=32768, n=1024, p=256, sigma=6.4, batch=256),
    "hint_1gib": dict(rows=32768, cols=32768, n=1024, p=256, sigma=6.4, batch=1024),
    "serving": dict(dbs=[(4096, 4096), (16384, 16384), (32768, 32768), (65536, 32768)],
                    n=1024, p=256, sigma=6.4, skew=(0.60, 0.25, 0.10, 0.05)),
    # Chor Response over GF(2): 1 GiB of bits, 32768 records of 32 KiB (262144 bits)
    "chor_1gib": dict(rows=32768, bits=262144, batches=(1, 8, 32, 128, 256, 1024)),
    # Sec. 5.3 compression: 2^28 sorted 32-bit entries (1 GiB as plain blocks of 8192 entries,
    # i.e. the 32768 x 32768 database) with gaps uniform in [0, 31], so differences fit one byte
    "delta_1gib": dict(entries=1 << 28, block=8192, max_gap=31, n=1024, p=256, sigma=6.4),
}
