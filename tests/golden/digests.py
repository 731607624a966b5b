"""SHA-256 digests of index arrays and labels, for full-size parity checks.

Plain hashing of raw little-endian array bytes; no part of the clustering
method lives here. ``make_digests.py`` writes the expected digests from the
CPU oracle; the GPU tests hash what the CUDA library exports and compare.
"""
from __future__ import annotations

import hashlib

import numpy as np

INDEX_KEYS = ("sim", "no_id", "no_sim", "co_off", "co_id", "co_thr")
DTYPES = {"sim": "<f8", "no_id": "<i4", "no_sim": "<f8", "co_off": "<i8", "co_id": "<i4",
          "co_thr": "<f8", "labels": "<i4", "off": "<i8", "adj": "<i4"}


def _feed(h, key: str, a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=DTYPES[key])
    h.update(f"{key}:{a.dtype.str}:{a.shape[0]}\n".encode())
    h.update(memoryview(a).cast("B"))


def array_digest(key: str, a: np.ndarray) -> str:
    h = hashlib.sha256()
    _feed(h, key, a)
    return h.hexdigest()


def combined_digest(items, n_hex: int = 64) -> str:
    """One digest over (key, array) pairs in the given order."""
    h = hashlib.sha256()
    for key, a in items:
        _feed(h, key, a)
    return h.hexdigest()[:n_hex]


def graph_digest(g, n_hex: int = 64) -> str:
    return combined_digest((("off", g.off), ("adj", g.adj)), n_hex)


def index_digest(ix: dict, n_hex: int = 64) -> str:
    """ix maps each of INDEX_KEYS to its array (an export or the oracle's index)."""
    return combined_digest(((k, ix[k]) for k in INDEX_KEYS), n_hex)


def labels_digest(labels, n_hex: int = 64) -> str:
    """labels: a sequence of label arrays, one per query, in query order."""
    return combined_digest((("labels", lab) for lab in labels), n_hex)
