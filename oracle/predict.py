"""Plain CPU oracle of KNN prediction on top of a KNN result.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and the
benchmark's CPU leg call it; the CUDA path shares nothing with it.

Sec. I of the paper: the predicted output of a query is computed from its
neighbours' values -- a majority vote for discrete classification, an
average for continuous regression.  Readings fixed here (the paper gives no
tie rule or precision):

* vote: over the valid neighbours (id >= 0), the label with the largest
  count; among equal counts the smallest label; no valid neighbour -> -1.
* mean: FP32 running sum of the valid neighbours' values in rank order
  (nearest first, starting from +0), divided in FP32 by their count; no
  valid neighbour -> NaN.
"""
from __future__ import annotations

import numpy as np


def knn_vote(ids: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """Majority label of each row of ids [m][k] (ids index labels [n])."""
    ids = np.asarray(ids)
    labels = np.asarray(labels, dtype=np.int32)
    out = np.full(ids.shape[0], -1, np.int32)
    for r in range(ids.shape[0]):
        row = ids[r]
        v = row[(row >= 0) & (row < labels.shape[0])]
        if v.size == 0:
            continue
        vals, counts = np.unique(labels[v], return_counts=True)   # ascending labels
        out[r] = vals[int(np.argmax(counts))]                     # first maximum: smallest label
    return out


def knn_mean(ids: np.ndarray, values: np.ndarray) -> np.ndarray:
    """FP32 mean of the neighbours' values, summed in rank order."""
    ids = np.asarray(ids)
    values = np.asarray(values, dtype=np.float32)
    m, k = ids.shape
    valid = (ids >= 0) & (ids < values.shape[0])
    gathered = values[np.where(valid, ids, 0)]
    s = np.zeros(m, np.float32)
    for j in range(k):
        # adding +0 for an invalid entry leaves a round-to-nearest sum unchanged
        s = (s + np.where(valid[:, j], gathered[:, j], np.float32(0.0))).astype(np.float32)
    cnt = valid.sum(axis=1)
    out = np.full(m, np.nan, np.float32)
    nz = cnt > 0
    out[nz] = (s[nz] / cnt[nz].astype(np.float32)).astype(np.float32)
    return out
