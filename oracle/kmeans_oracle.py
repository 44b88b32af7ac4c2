"""FP64 CPU oracle of the segmentation stage: k-means on an embedding.

TEST INFRASTRUCTURE ONLY.  Only the test-suite may import this module; the
CUDA library never calls it and shares no code with it.

Sec. IV (experiments): the segmentation is obtained "by k-means clustering on
the embeddings" (the rows of the embedding are the points).  The paper does
not state the initialisation or the stopping rule; this build uses
* a deterministic maximin start: centroid 0 is row 0, centroid t+1 the row
  farthest (squared Euclidean) from its nearest chosen centroid, ties to the
  smallest row index;
* Lloyd iterations: every row to its nearest centroid (ties to the smallest
  cluster index), every centroid to the mean of its rows (an empty cluster
  keeps its centroid), until no label changes or max_iter rounds.
Distances are accumulated over the columns in order, in FP64.
"""
from __future__ import annotations

import numpy as np


def sq_dist(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """|x_i - c_j|^2 for all rows i and centroids j, summed over columns in order."""
    D = np.zeros((X.shape[0], C.shape[0]))
    for c in range(X.shape[1]):
        diff = X[:, c][:, None] - C[:, c][None, :]
        D += diff * diff
    return D


def maximin_init(X: np.ndarray, k: int) -> np.ndarray:
    """Deterministic start: row 0, then repeatedly the farthest row."""
    C = [X[0].copy()]
    mind = sq_dist(X, X[0:1])[:, 0]
    for _ in range(1, k):
        i = int(np.argmax(mind))  # first maximum: smallest index on ties
        C.append(X[i].copy())
        mind = np.minimum(mind, sq_dist(X, X[i:i + 1])[:, 0])
    return np.array(C)


def lloyd(X: np.ndarray, C0: np.ndarray, max_iter: int = 100):
    """Lloyd's k-means from centroids C0: (labels, centroids, inertia, rounds)."""
    C = np.array(C0, dtype=np.float64, copy=True)
    labels = np.full(X.shape[0], -1, dtype=np.int64)
    rounds = 0
    for rounds in range(1, max_iter + 1):
        new = np.argmin(sq_dist(X, C), axis=1)  # first minimum: smallest cluster index
        changed = np.any(new != labels)
        labels = new
        for j in range(C.shape[0]):
            m = labels == j
            if np.any(m):
                C[j] = X[m].mean(axis=0)
        if not changed:
            break
    inertia = float(np.sum(np.min(sq_dist(X, C), axis=1)))
    return labels, C, inertia, rounds


def kmeans(X: np.ndarray, k: int, max_iter: int = 100):
    """Maximin start + Lloyd: (labels, centroids, inertia, rounds)."""
    return lloyd(X, maximin_init(X, k), max_iter)
