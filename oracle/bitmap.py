"""Column-pair comparison bitmap, from its plain definition.

For every ordered pair of distinct columns (a, b) and every 32-row group w, word G[a][b][w] holds
bit j = [x[32w + j, b] > x[32w + j, a]] (strict float32 comparison; rows past the end are 0).
A positive-trend pair (c_k, c_{k+1}) of an individual succeeds on exactly the rows whose bit is set
in G[c_k][c_{k+1}], a negative-trend pair in G[c_{k+1}][c_k] (Sec. 2.3 trend definition, with the
tie reading of ``counts``).  The diagonal words (a == b) are defined as 0.

Test infrastructure only (see the package docstring).
"""

import numpy as np


def pair_words(x, a, b):
    """The words G[a][b][0..ceil(R/32)) of one ordered column pair."""
    x = np.asarray(x, dtype=np.float32)
    R = x.shape[0]
    W = (R + 31) // 32
    if a == b:
        return np.zeros(W, dtype=np.uint32)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    bits = np.zeros(W * 32, dtype=np.uint64)
    bits[:R] = (x[:, b] > x[:, a])
    return (bits.reshape(W, 32) * weights).sum(axis=1).astype(np.uint32)


def pair_bitmap(x):
    x = np.asarray(x, dtype=np.float32)
    R, C = x.shape
    W = (R + 31) // 32
    G = np.zeros((C, C, W), dtype=np.uint32)
    for a in range(C):
        for b in range(C):
            G[a, b] = pair_words(x, a, b)
    return G
