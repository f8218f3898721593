"""fp64 oracle of the MLP fork/join job (branch A: GELU MLP; branch B: LayerNorm; join A + B).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product package.

The job's DAG (Sec. 4.1: a job is a DAG of copy and kernel nodes) forks after
the input copy into
  A = GELU(x W1^T) W2^T        (W1 [F, D], W2 [D, F], out_features x in_features)
  B = (x - mu) / sqrt(var + 1e-5)  per row, biased variance, no affine
and joins as out = A + B.  Everything is computed in fp64 from the bf16 values
of x, W1 and W2 with no intermediate rounding.  The matrix products are the
library matmul (a plain definition); GELU is the exact erf form
0.5 v (1 + erf(v / sqrt 2)), evaluated through erfc.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

LN_EPS = 1e-5


def gelu(v: np.ndarray) -> np.ndarray:
    # 0.5 v (1 + erf(v / sqrt 2)) written as 0.5 v erfc(-v / sqrt 2): the same function,
    # without the cancellation of 1 + erf(t) for t << 0.
    return 0.5 * v * erfc(-v / math.sqrt(2.0))


def layernorm(x: np.ndarray, eps: float = LN_EPS) -> np.ndarray:
    mu = x.mean(axis=1, keepdims=True)
    var = ((x - mu) ** 2).mean(axis=1, keepdims=True)
    return (x - mu) / np.sqrt(var + eps)


def branch_a(x: np.ndarray, w1: np.ndarray, w2: np.ndarray) -> np.ndarray:
    h = gelu(x @ w1.T)
    return h @ w2.T


def mlp_ln(x: np.ndarray, w1: np.ndarray, w2: np.ndarray) -> np.ndarray:
    """out = GELU(x W1^T) W2^T + LayerNorm(x), all fp64."""
    x = np.asarray(x, np.float64)
    return branch_a(x, np.asarray(w1, np.float64), np.asarray(w2, np.float64)) + layernorm(x)
