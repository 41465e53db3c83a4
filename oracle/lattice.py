"""Velocity sets for the oracle.  TEST INFRASTRUCTURE (see oracle/__init__).

D2Q9 is built from Eq. 2 (lattice speed c = 1) with the weights of Eq. 9.
D3Q19 is the textbook 3-D set (rest 1/3, six axis links 1/18, twelve
edge-diagonal links 1/36), which the paper does not print.  Vectors are
stored as (e_x, e_y, e_z).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def d2q9():
    E = [(0, 0, 0)]
    for a in range(1, 5):
        ang = (a - 1) * math.pi / 2
        E.append((round(math.cos(ang)), round(math.sin(ang)), 0))
    for a in range(5, 9):
        ang = (a - 5) * math.pi / 2 + math.pi / 4
        E.append((round(math.sqrt(2) * math.cos(ang)), round(math.sqrt(2) * math.sin(ang)), 0))
    W = [4.0 / 9.0] + [1.0 / 9.0] * 4 + [1.0 / 36.0] * 4
    return _finish(E, W)


def d3q19():
    E = [e for e in itertools.product((-1, 0, 1), repeat=3) if sum(c * c for c in e) <= 2]
    E.sort(key=lambda e: (sum(c * c for c in e), e))
    wt = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
    W = [wt[sum(c * c for c in e)] for e in E]
    return _finish(E, W)


def _finish(E, W):
    E = np.array(E, dtype=np.int64)
    W = np.array(W, dtype=np.float64)
    opp = np.array([int(np.where((E == -e).all(axis=1))[0][0]) for e in E])
    return E, W, opp


def for_dim(dim):
    return d2q9() if dim == 2 else d3q19()
