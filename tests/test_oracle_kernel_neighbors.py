"""Pins of the oracle's smoothing kernel, cell keys and neighbour search (CPU only).

Each pin checks the oracle against something other than itself: the kernel's
normalisation integral (Sec. "Kernel function": int W dV = 1), finite differences,
brute force O(N^2) neighbour search, and hand-computed Morton keys.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I


@pytest.mark.parametrize("dim,h", [(2, 0.3), (2, 0.5), (3, 0.3), (1, 0.4)])
def test_kernel_normalisation(dim, h):
    # int W dV = 1 in d dimensions (radial measure 2 for 1D, 2 pi r, 4 pi r^2)
    meas = {1: lambda r: 2.0, 2: lambda r: 2.0 * math.pi * r, 3: lambda r: 4.0 * math.pi * r * r}[dim]
    val = sum(integrate.quad(lambda r: O.W(r, h, dim) * meas(r), lo, hi, epsabs=1e-14, epsrel=1e-13)[0]
              for lo, hi in [(0.0, h), (h, 2.0 * h)])
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_shape_and_gradient(dim):
    h = 0.3
    # compact support, continuity of W and dW/dr at q = 1 and q = 2
    for q in (1.0, 2.0):
        r = q * h
        assert abs(O.W(r * (1 - 1e-12), h, dim) - O.W(r * (1 + 1e-12), h, dim)) < 1e-9
        assert abs(O.dWdr(r * (1 - 1e-12), h, dim) - O.dWdr(r * (1 + 1e-12), h, dim)) < 1e-8
    assert O.W(2.0 * h * (1 + 1e-9), h, dim) == 0.0
    # dW/dr against a central difference of W
    for r in np.linspace(0.01, 0.59, 41):
        eps = 1e-6
        fd = (O.W(r + eps, h, dim) - O.W(r - eps, h, dim)) / (2 * eps)
        assert abs(fd - O.dWdr(r, h, dim)) < 1e-6 * max(1.0, abs(fd))
    # W decreases monotonically on [0, 2h]
    ws = [O.W(r, h, dim) for r in np.linspace(0, 2 * h, 200)]
    assert all(a >= b for a, b in zip(ws, ws[1:]))


def test_morton_keys_by_hand():
    import ctypes as C
    lib = O.lib()

    def key(dim, c):
        arr = np.array(c + [0] * (3 - len(c)), dtype=np.int32)
        return lib.oc_morton(dim, arr.ctypes.data_as(C.c_void_p))

    # bit (dim*b + d) of the key is bit b of coordinate d
    assert key(2, [1, 0]) == 1 and key(2, [0, 1]) == 2 and key(2, [1, 1]) == 3
    assert key(2, [2, 0]) == 4 and key(2, [3, 3]) == 15 and key(2, [0, 4]) == 32
    assert key(3, [0, 0, 1]) == 4 and key(3, [1, 1, 1]) == 7 and key(3, [2, 0, 0]) == 8
    assert key(3, [0, 2, 0]) == 16 and key(3, [5, 0, 0]) == 1 + 64


def _faces_and_boundary_points(h):
    """Points exactly on cell faces and pairs exactly at r = 2h (which are not neighbours).
    All coordinates are dyadic rationals, so the distances are exact in binary."""
    two_h = 2.0 * h  # 0.625 for h = 0.3125
    pts = [(0.0, 0.0), (two_h, 0.0), (0.0, two_h), (2 * two_h, two_h), (two_h * 0.5, two_h * 1.5),
           (0.25, 0.375), (0.25 + two_h, 0.375), (1.0, 1.0), (1.375, 1.5)]
    return np.array(pts).T.copy()


@pytest.mark.parametrize("dim,n,seed", [(2, 400, 11), (3, 400, 12), (2, 1, 13), (3, 60, 14)])
def test_cells_equal_brute_force(dim, n, seed):
    h = 0.3
    x = I.random_points(n, dim, 1.5, seed)
    a1, b1 = O.neighbors(x, h, "brute")
    a2, b2 = O.neighbors(x, h, "cells")
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    # every particle is its own neighbour, the relation is symmetric
    assert np.sum(a1 == b1) == n
    pairs = set(zip(a1.tolist(), b1.tolist()))
    assert all((b, a) in pairs for a, b in pairs)


def test_boundary_cases():
    h = 0.3125
    x = _faces_and_boundary_points(h)
    a1, b1 = O.neighbors(x, h, "brute")
    a2, b2 = O.neighbors(x, h, "cells")
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    pairs = set(zip(a1.tolist(), b1.tolist()))
    assert (0, 1) not in pairs  # exactly r = 2h apart: W(2h) = 0, excluded
    assert (5, 6) not in pairs
    assert (7, 8) not in pairs  # 3-4-5 triangle (0.375, 0.5, 0.625) at r = 2h
    # duplicate points (r = 0) are neighbours
    x2 = np.concatenate([x, x[:, :2]], axis=1)
    a3, b3 = O.neighbors(x2, h, "cells")
    assert (0, x.shape[1]) in set(zip(a3.tolist(), b3.tolist()))


def test_sort_permutation():
    x = I.random_points(500, 2, 2.0, 21)
    cc, keys, perm = O.sort_by_cell(x, 0.3)
    # sorted by (key, id), and a permutation
    k = keys[perm]
    assert np.all((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (perm[1:] > perm[:-1])))
    assert np.array_equal(np.sort(perm), np.arange(500))
    # cell coordinates by the definition floor((x - min x) / (2h))
    xmin = x.min(axis=1, keepdims=True)
    assert np.array_equal(cc, np.floor((x - xmin) * (1.0 / 0.6)).astype(np.int32))
