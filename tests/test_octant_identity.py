"""The identity behind the stencil kernel's mask-free octant contributions, checked by brute force
on small grids (host arithmetic only; the kernel's results are checked against the oracle in the
GPU tests).

c_o(v) sums (-1)^dim w(cell) over the cells whose sign corner for octant o is v, a cell's weight
being the max of its vertex weights.  The kernel lets every vertex outside the grid stand in with
weight S = 2^31 - 1 and sums over all 2^n axis subsets without existence masks, in wrapping 32-bit
arithmetic; the stand-in terms cancel except at a grid corner of o, where c_o = w(v).
"""
import itertools

import numpy as np

S = 2**31 - 1


def _cell_max(w, v, o, e, n, L, sentinel):
    m = None
    for sub in itertools.product([0, 1], repeat=n):
        if any(sub[a] and not e[a] for a in range(n)):
            continue
        u = tuple(v[a] + (sub[a] * (-1 if (o >> a) & 1 else 1)) for a in range(n))
        inside = all(0 <= u[a] < L[a] for a in range(n))
        if not inside and not sentinel:
            return None
        x = int(w[u]) if inside else S
        m = x if m is None else max(m, x)
    return m


def _by_definition(w, v, o, n, L):
    tot = 0
    for e in itertools.product([0, 1], repeat=n):
        m = _cell_max(w, v, o, e, n, L, sentinel=False)
        if m is not None:
            tot += (-1) ** sum(e) * m
    return tot


def _mask_free(w, v, o, n, L):
    acc = 0
    for e in itertools.product([0, 1], repeat=n):
        acc = (acc + (-1) ** sum(e) * _cell_max(w, v, o, e, n, L, sentinel=True)) % 2**32
    inside = any(0 <= v[a] + (-1 if (o >> a) & 1 else 1) < L[a] for a in range(n))
    if not inside:
        return int(w[tuple(v)])
    return acc - 2**32 if acc >= 2**31 else acc


def test_mask_free_octant_sums_equal_the_definition():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3):
        for _ in range(12):
            L = tuple(int(x) for x in rng.integers(1, 5, n))          # axis lengths 1..4, corners included
            w = rng.integers(-(2**20), 2**20, L)
            for v in itertools.product(*[range(x) for x in L]):
                for o in range(2**n):
                    assert _mask_free(w, v, o, n, L) == _by_definition(w, v, o, n, L), (n, L, v, o)
