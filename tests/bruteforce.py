"""Brute-force references used to pin the oracle on tiny grids.

Nothing here imports the oracle's neighbour table: the neighbourhood is
rebuilt from the simplices of the Kuhn (Freudenthal) triangulation, the order
is Python tuple comparison on (value, index), and integral lines are followed
one step at a time.
"""
from __future__ import annotations

import itertools

import numpy as np


def kuhn_simplices(ndim: int):
    """Vertex lists (as 0/1 offset tuples) of the n! simplices of the unit cube:
    the chains 0 -> e_p1 -> e_p1 + e_p2 -> ... -> (1,..,1) for each permutation p."""
    out = []
    for perm in itertools.permutations(range(ndim)):
        v = [0] * ndim
        chain = [tuple(v)]
        for ax in perm:
            v[ax] = 1
            chain.append(tuple(v))
        out.append(chain)
    return out


def kuhn_neighbours(shape_xyz):
    """Map vertex (x,y[,z]) -> set of neighbour vertices in the triangulated grid."""
    ndim = len(shape_xyz)
    simp = kuhn_simplices(ndim)
    nb = {}
    cells = itertools.product(*[range(max(s - 1, 0)) for s in shape_xyz])
    for c in cells:
        for s in simp:
            verts = [tuple(ci + oi for ci, oi in zip(c, o)) for o in s]
            for a in verts:
                for b in verts:
                    if a != b:
                        nb.setdefault(a, set()).add(b)
    # grids with an axis of length 1 have no full cells along it: triangulate the
    # lower-dimensional grid spanned by the other axes instead
    if any(s == 1 for s in shape_xyz) and ndim > 1:
        keep = [k for k, s in enumerate(shape_xyz) if s > 1]
        if len(keep) < ndim:
            sub = kuhn_neighbours(tuple(shape_xyz[k] for k in keep)) if keep else {}
            nb = {}
            for v, ns in sub.items():
                full = [0] * ndim
                for k, vk in zip(keep, v):
                    full[k] = vk
                for u in ns:
                    fu = [0] * ndim
                    for k, uk in zip(keep, u):
                        fu[k] = uk
                    nb.setdefault(tuple(full), set()).add(tuple(fu))
    return nb


def xyz_shape(np_shape):
    return tuple(reversed(np_shape))


def lin(v, shape_xyz):
    i, stride = 0, 1
    for c, s in zip(v, shape_xyz):
        i += c * stride
        stride *= s
    return i


def coords(i, shape_xyz):
    out = []
    for s in shape_xyz:
        out.append(i % s)
        i //= s
    return tuple(out)


def slot_offsets(ndim):
    """The slot numbering of the public API: positive offsets of {0,1}^n minus 0
    in the documented order, then their negatives in the same order."""
    if ndim == 2:
        pos = [(1, 0), (0, 1), (1, 1)]
    else:
        pos = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    return pos + [tuple(-c for c in p) for p in pos]


def brute_codes(v: np.ndarray) -> np.ndarray:
    """Codes by brute force: n_max / n_min over the Kuhn neighbourhood under the
    (value, index) order; SELF (15) when the vertex itself is the extreme."""
    shape_xyz = xyz_shape(v.shape)
    ndim = len(shape_xyz)
    nb = kuhn_neighbours(shape_xyz)
    offs = slot_offsets(ndim)
    flat = v.reshape(-1)
    out = np.empty(flat.size, dtype=np.uint8)
    for i in range(flat.size):
        c = coords(i, shape_xyz)
        cand = [(float(flat[i]), i, 15)]
        for u in nb.get(c, ()):
            d = tuple(a - b for a, b in zip(u, c))
            j = lin(u, shape_xyz)
            cand.append((float(flat[j]), j, offs.index(d)))
        hi = max(cand, key=lambda t: (t[0], t[1]))
        lo = min(cand, key=lambda t: (t[0], t[1]))
        out[i] = hi[2] | (lo[2] << 4)
    return out.reshape(v.shape)


def brute_labels(codes: np.ndarray):
    """Follow n_min / n_max one step at a time until SELF."""
    shape_xyz = xyz_shape(codes.shape)
    ndim = len(shape_xyz)
    offs = slot_offsets(ndim)
    flat = codes.reshape(-1)
    res = []
    for shift in (4, 0):
        lab = np.empty(flat.size, dtype=np.int32)
        for i in range(flat.size):
            p = i
            steps = 0
            while True:
                s = (int(flat[p]) >> shift) & 15
                if s == 15:
                    break
                c = coords(p, shape_xyz)
                p = lin(tuple(a + b for a, b in zip(c, offs[s])), shape_xyz)
                steps += 1
                assert steps <= flat.size, "integral line longer than the grid"
            lab[i] = p
        res.append(lab.reshape(codes.shape))
    return res[0], res[1]
