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


def exact_floor(f, xi):
    """Smallest float32 >= f - xi, with f - xi taken as an exact rational."""
    from fractions import Fraction
    want = Fraction(float(np.float32(f))) - Fraction(float(np.float32(xi)))
    c = np.float32(float(want))  # nearest double, then nearest float: close, fixed up below
    while Fraction(float(c)) < want:
        c = np.nextafter(c, np.float32(np.inf), dtype=np.float32)
    while True:
        d = np.nextafter(c, np.float32(-np.inf), dtype=np.float32)
        if Fraction(float(d)) >= want:
            c = d
        else:
            return np.float32(c)


def _vertex(i, slot, shape_xyz):
    if slot == 15:
        return i
    c = coords(i, shape_xyz)
    d = slot_offsets(len(shape_xyz))[slot]
    return lin(tuple(a + b for a, b in zip(c, d)), shape_xyz)


def _above(v, j, i):
    return (float(v[j]), j) > (float(v[i]), i)


def brute_sweep(f, g, xi, rule):
    """One synchronous sweep written out from the reading of Sec. III-B / IV-A
    (no oracle code): returns (g', distorted, distinct targets, changed).
    Targets: an ascending mismatch lowers g's steepest ascent of i (i itself
    when g makes i a maximum); a descending mismatch lowers f's steepest
    descent of i (i itself when f makes i a minimum).  Edits: HALVE (0),
    SNAP (1), or BELOW-REFERENCE (2): the target drops to the largest value
    below its reference (f's steepest ascent of i, resp. g's steepest descent
    of i) in the (value, index) order, the smallest request winning; all
    computed from g, at or above the floor."""
    shape_xyz = xyz_shape(f.shape)
    cf = brute_codes(f).reshape(-1)
    cg = brute_codes(g).reshape(-1)
    gf = g.reshape(-1).astype(np.float32)
    ff = f.reshape(-1)
    req = {}
    distorted = 0
    for i in range(gf.size):
        if cf[i] == cg[i]:
            continue
        distorted += 1
        af, ag, df, dg = cf[i] & 15, cg[i] & 15, cf[i] >> 4, cg[i] >> 4
        pairs = []
        if af != ag:
            pairs.append((_vertex(i, int(ag), shape_xyz), _vertex(i, int(af), shape_xyz)))
        if df != dg:
            pairs.append((_vertex(i, int(df), shape_xyz), _vertex(i, int(dg), shape_xyz)))
        for t, r in pairs:
            if r > t:
                c = gf[r]
            else:
                c = np.nextafter(gf[r], np.float32(-np.inf), dtype=np.float32)
            key = (float(c), 0 if np.signbit(c) else 1)  # totalOrder on the candidates
            if t not in req or key < req[t][0]:
                req[t] = (key, np.float32(c))
    out = gf.copy()
    changed = 0
    for t, (_, c) in req.items():
        L = exact_floor(ff[t], xi)
        gt = gf[t]
        if rule == 2:
            h = L if c < L else c
            if not h < gt:
                continue
        else:
            if not gt > L:
                continue
            if rule == 1:
                h = L
            else:
                s = np.float32(gt - L)
                h = np.float32(gt - np.float32(np.float32(0.5) * s))
                if h < L:
                    h = L
                if not h < gt:
                    h = L
        out[t] = h
        changed += 1
    return out.reshape(g.shape), distorted, len(req), changed
