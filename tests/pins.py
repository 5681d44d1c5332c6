"""Independent references used to pin the oracle (test helpers only).

Nothing here calls the oracle.  Each helper computes a quantity the method
must reproduce, from a definition other than the raster scan:

* :func:`dijkstra_distance` - multi-source shortest paths on the 8- (2D) or
  26-connected (3D) grid with initial potentials v*M, via scipy's Dijkstra
  (library routine) on a graph with one extra source node.
* :func:`brute_force_paths` - minimum over every simple path (tiny grids).
* :func:`line_brute_force_f32` - 1D inputs: for each source, sums the edge
  costs outward one step at a time in float32 and takes the minimum.
* :func:`load_golden` - hand-derived fixtures under tests/golden/.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _spatial_offsets(ndim):
    rng = (-1, 0, 1)
    return [o for o in itertools.product(*([rng] * ndim)) if any(o)]


def _edge_weight(img_x, img_y, off, spacing, lam):
    """Geodesic/Euclidean mixture cost of one grid edge, float64."""
    s2 = sum((o * s) ** 2 for o, s in zip(off, spacing))
    di2 = float(np.sum((img_x - img_y) ** 2))
    return np.sqrt((1.0 - lam) * s2 + lam * di2)


def dijkstra_distance(image, mask, v, lam, spacing=None):
    """image (C, *spatial), mask (*spatial); returns float64 distances."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra

    image = np.asarray(image, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    spatial = mask.shape
    ndim = len(spatial)
    if spacing is None:
        spacing = (1.0,) * ndim
    n = int(np.prod(spatial))
    idx = np.arange(n).reshape(spatial)
    rows, cols, wts = [], [], []
    for off in _spatial_offsets(ndim):
        src = tuple(slice(max(0, -o), s - max(0, o)) for o, s in zip(off, spatial))
        dst = tuple(slice(max(0, o), s - max(0, -o)) for o, s in zip(off, spatial))
        a = idx[src].ravel()
        b = idx[dst].ravel()
        if a.size == 0:
            continue
        s2 = sum((o * s) ** 2 for o, s in zip(off, spacing))
        di2 = np.sum((image[(slice(None),) + src] - image[(slice(None),) + dst]) ** 2,
                     axis=0).ravel()
        w = np.sqrt((1.0 - lam) * s2 + lam * di2)
        rows.append(a)
        cols.append(b)
        wts.append(w)
    # extra source node n -> every element, weight v*M + 1 (the +1 keeps every
    # weight strictly positive so that no edge is dropped as an implicit zero)
    rows.append(np.full(n, n))
    cols.append(np.arange(n))
    wts.append(v * mask.ravel() + 1.0)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    w = np.concatenate(wts)
    # zero-cost grid edges (lambda = 1, equal intensities) are stored as a
    # tiny positive value below the comparison tolerance
    w = np.where(w == 0, 1e-300, w)
    g = coo_matrix((w, (r, c)), shape=(n + 1, n + 1)).tocsr()
    d = dijkstra(g, directed=True, indices=n)
    return (d[:n] - 1.0).reshape(spatial)


def brute_force_paths(image, mask, v, lam, spacing=None):
    """Minimum over all simple paths from every element (tiny grids only)."""
    image = np.asarray(image, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    spatial = mask.shape
    ndim = len(spatial)
    if spacing is None:
        spacing = (1.0,) * ndim
    coords = list(itertools.product(*[range(s) for s in spatial]))
    nbrs = {}
    for c in coords:
        lst = []
        for off in _spatial_offsets(ndim):
            y = tuple(ci + oi for ci, oi in zip(c, off))
            if all(0 <= yi < s for yi, s in zip(y, spatial)):
                w = _edge_weight(image[(slice(None),) + c], image[(slice(None),) + y], off,
                                 spacing, lam)
                lst.append((y, w))
        nbrs[c] = lst
    best = {c: np.inf for c in coords}

    def dfs(node, cost, seen):
        if cost < best[node]:
            best[node] = cost
        for y, w in nbrs[node]:
            if y not in seen:
                seen.add(y)
                dfs(y, cost + w, seen)
                seen.remove(y)

    for s in coords:
        dfs(s, v * mask[s], {s})
    out = np.empty(spatial)
    for c in coords:
        out[c] = best[c]
    return out


def line_brute_force_f32(image_line, mask_line, v, lam, step_spacing=1.0):
    """Exact float32 answer for a 1D input (one line of n elements).

    image_line: (C, n).  Every path to x is the straight walk from some source
    s; its cost is D0[s] plus the edge costs summed one step at a time towards
    x, which is the order in which a sweep adds them.  Costs follow the
    mixture formula with s2 = step_spacing^2, evaluated in float32.
    """
    f = np.float32
    img = np.asarray(image_line, dtype=f)
    m = np.asarray(mask_line, dtype=f)
    n = m.shape[0]
    lam = f(lam)
    one = f(1)
    sp = f(step_spacing)
    s2 = f(sp * sp)
    t = f((one - lam) * s2)

    def cost(i, j):
        di2 = f(0)
        for ch in range(img.shape[0]):
            d = f(img[ch, i] - img[ch, j])
            di2 = f(di2 + f(d * d))
        return f(np.sqrt(f(t + f(lam * di2))))

    d0 = (f(v) * m).astype(f)
    best = d0.copy()
    for s in range(n):
        acc = d0[s]
        for x in range(s + 1, n):
            acc = f(acc + cost(x, x - 1))
            best[x] = min(best[x], acc)
        acc = d0[s]
        for x in range(s - 1, -1, -1):
            acc = f(acc + cost(x, x + 1))
            best[x] = min(best[x], acc)
    return best


def load_golden(name):
    """Parses a key = value fixture; numbers may be decimal or hex floats."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, val = (s.strip() for s in line.split("=", 1))
            toks = val.split()
            nums = [float.fromhex(t) if t.startswith(("0x", "-0x")) else float(t) for t in toks]
            out[k] = nums if len(nums) > 1 else nums[0]
    return out
