"""Brute-force neighbor pairs with minimum-image periodic boundaries (FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Definition followed (Sec. 2.5.1, "Neighbor search and periodic boundary
conditions"): the edges of the graph are all ordered pairs (i, j), i != j,
of atoms in the same system (the batch vector's sample) whose distance is
below the cutoff; with periodic boundaries the distance is that of the
nearest periodic image.  The paper's brute-force strategy tests every pair
of the system, first for the batch and then for the distance; this module
does the same on the CPU.

Readings (the paper does not state them):
  * self pairs are excluded; the pair is kept when d < cutoff (strict);
  * the pair vector is r_ij = r_i - r_j and atom i is the receiver;
  * boxes are given as rows a, b, c of a lower-triangular matrix
    (a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)), rectangular or triclinic;
    the nearest image is taken by removing c*round(z/cz), then
    b*round(y/by), then a*round(x/ax).  That leaves r in the brick
    |x| <= ax/2, |y| <= by/2, |z| <= cz/2, which holds exactly one image of
    every vector.  The perpendicular widths obey w_c = cz, w_b <= by and
    w_a <= ax, so when all of them are >= 2*cutoff an image shorter than
    the cutoff lies in that brick: the pair set (d < cutoff) and the vectors
    of those pairs are exact, for any such box, reduced or not.

Pinned by: a second search that enumerates the 27 periodic images
explicitly, and scipy's k-d tree (tests/test_oracle_neighbors.py).
"""
from __future__ import annotations

import numpy as np


def box_widths(box: np.ndarray) -> np.ndarray:
    """Perpendicular widths of a lower-triangular box (rows a, b, c)."""
    a, b, c = (np.asarray(box, dtype=np.float64)[k] for k in range(3))
    vol = abs(np.dot(a, np.cross(b, c)))
    return np.array([vol / np.linalg.norm(np.cross(b, c)),
                     vol / np.linalg.norm(np.cross(c, a)),
                     vol / np.linalg.norm(np.cross(a, b))])


def check_box(box: np.ndarray, cutoff: float) -> None:
    """Raise ValueError unless the box is lower-triangular with every
    perpendicular width at least twice the cutoff."""
    B = np.asarray(box, dtype=np.float64)
    if B[0, 1] != 0 or B[0, 2] != 0 or B[1, 2] != 0:
        raise ValueError("box must be lower-triangular (a along x, b in the xy plane)")
    if np.any(np.diag(B) <= 0):
        raise ValueError("box diagonal must be positive")
    if np.any(box_widths(B) < 2.0 * cutoff):
        raise ValueError("box narrower than twice the cutoff")


def minimum_image(r: np.ndarray, box: np.ndarray | None) -> np.ndarray:
    """Nearest periodic image of pair vectors r [..., 3] for one box, or
    r unchanged when box is None."""
    r = np.array(r, dtype=np.float64, copy=True)
    if box is None:
        return r
    B = np.asarray(box, dtype=np.float64)
    r -= np.round(r[..., 2] / B[2, 2])[..., None] * B[2]
    r -= np.round(r[..., 1] / B[1, 1])[..., None] * B[1]
    r -= np.round(r[..., 0] / B[0, 0])[..., None] * B[0]
    return r


def _systems(batch: np.ndarray) -> list[np.ndarray]:
    b = np.asarray(batch)
    return [np.nonzero(b == s)[0] for s in np.unique(b)]


def neighbor_rows(pos, batch, box, cutoff: float, rows) -> list[np.ndarray]:
    """For each atom i in `rows`, the sorted array of j with (i, j) an edge."""
    pos = np.asarray(pos, dtype=np.float64)
    batch = np.asarray(batch)
    out = []
    for i in rows:
        s = batch[i]
        cand = np.nonzero(batch == s)[0]
        cand = cand[cand != i]
        B = None if box is None else np.asarray(box, np.float64)[s]
        r = minimum_image(pos[i] - pos[cand], B)
        d2 = np.einsum("ek,ek->e", r, r)
        out.append(np.sort(cand[d2 < cutoff * cutoff]))
    return out


def neighbor_pairs(pos, batch, box, cutoff: float, block: int = 2048):
    """All edges (i, j), sorted by i then j.  Returns (i, j) int64 arrays.

    O(N^2) per system: every pair of the system is tested (the CPU
    counterpart of the paper's thread-per-pair brute-force kernel)."""
    pos = np.asarray(pos, dtype=np.float64)
    ii, jj = [], []
    for s_idx, atoms in enumerate(_systems(batch)):
        s = int(np.asarray(batch)[atoms[0]])
        B = None if box is None else np.asarray(box, np.float64)[s]
        if B is not None:
            check_box(B, cutoff)
        P = pos[atoms]
        n = len(atoms)
        for a0 in range(0, n, block):
            a1 = min(n, a0 + block)
            r = minimum_image(P[a0:a1, None, :] - P[None, :, :], B)
            d2 = np.einsum("abk,abk->ab", r, r)
            mask = d2 < cutoff * cutoff
            mask[np.arange(a1 - a0), np.arange(a0, a1)] = False
            a, b = np.nonzero(mask)
            ii.append(atoms[a + a0])
            jj.append(atoms[b])
    if not ii:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    i = np.concatenate(ii).astype(np.int64)
    j = np.concatenate(jj).astype(np.int64)
    order = np.lexsort((j, i))
    return i[order], j[order]


def neighbor_pairs_images(pos, batch, box, cutoff: float, reach: int = 1):
    """Independent check of `neighbor_pairs` for small inputs: for every
    pair of the same system, enumerate the periodic images n.B with
    n in {-reach..reach}^3 of r_i - r_j (after wrapping both atoms into the
    cell) and keep the pair when any image is within the cutoff.  reach = 1
    (27 images) covers rectangular boxes; strongly tilted cells need 2."""
    pos = np.asarray(pos, dtype=np.float64)
    batch = np.asarray(batch)
    N = len(pos)
    ii, jj = [], []
    rr = range(-reach, reach + 1)
    shifts = np.array([[a, b, c] for a in rr for b in rr for c in rr], dtype=np.float64)
    for i in range(N):
        for j in range(N):
            if i == j or batch[i] != batch[j]:
                continue
            if box is None:
                ok = np.linalg.norm(pos[i] - pos[j]) < cutoff
            else:
                B = np.asarray(box, np.float64)[batch[i]]
                Binv = np.linalg.inv(B)
                fi = pos[i] @ Binv
                fj = pos[j] @ Binv
                wi = (fi - np.floor(fi)) @ B
                wj = (fj - np.floor(fj)) @ B
                imgs = (wi - wj)[None, :] + shifts @ B
                ok = bool(np.any(np.linalg.norm(imgs, axis=1) < cutoff))
            if ok:
                ii.append(i)
                jj.append(j)
    return np.array(ii, np.int64), np.array(jj, np.int64)
