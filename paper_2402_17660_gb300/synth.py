"""Seeded synthetic inputs: geometries, atomic numbers, batch vectors, boxes,
velocities and random-init TensorNet weights.

This module is shared by the FP64 oracle (test infrastructure) and the CUDA
path.  It draws random numbers and lays atoms out in space; it contains none
of the model's arithmetic (no cutoff, basis, message passing or gradient).

The workloads mirror the shapes of the paper's speed and stability
experiments (Sec. 3, "Speed performance", Table tab:prot; "Molecular
Simulations"): single small molecules in vacuum, batches of molecules of
uneven size (Sec. 2.5.1, batch handling), periodic water boxes and a
solvated box from thousands to ~100k atoms.  The paper's molecules, datasets
and trained weights are not available, so every input here is seeded and
synthetic.

Units: positions in Angstrom, masses in amu, velocities in Angstrom/fs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Element table used by the generators (atomic numbers and masses in amu).
Z_H, Z_C, Z_N, Z_O = 1, 6, 7, 8
MASS = {Z_H: 1.008, Z_C: 12.011, Z_N: 14.007, Z_O: 15.999}
KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
EV_PER_AMU_A2_FS2 = 9.64853321e-3  # 1 eV/(Angstrom amu) in Angstrom/fs^2

WATER_OH = 0.9572                # Angstrom
WATER_HOH_DEG = 104.52           # degrees


@dataclasses.dataclass
class System:
    """A batch of one or more systems, packed along the atom axis.

    z      int32 [N]       atomic numbers (embedding indices)
    pos    float32 [N][3]  positions, Angstrom
    batch  int32 [N]       system index of each atom, non-decreasing
    box    float32 [S][3][3] row-vector box per system, or None (no PBC)
    """
    name: str
    z: np.ndarray
    pos: np.ndarray
    batch: np.ndarray
    box: np.ndarray | None
    n_systems: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.z.shape[0])

    def masses(self) -> np.ndarray:
        return np.array([MASS[int(a)] for a in self.z], dtype=np.float32)


@dataclasses.dataclass(frozen=True)
class ModelShape:
    """TensorNet hyperparameters (Sec. 2.4 training example; Table S4):
    embedding dimension F, number of radial basis functions K, number of
    interaction layers L, embedding table size max_z and cutoffs in A."""
    F: int = 128
    K: int = 32
    L: int = 2
    max_z: int = 100
    cutoff_upper: float = 5.0
    cutoff_lower: float = 0.0


# ---------------------------------------------------------------- weights ---

def param_spec(shape: ModelShape) -> list[tuple[str, tuple[int, ...]]]:
    """Names and shapes of every TensorNet parameter, in blob order.

    Linear weights are stored (out, in): y = W x + b.  The three channel
    mixing matrices of a set are indexed [p] with p = 0 (I), 1 (A), 2 (S).
    """
    F, K, L, Zm = shape.F, shape.K, shape.L, shape.max_z
    spec: list[tuple[str, tuple[int, ...]]] = [
        ("emb", (Zm, F)),
        ("emb2_w", (F, 2 * F)), ("emb2_b", (F,)),
        ("dproj_w", (3, F, K)), ("dproj_b", (3, F)),
        ("emb_ln_g", (F,)), ("emb_ln_b", (F,)),
        ("emb_mlp1_w", (2 * F, F)), ("emb_mlp1_b", (2 * F,)),
        ("emb_mlp2_w", (3 * F, 2 * F)), ("emb_mlp2_b", (3 * F,)),
        ("emb_mix_w", (3, F, F)),
    ]
    for l in range(L):
        spec += [
            (f"l{l}_mlp1_w", (F, K)), (f"l{l}_mlp1_b", (F,)),
            (f"l{l}_mlp2_w", (2 * F, F)), (f"l{l}_mlp2_b", (2 * F,)),
            (f"l{l}_mlp3_w", (3 * F, 2 * F)), (f"l{l}_mlp3_b", (3 * F,)),
            (f"l{l}_mix1_w", (3, F, F)),
            (f"l{l}_mix2_w", (3, F, F)),
        ]
    spec += [
        ("out_ln_g", (3 * F,)), ("out_ln_b", (3 * F,)),
        ("out_w", (F, 3 * F)), ("out_b", (F,)),
        ("head1_w", (F // 2, F)), ("head1_b", (F // 2,)),
        ("head2_w", (1, F // 2)), ("head2_b", (1,)),
    ]
    return spec


def init_weights(shape: ModelShape = ModelShape(), seed: int = 0) -> dict[str, np.ndarray]:
    """Seeded random-init weights (the paper gives no initialiser).

    Linear W ~ U(+-sqrt(6/(fan_in+fan_out))), biases ~ U(+-0.1), LayerNorm
    gain ~ U(0.5, 1.5) and shift ~ U(+-0.1), embedding ~ N(0, 1).  Values are
    returned as float32; consumers that compute in FP64 upcast them exactly.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    out: dict[str, np.ndarray] = {}
    for name, shp in param_spec(shape):
        if name == "emb":
            v = rng.standard_normal(shp)
        elif name.endswith("_ln_g"):
            v = rng.uniform(0.5, 1.5, shp)
        elif name.endswith("_ln_b") or name.endswith("_b"):
            v = rng.uniform(-0.1, 0.1, shp)
        else:  # a linear weight (out, in), possibly stacked [3][out][in]
            fan_out, fan_in = shp[-2], shp[-1]
            a = math.sqrt(6.0 / (fan_in + fan_out))
            v = rng.uniform(-a, a, shp)
        out[name] = np.ascontiguousarray(v, dtype=np.float32)
    return out


def md_weights(shape: ModelShape = ModelShape(), seed: int = 0, scale: float = 0.05) -> dict[str, np.ndarray]:
    """Weights for molecular dynamics: `init_weights` with the last output
    layer scaled by `scale`.  Unscaled random-init weights give RMS forces of
    a few eV/A on water, too stiff for 0.5 fs steps with a 1 A skin rebuilt
    every 20 steps; scaled by 0.05 the forces are a few tenths of an eV/A,
    the magnitude of real liquid water."""
    w = init_weights(shape, seed)
    w["head2_w"] = (w["head2_w"] * scale).astype(np.float32)
    w["head2_b"] = (w["head2_b"] * scale).astype(np.float32)
    return w


# --------------------------------------------------------------- geometry ---

def _min_image_np(r: np.ndarray, L: np.ndarray | None) -> np.ndarray:
    """Coordinate-wise nearest periodic image for a rectangular box (used
    only to validate generated geometry against the margin rule)."""
    if L is None:
        return r
    return r - L * np.round(r / L)


def _near_radius_atoms(pos: np.ndarray, L: float | None, radii, margin: float) -> np.ndarray:
    """Indices of atoms in a pair whose distance lies within `margin` of any
    radius in `radii` (brute force in blocks; pos in float64)."""
    from scipy.spatial import cKDTree
    rmax = max(radii) + margin
    if L is not None:
        p = np.mod(pos, L)
        p[p >= L] = 0.0
        tree = cKDTree(p, boxsize=L)
    else:
        p = pos
        tree = cKDTree(p)
    pairs = tree.query_pairs(rmax, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, dtype=np.int64)
    d = np.linalg.norm(_min_image_np(pos[pairs[:, 0]] - pos[pairs[:, 1]],
                                     None if L is None else np.array([L, L, L])), axis=1)
    bad = np.zeros(len(pairs), dtype=bool)
    for R in radii:
        bad |= np.abs(d - R) < margin
    return np.unique(pairs[bad].ravel())


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from random unit quaternions."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_frame() -> np.ndarray:
    """O, H, H positions of a rigid water in its own frame (O at origin)."""
    t = math.radians(WATER_HOH_DEG) / 2
    return np.array([[0.0, 0.0, 0.0],
                     [WATER_OH * math.sin(t), WATER_OH * math.cos(t), 0.0],
                     [-WATER_OH * math.sin(t), WATER_OH * math.cos(t), 0.0]])


def _place_waters(rng, centres: np.ndarray, jitter: float) -> np.ndarray:
    n = len(centres)
    c = centres + rng.uniform(-jitter, jitter, (n, 3))
    R = _random_rotations(rng, n)
    xyz = c[:, None, :] + np.einsum("nab,kb->nka", R, _water_frame())
    return xyz.reshape(-1, 3)


def _fix_margins_waters(rng, centres, jitter, L, radii, margin, max_iter=200):
    """Place waters, then re-place any molecule whose atoms sit in a pair
    within `margin` of a radius in `radii`."""
    xyz = _place_waters(rng, centres, jitter)
    for _ in range(max_iter):
        x32 = np.mod(xyz, L).astype(np.float32).astype(np.float64)
        bad = _near_radius_atoms(x32, L, radii, margin)
        if bad.size == 0:
            return np.mod(xyz, L)
        mols = np.unique(bad // 3)
        xyz = xyz.reshape(-1, 3, 3)
        xyz[mols] = _place_waters(rng, centres[mols], jitter).reshape(-1, 3, 3)
        xyz = xyz.reshape(-1, 3)
    raise RuntimeError("could not satisfy the pair-distance margin")


def random_molecule(rng, n: int, side: float, z: np.ndarray, min_dist=0.9,
                    radii=(5.0,), margin=1e-4) -> np.ndarray:
    """n atoms uniform in a cube of the given side by random sequential
    addition, rejecting a new atom closer than `min_dist` to any placed atom
    or with a pair distance within `margin` of a radius in `radii`."""
    pos = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        p = rng.uniform(0.0, side, 3)
        p32 = p.astype(np.float32).astype(np.float64)
        if k:
            prev = pos[:k].astype(np.float32).astype(np.float64)
            d = np.linalg.norm(prev - p32, axis=1)
            if d.min() < min_dist or any(np.any(np.abs(d - R) < margin) for R in radii):
                tries += 1
                if tries > 100000:
                    raise RuntimeError("molecule packing failed")
                continue
        pos[k] = p
        k += 1
    return pos


def small_molecule(seed: int = 0, radii=(5.0,)) -> System:
    """Single molecule in vacuum: 32 atoms (12 H, 12 C, 4 N, 4 O), uniform
    in a 6 A cube, rejection below 0.9 A."""
    rng = np.random.default_rng(seed)
    z = np.array([Z_H] * 12 + [Z_C] * 12 + [Z_N] * 4 + [Z_O] * 4, dtype=np.int32)
    z = rng.permutation(z).astype(np.int32)
    pos = random_molecule(rng, 32, 6.0, z, radii=radii)
    return System("molecule32", z, pos.astype(np.float32), np.zeros(32, np.int32), None, 1)


def random_cluster(n: int, seed: int, side: float | None = None, radii=(5.0,),
                   min_dist=0.9, elements=(Z_H, Z_C, Z_N, Z_O),
                   probs=(0.5, 0.3, 0.1, 0.1)) -> System:
    """A molecule-like cluster of n atoms in vacuum at the density of the
    32-atom case (side = 6 (n/32)^(1/3) A unless given)."""
    rng = np.random.default_rng(seed)
    if side is None:
        side = 6.0 * (n / 32.0) ** (1.0 / 3.0)
    z = rng.choice(np.array(elements), size=n, p=np.array(probs)).astype(np.int32)
    pos = random_molecule(rng, n, side, z, min_dist=min_dist, radii=radii)
    return System(f"cluster{n}", z, pos.astype(np.float32), np.zeros(n, np.int32), None, 1)


def molecule_batch(n_mol: int = 512, nmin: int = 8, nmax: int = 96, seed: int = 2,
                   radii=(5.0,)) -> System:
    """Batch of independent molecules (atom counts uniform in [nmin, nmax],
    H/C/N/O with p = .5/.3/.1/.1, each packed like the 32-atom molecule in
    a cube scaled to its atom count), packed into one batch vector."""
    rng = np.random.default_rng(seed)
    zs, ps, bs = [], [], []
    for m in range(n_mol):
        n = int(rng.integers(nmin, nmax + 1))
        z = rng.choice(np.array([Z_H, Z_C, Z_N, Z_O]), size=n,
                       p=[0.5, 0.3, 0.1, 0.1]).astype(np.int32)
        side = 6.0 * (n / 32.0) ** (1.0 / 3.0)
        pos = random_molecule(rng, n, side, z, radii=radii)
        zs.append(z)
        ps.append(pos)
        bs.append(np.full(n, m, np.int32))
    return System(f"batch{n_mol}", np.concatenate(zs), np.concatenate(ps).astype(np.float32),
                  np.concatenate(bs), None, n_mol)


def water_box(n_side: int = 10, L: float = 31.04, seed: int = 1, jitter: float = 0.3,
              n_keep: int | None = None, radii=(5.0,), margin=1e-4) -> System:
    """Rigid waters (O-H 0.9572 A, H-O-H 104.52 deg) on a jittered cubic
    lattice of n_side^3 sites with random orientations, in a periodic cube
    of side L; optionally a random subset of n_keep sites."""
    rng = np.random.default_rng(seed)
    a = L / n_side
    g = (np.arange(n_side) + 0.5) * a
    centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if n_keep is not None:
        centres = centres[np.sort(rng.choice(len(centres), n_keep, replace=False))]
    xyz = _fix_margins_waters(rng, centres, jitter, L, radii, margin)
    nw = len(centres)
    z = np.tile(np.array([Z_O, Z_H, Z_H], np.int32), nw)
    box = np.diag([L, L, L]).astype(np.float32)[None]
    return System(f"water{3 * nw}", z, xyz.astype(np.float32), np.zeros(3 * nw, np.int32),
                  box, 1, {"L": L})


def solvated_box(L: float = 62.0, n_solute: int = 2500, step: float = 1.5,
                 min_nonbonded: float = 1.2, n_total: int = 24000, seed: int = 3,
                 radii=(5.0,), margin=1e-4) -> System:
    """Periodic solvated box: a seeded self-avoiding random walk solute
    (1.5 A steps, non-bonded distance >= 1.2 A, H/C/N/O mix) surrounded by
    rigid waters on a lattice at 1 g/cm^3, dropping sites within 2.4 A of
    the solute, then trimmed at random to about n_total atoms."""
    rng = np.random.default_rng(seed)
    cell = min_nonbonded
    nc = int(L // cell)
    grid: dict[tuple[int, int, int], list[int]] = {}

    def key(p):
        return tuple((np.floor(np.mod(p, L) / (L / nc)).astype(int) % nc).tolist())

    def clash(p, skip):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % nc, (k[1] + dy) % nc, (k[2] + dz) % nc)
                    for idx in grid.get(kk, ()):
                        if idx == skip:
                            continue
                        r = _min_image_np(walk[idx] - p, np.array([L, L, L]))
                        if r @ r < min_nonbonded ** 2:
                            return True
        return False

    walk = np.zeros((n_solute, 3))
    walk[0] = rng.uniform(0, L, 3)
    grid.setdefault(key(walk[0]), []).append(0)
    k = 1
    while k < n_solute:
        for _ in range(1000):
            v = rng.standard_normal(3)
            p = walk[k - 1] + step * v / np.linalg.norm(v)
            if not clash(p, k - 1):
                break
        else:
            raise RuntimeError("random walk stuck")
        walk[k] = p
        grid.setdefault(key(p), []).append(k)
        k += 1
    walk = np.mod(walk, L)
    zs = rng.choice(np.array([Z_H, Z_C, Z_N, Z_O]), size=n_solute,
                    p=[0.5, 0.3, 0.1, 0.1]).astype(np.int32)

    # water lattice: the 1 g/cm^3 spacing (3.104 A), refined by one site per
    # edge at a time until enough sites survive the solute exclusion to reach
    # n_total atoms
    from scipy.spatial import cKDTree
    tree = cKDTree(walk, boxsize=L)
    n_w = (n_total - n_solute) // 3
    n_side = int(round(L / 3.104))
    while True:
        a = L / n_side
        g = (np.arange(n_side) + 0.5) * a
        centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        near = tree.query_ball_point(np.mod(centres, L), 2.4)
        centres = centres[np.array([len(x) == 0 for x in near])]
        if len(centres) >= n_w:
            break
        n_side += 1
    if n_w < len(centres):
        centres = centres[np.sort(rng.choice(len(centres), n_w, replace=False))]
    nw = len(centres)

    # place waters, then fix margins over the whole box (waters are re-placed,
    # the solute is left where it is)
    xyz = _place_waters(rng, centres, 0.3)
    for _ in range(200):
        allpos = np.mod(np.concatenate([walk, xyz]), L)
        bad = _near_radius_atoms(allpos.astype(np.float32).astype(np.float64), L, radii, margin)
        badw = bad[bad >= n_solute] - n_solute
        bads = bad[bad < n_solute]
        if bad.size == 0:
            break
        if badw.size == 0 and bads.size:
            # a solute-solute pair on the margin: nudge one solute atom
            walk[bads[0]] += rng.uniform(-1e-3, 1e-3, 3)
            continue
        mols = np.unique(badw // 3)
        xyz = xyz.reshape(-1, 3, 3)
        xyz[mols] = _place_waters(rng, centres[mols], 0.3).reshape(-1, 3, 3)
        xyz = xyz.reshape(-1, 3)
    else:
        raise RuntimeError("could not satisfy the pair-distance margin")
    pos = np.mod(np.concatenate([walk, xyz]), L)
    z = np.concatenate([zs, np.tile(np.array([Z_O, Z_H, Z_H], np.int32), nw)])
    box = np.diag([L, L, L]).astype(np.float32)[None]
    return System(f"solvated{len(z)}", z, pos.astype(np.float32), np.zeros(len(z), np.int32),
                  box, 1, {"L": L, "n_solute": n_solute})


def big_water_box(seed: int = 4, radii=(5.0, 6.0)) -> System:
    """32,000 rigid waters chosen at random from a 32^3 lattice in a 98.6 A
    periodic cube (96,000 atoms); the margin rule is applied at both the
    5 A cutoff and the 6 A cutoff-plus-skin."""
    return water_box(n_side=32, L=98.6, seed=seed, n_keep=32000, radii=radii)


def million_water_box(seed: int = 5) -> System:
    """343,000 rigid waters (1,029,000 atoms) on a jittered 70^3 lattice at
    the 1 g/cm^3 spacing (3.104 A) in a 217.28 A periodic cube: the stress
    case of the neighbor search; pairs are kept clear of both the 5 A cutoff
    and the 6 A cutoff-plus-skin."""
    return water_box(n_side=70, L=217.28, seed=seed, radii=(5.0, 6.0))


def maxwell_boltzmann(sys: System, T: float = 300.0, seed: int = 0) -> np.ndarray:
    """Initial velocities (A/fs) at temperature T with zero centre-of-mass
    momentum per system."""
    rng = np.random.default_rng(seed)
    m = sys.masses().astype(np.float64)
    sig = np.sqrt(KB_EV * T / m * EV_PER_AMU_A2_FS2)
    v = rng.standard_normal((sys.n_atoms, 3)) * sig[:, None]
    for s in range(sys.n_systems):
        sel = sys.batch == s
        p = (m[sel, None] * v[sel]).sum(0) / m[sel].sum()
        v[sel] -= p
    return v.astype(np.float32)


def perturb(sys: System, seed: int, scale: float = 0.02) -> System:
    """A copy with positions displaced by U(+-scale) A (used for MD-like
    repeated evaluations)."""
    rng = np.random.default_rng(seed)
    pos = (sys.pos.astype(np.float64) + rng.uniform(-scale, scale, sys.pos.shape)).astype(np.float32)
    return dataclasses.replace(sys, pos=pos)


def _lower_image_np(r: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Nearest image for a lower-triangular box with rows a, b, c (remove c,
    then b, then a; used only to validate generated geometry)."""
    r = np.array(r, dtype=np.float64, copy=True)
    for k in (2, 1, 0):
        r -= np.round(r[:, k] / B[k, k])[:, None] * B[k]
    return r


def triclinic_water(n_side: int = 10, L: float = 31.04, tilt=(0.3, 0.2, -0.25), seed: int = 5,
                    jitter: float = 0.3, radii=(5.0,), margin=1e-4) -> System:
    """Rigid waters on a jittered lattice in a triclinic cell with rows
    a = (L,0,0), b = (tb L, L, 0), c = (tc1 L, tc2 L, L) (tilt = (tb, tc1,
    tc2); the volume, and so the density, of the cube of side L): lattice
    sites at fractional coordinates (k + 1/2)/n_side, random orientations,
    and no pair within `margin` of a radius in `radii` (checked by brute
    force under the cell's nearest image)."""
    rng = np.random.default_rng(seed)
    tb, tc1, tc2 = tilt
    B = np.array([[L, 0, 0], [tb * L, L, 0], [tc1 * L, tc2 * L, L]], dtype=np.float64)
    g = (np.arange(n_side) + 0.5) / n_side
    frac = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    centres = frac @ B
    xyz = _place_waters(rng, centres, jitter)
    n = len(xyz)
    for _ in range(200):
        x = xyz.astype(np.float32).astype(np.float64)
        bad = np.zeros(n, dtype=bool)
        for a0 in range(0, n, 512):
            r = (x[a0:a0 + 512, None, :] - x[None, :, :]).reshape(-1, 3)
            d = np.linalg.norm(_lower_image_np(r, B), axis=1).reshape(-1, n)
            hit = np.zeros_like(d, dtype=bool)
            for R in radii:
                hit |= np.abs(d - R) < margin
            ia, ib = np.nonzero(hit)
            bad[ia + a0] = True
            bad[ib] = True
        if not bad.any():
            break
        mols = np.unique(np.nonzero(bad)[0] // 3)
        xyz = xyz.reshape(-1, 3, 3)
        xyz[mols] = _place_waters(rng, centres[mols], jitter).reshape(-1, 3, 3)
        xyz = xyz.reshape(-1, 3)
    else:
        raise RuntimeError("could not satisfy the pair-distance margin")
    nw = len(centres)
    z = np.tile(np.array([Z_O, Z_H, Z_H], np.int32), nw)
    return System(f"triclinic_water{3 * nw}", z, xyz.astype(np.float32), np.zeros(3 * nw, np.int32),
                  B.astype(np.float32)[None], 1, {"L": L, "tilt": tilt})


def random_walk_molecule(n: int, seed: int = 0, step: float = 1.5, min_nonbonded: float = 1.2,
                         radii=(4.5,), margin=1e-4) -> System:
    """A molecule-like cluster in vacuum: a seeded self-avoiding random walk
    of n atoms with `step` A bonds, every non-bonded distance >= min_nonbonded,
    elements H/C/N/O with probabilities .5/.3/.1/.1, and no pair distance
    within `margin` of a radius in `radii` (the stand-in for the paper's
    single molecules of the same atom counts)."""
    rng = np.random.default_rng(seed)
    cell = max(min_nonbonded, 1.0)
    grid: dict[tuple[int, int, int], list[int]] = {}
    walk = np.zeros((n, 3))

    def key(p):
        return tuple(np.floor(p / cell).astype(int).tolist())

    def ok(p, prev):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for idx in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if idx != prev and np.sum((walk[idx] - p) ** 2) < min_nonbonded ** 2:
                            return False
        return True

    grid.setdefault(key(walk[0]), []).append(0)
    k = 1
    while k < n:
        for _ in range(200):
            d = rng.standard_normal(3)
            p = walk[k - 1] + step * d / np.linalg.norm(d)
            if ok(p, k - 1):
                break
        else:
            raise RuntimeError("random walk stuck")
        walk[k] = p
        grid.setdefault(key(p), []).append(k)
        k += 1
    for _ in range(100):
        bad = _near_radius_atoms(walk.astype(np.float32).astype(np.float64), None, radii, margin)
        if bad.size == 0:
            break
        walk[bad] += rng.uniform(-1e-3, 1e-3, (len(bad), 3))
    else:
        raise RuntimeError("could not satisfy the pair-distance margin")
    z = rng.choice(np.array([Z_H, Z_C, Z_N, Z_O], np.int32), n, p=[0.5, 0.3, 0.1, 0.1])
    return System(f"walk{n}", z, walk.astype(np.float32), np.zeros(n, np.int32), None, 1)


def workload(name: str) -> System:
    """The five named workloads:
    molecule32  - 32-atom molecule in vacuum
    water3000   - 1,000 waters, periodic 31.04 A cube
    batch512    - 512 molecules of 8..96 atoms in vacuum
    solvated24k - ~24,000-atom periodic solvated box, 62 A cube
    water96k    - 32,000 waters (96,000 atoms), periodic 98.6 A cube
    """
    if name == "molecule32":
        return small_molecule(0)
    if name == "water3000":
        return water_box(10, 31.04, seed=1)
    if name == "batch512":
        return molecule_batch(512, seed=2)
    if name == "solvated24k":
        return solvated_box(seed=3)
    if name == "water96k":
        return big_water_box(seed=4)
    raise KeyError(name)


WORKLOADS = ("molecule32", "water3000", "batch512", "solvated24k", "water96k")
