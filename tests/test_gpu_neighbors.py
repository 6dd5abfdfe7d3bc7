"""GPU parity of tnet_neighbors against the oracle's brute-force pairs: the
pair set must match exactly (rows sorted, columns ascending), plus the
device-side error paths (capacity, box, NaN)."""
import numpy as np
import pytest
import torch

from oracle.neighbors import neighbor_pairs, neighbor_rows
from paper_2402_17660_gb300 import synth

from .gpu_helpers import RC, csr_to_pairs, gpu_energy_forces, gpu_pairs, make_model, margin_ok, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

W = synth.init_weights(synth.ModelShape(), seed=0)


def _check_exact(sys, cutoff=RC, cap=None):
    m = make_model(W, sys, max_pairs=None, cutoff=cutoff)
    nl = gpu_pairs(m, sys, cutoff=cutoff, cap=cap)
    assert int(m.status.item()) == 0
    gi, gj = csr_to_pairs(nl)
    oi, oj = neighbor_pairs(sys.pos, sys.batch, sys.box, cutoff)
    assert int(nl.n_pairs.item()) == len(oi)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    return nl


def _pbc_case(seed, n=40, L=(10.5, 11.0, 12.25)):
    rng = np.random.default_rng(seed)
    L = np.array(L)
    pos = rng.uniform(-0.5, 1.5, (n, 3)) * L
    pos[0] = [0.0, 0.0, 0.0]
    pos[1] = L - 1e-3
    pos[2] = [L[0], 0.5 * L[1], 0.0]
    pos[3] = [-L[0] + 0.7, -2 * L[1] + 0.3, 3 * L[2] + 0.2]
    s = synth.System(f"pbc{seed}", rng.choice([1, 6, 7, 8], n).astype(np.int32), pos.astype(np.float32),
                     np.zeros(n, np.int32), np.diag(L)[None].astype(np.float32), 1)
    return s


@pytest.mark.parametrize("n", [2, 3, 8, 64, 300])
def test_clusters_exact(n):
    seed = 0
    while True:
        s = synth.random_cluster(n, seed=100 + seed, side=None if n > 3 else 4.0)
        if margin_ok(s):
            break
        seed += 1
    _check_exact(s)


def test_pbc_edge_cases_exact():
    done = 0
    for seed in range(40):
        s = _pbc_case(seed)
        if not margin_ok(s):
            continue
        _check_exact(s)
        done += 1
        if done == 4:
            break
    assert done == 4


def test_batched_boxes_exact():
    parts = []
    for s in range(60):
        c = _pbc_case(s, n=25, L=(10.5 + 0.25 * (s % 4), 10.6, 11.0))
        if margin_ok(c):
            parts.append(c)
        if len(parts) == 3:
            break
    sys = synth.System("pbcbatch", np.concatenate([p.z for p in parts]), np.concatenate([p.pos for p in parts]),
                       np.concatenate([np.full(25, k, np.int32) for k in range(3)]),
                       np.concatenate([p.box for p in parts]), 3)
    _check_exact(sys)


@pytest.mark.parametrize("name", ["molecule32", "water3000", "batch512"])
def test_workloads_exact(name):
    _check_exact(synth.workload(name))


def test_rows_longer_than_the_row_slab_exact():
    """A dense cloud whose rows exceed the one-pass search's 128-column row
    slab at a 6 A cutoff: the search falls back to the count and fill passes
    and the pair list is still exact."""
    rng = np.random.default_rng(21)
    for _ in range(20):
        pos = rng.uniform(0.0, 12.0, (400, 3)).astype(np.float32)
        s = synth.System("dense400", rng.choice([1, 6, 7, 8], 400).astype(np.int32), pos, np.zeros(400, np.int32),
                         None, 1)
        if margin_ok(s, cutoff=6.0):
            break
    oi, _ = neighbor_pairs(s.pos, s.batch, None, 6.0)
    assert np.bincount(oi).max() > 128
    _check_exact(s, cutoff=6.0)


def test_skin_cutoff_exact():
    s = synth.water_box(10, 31.04, seed=1, radii=(5.0, 6.0))
    _check_exact(s, cutoff=6.0)


@pytest.mark.parametrize("name", ["solvated24k", "water96k"])
def test_large_sampled_rows(name):
    s = synth.workload(name)
    m = make_model(W, s, max_pairs=120 * s.n_atoms)
    nl = gpu_pairs(m, s)
    assert int(m.status.item()) == 0
    gi, gj = csr_to_pairs(nl)
    rp = nl.row_ptr.cpu().numpy()
    rows = np.random.default_rng(0).choice(s.n_atoms, 256, replace=False)
    ref = neighbor_rows(s.pos, s.batch, s.box, RC, rows)
    for a, r in zip(rows, ref):
        assert np.array_equal(gj[rp[a]:rp[a + 1]], r), a
    # whole-list properties: no self pairs, symmetric, rows ascending
    assert np.all(gi != gj)
    key = gi * s.n_atoms + gj
    assert np.all(np.diff(key) > 0)
    rkey = np.sort(gj * s.n_atoms + gi)
    assert np.array_equal(rkey, key)


def test_million_atom_water_box_sampled_rows():
    """The neighbor search's stress case, 1,029,000 atoms in a 217 A periodic
    water box, at the cutoff and at cutoff + skin: 256 sampled rows against
    the oracle's brute force over all atoms, and the whole-list properties.
    The context is built with tabulated radial functions and no interaction
    layer, so its workspace holds no per-pair radial-MLP activations."""
    from paper_2402_17660_gb300.tnet import TensorNet
    s = synth.million_water_box()
    shape = synth.ModelShape(F=64, K=8, L=0)
    m = TensorNet(synth.init_weights(shape, seed=0), F=64, K=8, L=0, max_atoms=s.n_atoms, max_systems=1,
                  max_pairs=100 * s.n_atoms, device=torch.device("cuda:0"), radial_table=256)
    rows = np.random.default_rng(3).choice(s.n_atoms, 256, replace=False)
    for cutoff in (5.0, 6.0):
        nl = gpu_pairs(m, s, cutoff=cutoff)
        assert int(m.status.item()) == 0
        n = int(nl.n_pairs.item())
        rp = nl.row_ptr.cpu().numpy().astype(np.int64)
        col = nl.col[:n].cpu().numpy().astype(np.int64)
        assert rp[-1] == n
        ref = neighbor_rows(s.pos, s.batch, s.box, cutoff, rows)
        for a, r in zip(rows, ref):
            assert np.array_equal(col[rp[a]:rp[a + 1]], r), (cutoff, a)
        gi = np.repeat(np.arange(s.n_atoms, dtype=np.int64), np.diff(rp))
        assert np.all(gi != col)
        key = gi * s.n_atoms + col
        assert np.all(np.diff(key) > 0)
        assert np.array_equal(np.sort(col * s.n_atoms + gi), key)
        print(f"water1029000 cutoff {cutoff}: {n} pairs ({n / s.n_atoms:.1f} per atom), 256 sampled rows exact")


def test_capacity_overflow_reports_needed_size():
    s = synth.workload("water3000")
    oi, oj = neighbor_pairs(s.pos, s.batch, s.box, RC)
    m = make_model(W, s, max_pairs=len(oi) + 100)
    cap = len(oi) // 2
    nl = gpu_pairs(m, s, cap=cap)
    assert int(m.status.item()) == 2
    assert int(nl.n_pairs.item()) == len(oi)
    # the row offsets are clamped to the capacity, so readers stay inside col;
    # the rows that fit are complete
    counts = np.bincount(oi, minlength=s.n_atoms)
    full = np.concatenate([[0], np.cumsum(counts)])
    rp = nl.row_ptr.cpu().numpy().astype(np.int64)
    assert np.array_equal(rp, np.minimum(full, cap))
    last = int(np.searchsorted(full, cap, side="right")) - 1      # rows [0, last) fit whole
    got_i, got_j = csr_to_pairs(nl)
    o = np.lexsort((oj, oi))
    ref_i, ref_j = oi[o], oj[o]
    keep, sel = got_i < last, ref_i < last
    assert np.array_equal(got_i[keep], ref_i[sel]) and np.array_equal(got_j[keep], ref_j[sel])


@pytest.mark.parametrize("slack", [0, -1])
def test_capacity_at_the_exact_pair_count(slack):
    """A capacity equal to the pair count holds the whole list with no error;
    one entry less overflows by one: CAPACITY, the exact count reported, the
    last row offset clamped, and every row but the last complete."""
    s = synth.workload("molecule32")
    oi, oj = neighbor_pairs(s.pos, s.batch, s.box, RC)
    n = len(oi)
    m = make_model(W, s, max_pairs=n + 100)
    nl = gpu_pairs(m, s, cap=n + slack)
    assert int(nl.n_pairs.item()) == n
    got_i, got_j = csr_to_pairs(nl)
    if slack == 0:
        assert int(m.status.item()) == 0
        assert np.array_equal(got_i, oi) and np.array_equal(got_j, oj)
        return
    assert int(m.status.item()) == 2
    rp = nl.row_ptr.cpu().numpy().astype(np.int64)
    full = np.concatenate([[0], np.cumsum(np.bincount(oi, minlength=s.n_atoms))])
    assert np.array_equal(rp, np.minimum(full, n - 1))
    last_row = int(oi[-1])
    keep, sel = got_i < last_row, oi < last_row
    assert np.array_equal(got_i[keep], oi[sel]) and np.array_equal(got_j[keep], oj[sel])


def test_energy_forces_on_truncated_list_is_flagged_and_safe():
    """An overflowed (truncated) list is not symmetric: tnet_energy_forces
    flags it and treats the unmatched edges as inactive, touching nothing
    outside its buffers; the context then evaluates a full list correctly."""
    s = synth.workload("molecule32")
    oi, _ = neighbor_pairs(s.pos, s.batch, s.box, RC)
    m = make_model(W, s, max_pairs=len(oi) + 100)
    nl = gpu_pairs(m, s, cap=len(oi) // 2)
    assert int(m.status.item()) == 2
    z, pos, batch, box = to_dev(s)
    m.reset_status()
    m.energy_forces(z, pos, nl)
    torch.cuda.synchronize()
    assert int(m.status.item()) != 0
    E, F = gpu_energy_forces(m, s)
    assert np.isfinite(E).all() and np.isfinite(F).all()


def test_box_too_small_and_nan_flagged():
    s = synth.random_cluster(20, seed=1)
    s.box = (np.eye(3) * 9.0)[None].astype(np.float32)
    m = make_model(W, s, max_pairs=1000)
    gpu_pairs(m, s)
    assert int(m.status.item()) == 3
    s2 = synth.random_cluster(20, seed=2)
    s2.pos[5, 1] = np.nan
    m2 = make_model(W, synth.random_cluster(20, seed=2), max_pairs=1000)
    gpu_pairs(m2, s2)
    assert int(m2.status.item()) == 4


def test_deterministic_and_graph_capturable():
    s = synth.workload("water3000")
    m = make_model(W, s)
    a = gpu_pairs(m, s)
    ga = a.col.clone()
    from .gpu_helpers import to_dev
    _, pos, _, box = to_dev(s)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        m.reset_status()
        out = m.neighbors(pos, None, box)          # warm-up on the side stream
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream):
            out = m.neighbors(pos, None, box, out=out)
    out.col.zero_()
    g.replay()
    torch.cuda.synchronize()
    n = int(a.n_pairs.item())
    assert torch.equal(out.col[:n], ga[:n])


# ---------------------------------------------------------------- triclinic
TRICLINIC_BOXES = [
    np.array([[12.0, 0, 0], [3.6, 11.5, 0], [2.4, -2.9, 12.2]]),      # reduced tilts
    np.array([[20.0, 0, 0], [14.0, 13.0, 0], [-9.0, 8.0, 13.0]]),     # not reduced, widths >= 2 rc
]


def _tri_case(seed, B, n=60):
    for s0 in range(seed, seed + 100):
        rng = np.random.default_rng(s0)
        frac = rng.uniform(-0.5, 1.5, (n, 3))
        pos = frac @ B
        s = synth.System(f"tri{s0}", rng.choice([1, 6, 7, 8], n).astype(np.int32), pos.astype(np.float32),
                         np.zeros(n, np.int32), B.astype(np.float32)[None], 1)
        if margin_ok(s):
            return s
    raise RuntimeError


@pytest.mark.parametrize("k", range(len(TRICLINIC_BOXES)))
@pytest.mark.parametrize("seed", [0, 100, 200])
def test_triclinic_pairs_exact(k, seed):
    _check_exact(_tri_case(seed, TRICLINIC_BOXES[k]))


def test_triclinic_water_pairs_exact():
    _check_exact(synth.triclinic_water(10, 31.04, seed=5))


def test_cube_and_equivalent_tilted_cell_give_same_pairs():
    """Same lattice, two bases: the cube of side L and a = (L,0,0),
    b = (L,L,0), c = (0,L,L)."""
    s = synth.workload("water3000")
    L = 31.04
    nl_a = _check_exact(s)
    t = synth.System(s.name, s.z, s.pos, s.batch, np.array([[[L, 0, 0], [L, L, 0], [0, L, L]]], np.float32), 1)
    nl_b = _check_exact(t)
    n = int(nl_a.n_pairs.item())
    assert torch.equal(nl_a.row_ptr, nl_b.row_ptr) and torch.equal(nl_a.col[:n], nl_b.col[:n])


def test_narrow_triclinic_box_flagged():
    L = 17.0   # widths L, L/sqrt(2), L/sqrt(3): the last is below 2 rc
    s = synth.random_cluster(20, seed=1)
    s.box = np.array([[[L, 0, 0], [L, L, 0], [0, L, L]]], np.float32)
    m = make_model(W, s, max_pairs=1000)
    gpu_pairs(m, s)
    assert int(m.status.item()) == 3

