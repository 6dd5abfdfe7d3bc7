"""GPU parity of tnet_energy_forces against the FP64 oracle: energies within
1e-5 relative (|dE_s| <= 1e-5 max(|E_s|, sum_i |E_i|)) and forces within
1e-4 of the RMS force, on seeded inputs; at full size, the invariances the
model fixes and a finite-difference check of the forces."""
import numpy as np
import pytest
import torch

from oracle.neighbors import neighbor_pairs
from paper_2402_17660_gb300 import synth
from paper_2402_17660_gb300.tnet import EnergyFn, NeighborList, TensorNet

from .gpu_helpers import (BF16_F_MAX_TOL, BF16_F_TOL, DEV, E_TOL, F_MAX_TOL, F_TOL, RC, energy_errors,
                          force_error, force_errors, gpu_energy_forces, gpu_pairs, make_model, margin_ok,
                          oracle_energy_forces, to_dev)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

SHAPE = synth.ModelShape()
W = synth.init_weights(SHAPE, seed=0)


def _compare(sys, shape=SHAPE, weights=W, seed=None):
    m = make_model(weights, sys, shape=shape)
    E, F = gpu_energy_forces(m, sys, seed=seed)
    Es, Ei, Fo = oracle_energy_forces(weights, sys, shape, seed=seed)
    e_err = energy_errors(E, Es, Ei, sys.batch)
    f_err, f_max = force_errors(F, Fo)
    print(f"{sys.name}: N={sys.n_atoms} max rel energy err {e_err.max():.2e}, rel RMS force err {f_err:.2e}, "
          f"worst atom {f_max:.2e}")
    assert np.all(e_err <= E_TOL), e_err
    assert f_err <= F_TOL and f_max <= F_MAX_TOL, (f_err, f_max)
    return m, E, F


def _cluster(n, seed0=200):
    for s in range(seed0, seed0 + 50):
        c = synth.random_cluster(n, seed=s, side=None if n > 3 else 4.0)
        if margin_ok(c):
            return c
    raise RuntimeError


@pytest.mark.parametrize("n", [2, 3, 8, 64])
def test_small_clusters(n):
    _compare(_cluster(n))


def test_isolated_atom_and_far_pair():
    s = synth.System("sparse", np.array([1, 6, 8, 7], np.int32),
                     np.array([[0, 0, 0], [20, 0, 0], [20, 4.2, 0], [0, 0, 30]], np.float32),
                     np.zeros(4, np.int32), None, 1)
    _compare(s)


def test_periodic_small_box():
    for seed in range(300, 340):
        c = synth.random_cluster(30, seed=seed, side=10.5, min_dist=1.2)
        c.box = (np.eye(3) * 10.5)[None].astype(np.float32)
        if margin_ok(c):
            break
    _compare(c)


def test_molecule32():
    _compare(synth.workload("molecule32"))


def test_batch_of_molecules_uneven_sizes():
    s = synth.molecule_batch(48, seed=2)
    _compare(s)


def test_energy_seed_weights_forces():
    s = synth.molecule_batch(5, nmin=8, nmax=30, seed=9)
    seed = np.array([0.5, -1.0, 2.0, 0.0, 1.5])
    _compare(s, seed=seed)


@pytest.mark.parametrize("L", [0, 1, 3])
def test_other_layer_counts(L):
    shape = synth.ModelShape(L=L)
    _compare(_cluster(40, 400), shape=shape, weights=synth.init_weights(shape, seed=1))


def test_water3000():
    _compare(synth.workload("water3000"))


@pytest.mark.parametrize("L", [0, 1, 2])
def test_paper_shape_molecule_cutoff_4_5(L):
    """The shapes of the paper's single-molecule table: cutoff 4.5 A, 0, 1 or
    2 interaction layers, on a 166-atom random-walk molecule."""
    shape = synth.ModelShape(L=L, cutoff_upper=4.5)
    Wl = synth.init_weights(shape, seed=0)
    s = synth.random_walk_molecule(166, seed=166)
    m = make_model(Wl, s, shape=shape, cutoff=4.5)
    E, F = gpu_energy_forces(m, s, cutoff=4.5)
    Es, Ei, Fo = oracle_energy_forces(Wl, s, shape)
    e_err, (f_err, f_max) = energy_errors(E, Es, Ei, s.batch), force_errors(F, Fo)
    print(f"walk166 L={L}: rel energy err {e_err.max():.2e}, rel RMS force err {f_err:.2e}, worst atom {f_max:.2e}")
    assert np.all(e_err <= E_TOL) and f_err <= F_TOL and f_max <= F_MAX_TOL


def test_triclinic_water():
    _compare(synth.triclinic_water(6, 18.6, seed=5))


def test_cube_and_equivalent_tilted_cell_agree():
    """Same lattice, other basis: the pair vectors differ only by rounding."""
    s = synth.workload("water3000")
    L = 31.04
    t = synth.System(s.name, s.z, s.pos, s.batch, np.array([[[L, 0, 0], [L, L, 0], [0, L, L]]], np.float32), 1)
    m = make_model(W, s)
    E0, F0 = gpu_energy_forces(m, s)
    E1, F1 = gpu_energy_forces(m, t)
    assert abs(E1[0] - E0[0]) <= 1e-6 * abs(E0[0])
    assert force_error(F1, F0) <= 1e-5


def test_skin_list_gives_identical_results():
    s = synth.water_box(10, 31.04, seed=1, radii=(5.0, 6.0))
    m = make_model(W, s, max_pairs=400000)
    E1, F1 = gpu_energy_forces(m, s, nl=gpu_pairs(m, s, cutoff=5.0))
    E2, F2 = gpu_energy_forces(m, s, nl=gpu_pairs(m, s, cutoff=6.0))
    assert np.array_equal(E1, E2) and np.array_equal(F1, F2)


def test_deterministic():
    s = synth.workload("water3000")
    m = make_model(W, s)
    nl = gpu_pairs(m, s)
    E1, F1 = gpu_energy_forces(m, s, nl=nl)
    E2, F2 = gpu_energy_forces(m, s, nl=nl)
    assert np.array_equal(E1, E2) and np.array_equal(F1, F2)


def test_bad_atomic_number_flagged():
    s = _cluster(8)
    s.z[3] = 120
    m = make_model(W, s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    m.reset_status()
    m.energy_forces(z, pos, nl)
    torch.cuda.synchronize()
    assert int(m.status.item()) == 8


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_recompute_edges_bitwise_equal(precision):
    """Keeping the radial-MLP activations and recomputing them in the reverse
    pass run the same kernels on the same inputs: identical results."""
    s = synth.workload("water3000")
    z, pos, batch, box = to_dev(s)
    out = []
    for rec in (False, True):
        m = TensorNet(W, max_atoms=s.n_atoms, max_pairs=200000, precision=precision, device=DEV,
                      recompute_edges=rec)
        nl = gpu_pairs(m, s)
        m.reset_status()
        E, F, G = m.energy_forces(z, pos, nl, None, box, 1, forces=True, grad_weights=True)
        torch.cuda.synchronize()
        m.check_status("recompute_edges")
        out.append((E.cpu().numpy(), F.cpu().numpy(), G.cpu().numpy()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_unsorted_row_rejected():
    """Rows must ascend strictly (the reverse-edge search and the upper-edge
    split rely on it); a swapped pair of columns is reported as ARG."""
    s = _cluster(16)
    m = make_model(W, s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    rp, col = nl.row_ptr.cpu().numpy(), nl.col.cpu().numpy().copy()
    i = int(np.argmax(np.diff(rp)))
    assert rp[i + 1] - rp[i] >= 2
    a = rp[i]
    col[a], col[a + 1] = col[a + 1], col[a]
    bad = NeighborList(nl.row_ptr, torch.from_numpy(col).to(DEV), nl.n_pairs, nl.cutoff)
    m.reset_status()
    m.energy_forces(z, pos, bad)
    torch.cuda.synchronize()
    assert int(m.status.item()) == 1


def test_autograd_function_positions():
    s = _cluster(16, 500)
    m = make_model(W, s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    p = pos.clone().requires_grad_(True)
    E = EnergyFn.apply(p, m.weights, m, z, nl, None, None, 1)
    (3.0 * E.sum()).backward()
    _, Fo = gpu_energy_forces(m, s, nl=nl)
    assert torch.allclose(p.grad.cpu(), torch.from_numpy(-3.0 * Fo), rtol=0, atol=1e-6)


# ------------------------------------------------------------ full size ---
def _axis_permuted(sys, perm):
    s = synth.System(sys.name + "perm", sys.z.copy(), np.ascontiguousarray(sys.pos[:, perm]), sys.batch.copy(),
                     None if sys.box is None else sys.box.copy(), sys.n_systems)
    return s


@pytest.mark.parametrize("name", ["solvated24k", "water96k"])
def test_full_size_invariances(name):
    s = synth.workload(name)
    m = make_model(W, s, max_pairs=70 * s.n_atoms)
    E0, F0 = gpu_energy_forces(m, s)
    rmsF = np.sqrt(np.mean(np.sum(F0 ** 2, 1)))
    # net force vanishes (E depends only on pair vectors)
    assert np.linalg.norm(F0.astype(np.float64).sum(0)) <= 1e-5 * rmsF * s.n_atoms
    # cubic box: permuting the axes is a symmetry (E invariant, F permuted)
    perm = [1, 2, 0]
    E1, F1 = gpu_energy_forces(m, _axis_permuted(s, perm))
    scale = np.abs(E0).max()
    assert abs(E1[0] - E0[0]) <= 1e-5 * max(scale, 1.0)
    assert force_error(F1, F0[:, perm]) <= F_TOL
    # lattice shifts of a third of the atoms leave everything unchanged
    sh = synth.System(s.name, s.z, s.pos.copy(), s.batch, s.box, 1)
    L = float(s.box[0, 0, 0])
    sh.pos[::3] += np.array([L, -L, 2 * L], np.float32)
    E2, F2 = gpu_energy_forces(m, sh)
    assert abs(E2[0] - E0[0]) <= 1e-5 * max(scale, 1.0)
    assert force_error(F2, F0) <= F_TOL


@pytest.mark.parametrize("name", ["water3000", "solvated24k"])
def test_full_size_directional_finite_difference(name):
    """Central difference of the GPU energy (reduced in FP64) along the force
    field itself, E(x + h v) - E(x - h v), against -sum F . dx."""
    s = synth.workload(name)
    m = make_model(W, s, max_pairs=100 * s.n_atoms)
    E0, F0 = gpu_energy_forces(m, s)
    v = F0.astype(np.float64) / np.sqrt(np.mean(np.sum(F0.astype(np.float64) ** 2, 1)))
    h = 1e-3
    sp = synth.System(s.name, s.z, (s.pos + h * v).astype(np.float32), s.batch, s.box, 1)
    sm = synth.System(s.name, s.z, (s.pos - h * v).astype(np.float32), s.batch, s.box, 1)
    dp = (sp.pos.astype(np.float64) - sm.pos.astype(np.float64))   # the displacement actually applied
    Ep, _ = gpu_energy_forces(m, sp, nl=gpu_pairs(m, sp, cutoff=6.0))
    Em, _ = gpu_energy_forces(m, sm, nl=gpu_pairs(m, sm, cutoff=6.0))
    fd = Ep[0] - Em[0]
    an = -np.sum(F0.astype(np.float64) * dp)
    print(f"{name}: FD {fd:.6e} analytic {an:.6e} rel {abs(fd - an) / abs(an):.2e}")
    assert abs(fd - an) <= 1e-3 * abs(an)


# ---------------------------------------------------------- weight grads ---
def _compare_weight_grads(sys, shape=SHAPE, weights=W, seed=None):
    from oracle.tensornet import TensorNet as Oracle
    from paper_2402_17660_gb300.tnet import unpack_weights
    m = make_model(weights, sys, shape=shape)
    z, pos, batch, box = to_dev(sys)
    nl = gpu_pairs(m, sys)
    m.reset_status()
    sd = None if seed is None else torch.tensor(seed, dtype=torch.float32, device=DEV)
    E, F, G = m.energy_forces(z, pos, nl, batch if sys.n_systems > 1 else None, box, sys.n_systems,
                              forces=True, grad_weights=True, seed=sd)
    torch.cuda.synchronize()
    m.check_status("energy_forces(grad_weights)")
    Gg = unpack_weights(G.cpu().numpy(), shape.F, shape.K, shape.L, shape.max_z)
    o = Oracle(weights, F=shape.F, K=shape.K, L=shape.L)
    _, _, Fo, Go = o.energy_forces(sys.z, sys.pos, sys.batch, sys.box, n_systems=sys.n_systems, want_weights=True,
                                   seed=seed)
    f_err, f_max = force_errors(F.cpu().numpy(), Fo)
    assert f_err <= F_TOL and f_max <= F_MAX_TOL, (f_err, f_max)
    worst = 0.0
    for k in Go:
        ref = Go[k]
        rms = np.sqrt(np.mean(ref ** 2))
        err = np.sqrt(np.mean((Gg[k].astype(np.float64) - ref) ** 2))
        rel = err / max(rms, 1e-30)
        worst = max(worst, rel)
        assert rel <= F_TOL, (k, rel)
    print(f"{sys.name}: worst per-tensor rel RMS weight-gradient error {worst:.2e}")


def test_weight_gradients_cluster():
    _compare_weight_grads(_cluster(24, 600))


def test_weight_gradients_periodic_batch_and_seed():
    parts = [synth.random_cluster(20, seed=700 + k, side=10.5, min_dist=1.2) for k in range(3)]
    s = synth.System("pbcbatch", np.concatenate([p.z for p in parts]), np.concatenate([p.pos for p in parts]),
                     np.repeat(np.arange(3, dtype=np.int32), 20), np.tile((np.eye(3) * 10.5)[None], (3, 1, 1)).astype(np.float32), 3)
    _compare_weight_grads(s, seed=np.array([1.0, -0.5, 2.0]))


@pytest.mark.parametrize("L", [0, 1])
def test_weight_gradients_other_layer_counts(L):
    shape = synth.ModelShape(L=L)
    _compare_weight_grads(_cluster(20, 800), shape=shape, weights=synth.init_weights(shape, seed=2))


def test_weight_gradients_water3000():
    _compare_weight_grads(synth.workload("water3000"))


def test_autograd_function_weights():
    s = _cluster(16, 900)
    m = make_model(W, s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    w = m.weights.clone().requires_grad_(True)
    E = EnergyFn.apply(pos, w, m, z, nl, None, None, 1)
    (2.0 * E.sum()).backward()
    _, _, G = m.energy_forces(z, pos, nl, grad_weights=True)
    torch.cuda.synchronize()
    assert torch.allclose(w.grad, 2.0 * G, rtol=1e-5, atol=1e-7)


# --------------------------------------------------------------- BF16 mode ---
# BF16 tensor-core GEMMs: RMS force error <= 1e-2 of the RMS force (BF16_F_TOL),
# worst atom <= 1e-1 of it (BF16_F_MAX_TOL)


def _make_bf16(sys, weights=W, shape=SHAPE, max_pairs=None):
    from paper_2402_17660_gb300.tnet import TensorNet
    m32 = make_model(weights, sys, shape=shape, max_pairs=max_pairs)
    return TensorNet(weights, F=shape.F, K=shape.K, L=shape.L, max_z=shape.max_z, max_atoms=sys.n_atoms,
                     max_systems=sys.n_systems, max_pairs=m32.max_pairs, precision=1, device=DEV), m32


@pytest.mark.parametrize("name", ["molecule32", "water3000"])
def test_bf16_mode_against_oracle(name):
    s = synth.workload(name)
    mb, m32 = _make_bf16(s)
    Eb, Fb = gpu_energy_forces(mb, s)
    E32, F32 = gpu_energy_forces(m32, s)
    Es, Ei, Fo = oracle_energy_forces(W, s)
    e_err = energy_errors(Eb, Es, Ei, s.batch).max()
    f_err, f_max = force_errors(Fb, Fo)
    f_err32 = force_error(Fb, F32)
    print(f"{name} BF16: rel energy err {e_err:.2e}, rel RMS force err vs oracle {f_err:.2e} (worst atom "
          f"{f_max:.2e}), vs FP32 {f_err32:.2e}")
    assert f_err <= BF16_F_TOL and f_err32 <= BF16_F_TOL and f_max <= BF16_F_MAX_TOL
    assert e_err <= 1e-2


def test_bf16_mode_batch_and_weight_grads():
    from paper_2402_17660_gb300.tnet import unpack_weights
    s = synth.molecule_batch(40, seed=3)
    mb, m32 = _make_bf16(s)
    Eb, Fb = gpu_energy_forces(mb, s)
    E32, F32 = gpu_energy_forces(m32, s)
    assert force_error(Fb, F32) <= BF16_F_TOL
    z, pos, batch, box = to_dev(s)
    outs = []
    for m in (mb, m32):
        nl = gpu_pairs(m, s)
        m.reset_status()
        _, _, G = m.energy_forces(z, pos, nl, batch, box, s.n_systems, grad_weights=True)
        torch.cuda.synchronize()
        m.check_status("bf16 grads")
        outs.append(unpack_weights(G.cpu().numpy(), 128, 32, 2, 100))
    worst = max(np.sqrt(np.mean((outs[0][k] - outs[1][k]) ** 2)) / max(np.sqrt(np.mean(outs[1][k] ** 2)), 1e-30)
                for k in outs[1])
    print(f"BF16 vs FP32 worst per-tensor weight-gradient rel RMS diff {worst:.2e}")
    assert worst <= 5e-2


def test_autotuner_knobs_change_speed_not_results(tmp_path):
    from paper_2402_17660_gb300.tnet import autotune, tuning_knobs
    s = synth.workload("water3000")
    for prec in (0, 1):
        from paper_2402_17660_gb300.tnet import TensorNet
        m = TensorNet(W, max_atoms=s.n_atoms, max_systems=1, max_pairs=250000, precision=prec, device=DEV)
        z, pos, batch, box = to_dev(s)
        nl = gpu_pairs(m, s)
        E0, F0 = gpu_energy_forces(m, s, nl=nl)
        knobs, timings = autotune(m, z, pos, nl, None, box, 1, reps=1, cache=str(tmp_path / "t.json"))
        assert len(timings) == len(tuning_knobs())
        # every candidate of every knob gives the same result within rounding
        for k, (name, cands) in enumerate(tuning_knobs()):
            for v in cands:
                trial = list(knobs)
                trial[k] = v
                m.set_tuning(trial)
                E1, F1 = gpu_energy_forces(m, s, nl=nl)
                assert abs(E1[0] - E0[0]) <= 1e-6 * abs(E0[0]), (prec, name, v)
                assert force_error(F1, F0) <= 1e-5, (prec, name, v, force_error(F1, F0))
        # the cache is read back
        knobs2, _ = autotune(m, z, pos, nl, None, box, 1, cache=str(tmp_path / "t.json"))
        assert knobs2 == knobs



# -------------------------------------------------------- 3xTF32 mode ---
def _make_x3(sys, weights=W, shape=SHAPE):
    from paper_2402_17660_gb300.tnet import TensorNet
    m32 = make_model(weights, sys, shape=shape)
    return TensorNet(weights, F=shape.F, K=shape.K, L=shape.L, max_z=shape.max_z, max_atoms=sys.n_atoms,
                     max_systems=sys.n_systems, max_pairs=m32.max_pairs, precision=2, device=DEV)


@pytest.mark.parametrize("name", ["molecule32", "water3000"])
def test_tf32x3_mode_meets_fp32_tolerances(name):
    s = synth.workload(name)
    m = _make_x3(s)
    E, F = gpu_energy_forces(m, s)
    Es, Ei, Fo = oracle_energy_forces(W, s)
    e_err = energy_errors(E, Es, Ei, s.batch).max()
    f_err, f_max = force_errors(F, Fo)
    print(f"{name} 3xTF32: rel energy err {e_err:.2e}, rel RMS force err {f_err:.2e}, worst atom {f_max:.2e}")
    assert e_err <= E_TOL and f_err <= F_TOL and f_max <= F_MAX_TOL


def test_tf32x3_mode_batch_and_weight_grads():
    from oracle.tensornet import TensorNet as Oracle
    from paper_2402_17660_gb300.tnet import unpack_weights
    s = synth.molecule_batch(24, seed=6)
    m = _make_x3(s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    m.reset_status()
    E, Fg, G = m.energy_forces(z, pos, nl, batch, box, s.n_systems, grad_weights=True)
    torch.cuda.synchronize()
    m.check_status("3xtf32")
    Es, Ei, Fo, Go = Oracle(W).energy_forces(s.z, s.pos, s.batch, None, n_systems=s.n_systems, want_weights=True)
    assert np.all(energy_errors(E.cpu().numpy(), Es, Ei, s.batch) <= E_TOL)
    f_err, f_max = force_errors(Fg.cpu().numpy(), Fo)
    assert f_err <= F_TOL and f_max <= F_MAX_TOL, (f_err, f_max)
    Gg = unpack_weights(G.cpu().numpy(), 128, 32, 2, 100)
    for k in Go:
        rms = np.sqrt(np.mean(Go[k] ** 2))
        assert np.sqrt(np.mean((Gg[k] - Go[k]) ** 2)) <= F_TOL * max(rms, 1e-30), k
