"""Full-size GPU parity at the shapes of the paper's workloads and in every
precision mode the library offers (0: FP32 SIMT GEMMs, 1: BF16 tensor-core
GEMMs, 2: 3xTF32 tensor-core GEMMs, the benchmark's default):

- the ~24,000-atom solvated box and the 512-molecule batch against stored
  FP64 oracle energies and forces (tests/golden, written by
  make_oracle_refs.py, which calls only the oracle), per-system energies and
  every atom's force;
- a 64-atom cluster carved from the solvated box (the precision and
  differentiation workload): energies, forces and every weight gradient
  against the oracle, and central finite differences of the GPU energy;
- the 96,000-atom water box in the benchmark's launch configuration
  (activations recomputed in the reverse pass): invariances the model fixes
  and a directional central difference.

Tolerances (derived from the arithmetic; see the module gpu_helpers):
FP32-accurate modes |dE_s| <= 1e-5 max(|E_s|, sum |E_i|), RMS force error
<= 1e-4 and worst atom <= 2e-3 of the RMS force; BF16 mode 1e-2, 1e-2 and
1e-1."""
import os

import numpy as np
import pytest
import torch

from oracle.neighbors import minimum_image
from oracle.tensornet import TensorNet as Oracle
from paper_2402_17660_gb300 import synth
from paper_2402_17660_gb300.tnet import TensorNet, unpack_weights

from .gpu_helpers import (BF16_E_TOL, BF16_F_MAX_TOL, BF16_F_TOL, DEV, E_TOL, F_MAX_TOL, F_TOL, energy_errors,
                          force_errors, gpu_energy_forces, gpu_pairs, margin_ok, to_dev)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

SHAPE = synth.ModelShape()
W = synth.init_weights(SHAPE, seed=0)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PRECISIONS = {0: "fp32", 1: "bf16", 2: "3xtf32"}


def _tols(prec):
    return (BF16_E_TOL, BF16_F_TOL, BF16_F_MAX_TOL) if prec == 1 else (E_TOL, F_TOL, F_MAX_TOL)


def _weights_checksum(Wd):
    v = np.concatenate([np.asarray(Wd[k], np.float64).ravel() for k, _ in synth.param_spec(SHAPE)])
    return np.array([v.sum(), (v * v).sum()])


def _golden(name):
    d = np.load(os.path.join(GOLDEN, f"oracle_{name}.npz"))
    assert np.allclose(_weights_checksum(W), d["weights_checksum"], rtol=1e-13, atol=0), \
        "the weights differ from the ones the stored oracle results were computed with"
    box = d["box"] if d["box"].shape[0] else None
    s = synth.System(name, d["z"].astype(np.int32), d["pos"], d["batch"], box, int(d["n_systems"]))
    return s, d


def _model(sys, prec, max_pairs, recompute=False):
    return TensorNet(W, max_atoms=sys.n_atoms, max_systems=sys.n_systems, max_pairs=max_pairs, precision=prec,
                     device=DEV, recompute_edges=recompute)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", ["solvated24k", "batch512"])
def test_full_size_against_stored_oracle(name, prec):
    s, ref = _golden(name)
    m = _model(s, prec, 64 * s.n_atoms)
    E, F = gpu_energy_forces(m, s)
    Es, abs_ei, Fo = ref["energy"], ref["abs_ei"], ref["forces"].astype(np.float64)
    e_err = np.abs(E - Es) / np.maximum(np.abs(Es), abs_ei)
    f_err, f_max = force_errors(F, Fo)
    e_tol, f_tol, f_max_tol = _tols(prec)
    print(f"{name} {PRECISIONS[prec]}: N={s.n_atoms} systems={s.n_systems} worst rel energy err {e_err.max():.2e}, "
          f"rel RMS force err {f_err:.2e}, worst atom {f_max:.2e}")
    assert np.all(e_err <= e_tol), e_err.max()
    assert f_err <= f_tol and f_max <= f_max_tol, (f_err, f_max)


# ------------------------------------------- 64-atom cluster of the solvated box ---
def _cluster64():
    """The 64 atoms nearest (nearest image) to a solute atom near the box
    centre, unwrapped around it, without a box: a non-periodic cluster (a
    64-atom periodic box at 1 g/cm^3 would be narrower than two cutoffs)."""
    s = synth.workload("solvated24k")
    L = float(s.box[0, 0, 0])
    n_sol = 2500
    centre = np.full(3, L / 2)
    order = np.argsort(np.linalg.norm(minimum_image(s.pos[:n_sol].astype(np.float64) - centre, s.box[0]), axis=1))
    for c in order[:50]:
        r = minimum_image(s.pos.astype(np.float64) - s.pos[c].astype(np.float64), s.box[0])
        idx = np.sort(np.argsort(np.linalg.norm(r, axis=1))[:64])
        pos = (s.pos[c].astype(np.float64) + r[idx]).astype(np.float32)
        cl = synth.System("solvated24k_cluster64", s.z[idx].copy(), pos, np.zeros(64, np.int32), None, 1)
        if margin_ok(cl):
            return cl
    raise RuntimeError("no 64-atom cluster keeps its pairs away from the cutoff")


def _directional_fd(m, s, F0, v, h=1e-3):
    """E(x + h v) - E(x - h v) against -sum F . dx (dx the displacement
    actually applied after rounding to float32)."""
    sp = synth.System(s.name, s.z, (s.pos + h * v).astype(np.float32), s.batch, s.box, s.n_systems)
    sm = synth.System(s.name, s.z, (s.pos - h * v).astype(np.float32), s.batch, s.box, s.n_systems)
    dp = sp.pos.astype(np.float64) - sm.pos.astype(np.float64)
    Ep, _ = gpu_energy_forces(m, sp, nl=gpu_pairs(m, sp, cutoff=6.0))
    Em, _ = gpu_energy_forces(m, sm, nl=gpu_pairs(m, sm, cutoff=6.0))
    fd = float(np.sum(Ep - Em))
    an = -float(np.sum(F0.astype(np.float64) * dp))
    return fd, an


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cluster64_energy_forces_weight_grads_and_fd(prec):
    s = _cluster64()
    m = _model(s, prec, 64 * 63)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    m.reset_status()
    E, F, G = m.energy_forces(z, pos, nl, None, None, 1, forces=True, grad_weights=True)
    torch.cuda.synchronize()
    m.check_status("cluster64")
    E, F = E.cpu().numpy(), F.cpu().numpy()
    Gg = unpack_weights(G.cpu().numpy(), SHAPE.F, SHAPE.K, SHAPE.L, SHAPE.max_z)
    o = Oracle(W)
    Es, Ei, Fo, Go = o.energy_forces(s.z, s.pos, s.batch, None, want_weights=True)
    e_tol, f_tol, f_max_tol = _tols(prec)
    e_err = energy_errors(E, Es, Ei, s.batch).max()
    f_err, f_max = force_errors(F, Fo)
    g_tol = 5e-2 if prec == 1 else F_TOL
    worst_k, worst = "", 0.0
    for k in Go:
        rms = np.sqrt(np.mean(Go[k] ** 2))
        rel = np.sqrt(np.mean((Gg[k].astype(np.float64) - Go[k]) ** 2)) / max(rms, 1e-30)
        if rel > worst:
            worst_k, worst = k, rel
    # central differences of the GPU energy: along the forces and along a
    # seeded random field, both normalised to unit RMS displacement per atom.
    # h = 1e-3 A (truncation error ~7e-4 along the forces).  BF16 energies
    # move in steps as rounded operands cross bf16 boundaries, which a random
    # direction (whose slope is ~sqrt(N) times smaller than along the forces)
    # resolves only with a wider step: h = 1e-2 A there in BF16 mode (its
    # truncation error is smaller along that direction).
    rng = np.random.default_rng(11)
    fd_rel = []
    for v, h_fd in ((F.astype(np.float64), 1e-3), (rng.standard_normal(F.shape), 1e-2 if prec == 1 else 1e-3)):
        v = v / np.sqrt(np.mean(np.sum(v * v, 1)))
        fd, an = _directional_fd(m, s, F, v, h=h_fd)
        fd_rel.append(abs(fd - an) / abs(an))
    # and of the oracle energy along the forces (FP64, h = 1e-5 A: truncation
    # error ~h^2, rounding ~1e-16 |E| / h, both far below the bar)
    v = Fo / np.sqrt(np.mean(np.sum(Fo * Fo, 1)))
    h = 1e-5
    fdo = (o.forward(s.z, s.pos.astype(np.float64) + h * v, s.batch, None)[0][0]
           - o.forward(s.z, s.pos.astype(np.float64) - h * v, s.batch, None)[0][0])
    ano = -2 * h * float(np.sum(Fo * v))
    print(f"cluster64 {PRECISIONS[prec]}: rel energy err {e_err:.2e}, rel RMS force err {f_err:.2e}, worst atom "
          f"{f_max:.2e}, worst weight-gradient tensor {worst_k} {worst:.2e}, GPU FD rel err "
          f"{fd_rel[0]:.2e} / {fd_rel[1]:.2e}, oracle FD rel err {abs(fdo - ano) / abs(ano):.2e}")
    assert e_err <= e_tol
    assert f_err <= f_tol and f_max <= f_max_tol, (f_err, f_max)
    assert worst <= g_tol, (worst_k, worst)
    assert max(fd_rel) <= (3e-2 if prec == 1 else 1e-3), fd_rel
    assert abs(fdo - ano) <= 1e-6 * abs(ano)


# ------------------------------------------------ 96,000-atom water box ---
def _axis_permuted(s, perm):
    return synth.System(s.name + "perm", s.z.copy(), np.ascontiguousarray(s.pos[:, perm]), s.batch.copy(),
                        s.box.copy(), s.n_systems)


@pytest.mark.parametrize("recompute", [False, True], ids=["kept", "recomputed"])
@pytest.mark.parametrize("prec", [1, 2])
def test_water96k_invariances_and_fd_in_tensor_core_modes(prec, recompute):
    """In the benchmark's launch configuration (radial-MLP activations kept
    from the forward pass) and with them recomputed in the reverse pass: zero
    net force; a cyclic permutation of the axes of the cubic box permutes the
    forces and keeps the energy; lattice shifts of a third of the atoms change
    nothing; a central difference along the force field matches the forces."""
    s = synth.workload("water96k")
    m = _model(s, prec, 100 * s.n_atoms, recompute=recompute)   # room for the 6 A lists of the FD
    E0, F0 = gpu_energy_forces(m, s)
    rmsF = np.sqrt(np.mean(np.sum(F0.astype(np.float64) ** 2, 1)))
    e_inv = 1e-3 if prec == 1 else 1e-5
    f_inv = 1e-2 if prec == 1 else F_TOL
    net = np.linalg.norm(F0.astype(np.float64).sum(0))
    perm = [1, 2, 0]
    E1, F1 = gpu_energy_forces(m, _axis_permuted(s, perm))
    sh = synth.System(s.name, s.z, s.pos.copy(), s.batch, s.box, 1)
    L = float(s.box[0, 0, 0])
    sh.pos[::3] += np.array([L, -L, 2 * L], np.float32)
    E2, F2 = gpu_energy_forces(m, sh)
    v = F0.astype(np.float64) / rmsF
    fd, an = _directional_fd(m, s, F0, v)
    print(f"water96k {PRECISIONS[prec]}: net force {net / (rmsF * s.n_atoms):.2e} of N RMS F, axis-permutation dE "
          f"{abs(E1[0] - E0[0]) / abs(E0[0]):.2e}, lattice-shift dE {abs(E2[0] - E0[0]) / abs(E0[0]):.2e}, "
          f"FD rel err {abs(fd - an) / abs(an):.2e}")
    assert net <= 1e-5 * rmsF * s.n_atoms
    assert abs(E1[0] - E0[0]) <= e_inv * abs(E0[0])
    assert force_errors(F1, F0[:, perm])[0] <= f_inv
    assert abs(E2[0] - E0[0]) <= e_inv * abs(E0[0])
    assert force_errors(F2, F0)[0] <= f_inv
    assert abs(fd - an) <= (3e-2 if prec == 1 else 1e-3) * abs(an)


@pytest.mark.parametrize("prec", [1, 2])
def test_water96k_kept_and_recomputed_activations_agree_bitwise(prec):
    """Recomputing the radial-MLP activations in the reverse pass repeats the
    forward pass's arithmetic, so energies, forces and weight gradients are
    bitwise those of the run that keeps them, with and without weight
    gradients."""
    s = synth.workload("water96k")
    z, pos, _, box = to_dev(s)
    out = []
    for rec in (False, True):
        m = _model(s, prec, 75 * s.n_atoms, recompute=rec)
        nl = gpu_pairs(m, s)
        m.reset_status()
        E, F, G = m.energy_forces(z, pos, nl, None, box, 1, forces=True, grad_weights=True)
        # forces alone (in 3xTF32 layers 1-2 then store only pre-activations)
        E2, F2, _ = m.energy_forces(z, pos, nl, None, box, 1, forces=True)
        torch.cuda.synchronize()
        m.check_status("energy_forces")
        out.append((E.cpu().numpy(), F.cpu().numpy(), G.cpu().numpy(), E2.cpu().numpy(), F2.cpu().numpy()))
        del m, nl, E, F, G, E2, F2
        torch.cuda.empty_cache()
    for k in range(5):
        assert np.array_equal(out[0][k], out[1][k]), k
    # the energy does not depend on which reverse pass follows
    assert np.array_equal(out[0][0], out[0][3])
