"""Degenerate and ragged inputs of the energy-and-force path against the
FP64 oracle (Sec. 2: per-sample energies as sums over the sample's atoms,
forces as their negative gradient): one atom, a batch in which no pair is
within the cutoff (every per-pair kernel and GEMM then runs on zero
device-side rows), batches with empty systems, whose energy is an empty sum
(exactly 0), and a periodic batch of unlike boxes; and the whole step
captured in a CUDA graph against eager calls, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2402_17660_gb300 import synth
from paper_2402_17660_gb300.tnet import TensorNet

from .gpu_helpers import (DEV, E_TOL, F_MAX_TOL, F_TOL, force_errors, gpu_energy_forces, margin_ok,
                          oracle_energy_forces)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

SHAPE = synth.ModelShape()
W = synth.init_weights(SHAPE, seed=0)
PRECISIONS = [0, 2, 1]


def _model(sys, precision):
    return TensorNet(W, F=SHAPE.F, K=SHAPE.K, L=SHAPE.L, max_z=SHAPE.max_z, max_atoms=sys.n_atoms,
                     max_systems=sys.n_systems, max_pairs=64 + 40 * sys.n_atoms, precision=precision, device=DEV)


def _system(name, z, pos, batch, n_systems):
    return synth.System(name, np.asarray(z, np.int32), np.asarray(pos, np.float32),
                        np.asarray(batch, np.int32), None, n_systems)


def _check(sys, precision, zero_forces=False):
    m = _model(sys, precision)
    E, F = gpu_energy_forces(m, sys)
    Es, Ei, Fo = oracle_energy_forces(W, sys, SHAPE)
    counts = np.bincount(sys.batch, minlength=sys.n_systems)
    empty = counts == 0
    # an empty system's energy is an empty sum: exactly zero on both sides
    assert np.all(E[empty] == 0.0) and np.all(Es[empty] == 0.0)
    tol = E_TOL if precision != 1 else 1e-2
    scale = np.maximum(np.abs(Es), np.bincount(sys.batch, weights=np.abs(Ei), minlength=sys.n_systems))
    err = np.abs(E[~empty] - Es[~empty]) / scale[~empty]
    assert np.all(err <= tol), (precision, err)
    if zero_forces:
        assert np.all(F == 0.0) and np.all(Fo == 0.0)
    else:
        f_err, f_max = force_errors(F, Fo)
        f_tol, fm_tol = (F_TOL, F_MAX_TOL) if precision != 1 else (1e-2, 1e-1)
        assert f_err <= f_tol and f_max <= fm_tol, (precision, f_err, f_max)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_atom(precision):
    _check(_system("one_atom", [6], [[0.3, -0.2, 1.0]], [0], 1), precision, zero_forces=True)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch_without_any_pair(precision):
    """Three systems of isolated atoms, every distance above the 5 A cutoff."""
    z = [1, 6, 8, 7, 1]
    pos = [[0, 0, 0], [6.0, 0, 0], [0, 0, 0], [0, 7.5, 0], [0, 0, 0]]
    _check(_system("no_pairs", z, pos, [0, 0, 1, 1, 2], 3), precision, zero_forces=True)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch_with_empty_systems(precision):
    """Systems 0, 2, 3 and 5 of six hold no atom (at both ends of the range
    and in the middle): their energies are exactly zero, and the molecules of
    systems 1 and 4 match the oracle."""
    a = synth.random_cluster(20, seed=41)
    b = synth.random_cluster(14, seed=42)
    z = np.concatenate([a.z, b.z])
    pos = np.concatenate([a.pos, b.pos + np.float32(50.0)])
    batch = np.concatenate([np.full(20, 1), np.full(14, 4)])
    _check(_system("empty_systems", z, pos, batch, 6), precision)


def _unlike_boxes():
    """Two periodic systems in one batch with unlike cells: a rectangular
    10.5 x 11 x 12 A box and a strongly tilted triclinic one (perpendicular
    widths 10.35, 10.75 and 11.5 A, all above two cutoffs)."""
    boxes = np.array([np.diag([10.5, 11.0, 12.0]), [[11.0, 0, 0], [3.0, 11.0, 0], [2.0, -2.5, 11.5]]], np.float32)
    p0 = synth.random_cluster(30, seed=100, side=10.0, min_dist=1.2)
    p1 = synth.random_cluster(24, seed=1100, side=10.0, min_dist=1.2)
    s = synth.System("unlike_boxes", np.concatenate([p0.z, p1.z]), np.concatenate([p0.pos, p1.pos]),
                     np.concatenate([np.zeros(30, np.int32), np.ones(24, np.int32)]), boxes, 2)
    assert margin_ok(s)
    return s


@pytest.mark.parametrize("precision", PRECISIONS)
def test_periodic_batch_of_unlike_boxes(precision):
    """A ragged periodic batch (Sec. 2.5.1: rectangular and triclinic boxes,
    one cell list per system): energies and forces against the oracle."""
    _check(_unlike_boxes(), precision)


@pytest.mark.parametrize("precision", [0, 2])
def test_whole_step_graph_replay_equals_eager(precision):
    """The whole step (neighbor search, energy and forces) captured once in a
    CUDA graph and replayed on positions updated in place gives bit for bit
    what eager calls give on the same positions (the path is deterministic:
    sorted rows, no atomics in the sums)."""
    s = synth.workload("water3000")
    N = s.n_atoms
    m = TensorNet(W, F=SHAPE.F, K=SHAPE.K, L=SHAPE.L, max_z=SHAPE.max_z, max_atoms=N, max_systems=1,
                  max_pairs=250000, precision=precision, device=DEV)
    z = torch.from_numpy(s.z).to(DEV)
    pos = torch.from_numpy(s.pos).to(DEV)
    box = torch.from_numpy(s.box).to(DEV)
    m.reset_status()
    nl = m.neighbors(pos, None, box, 1)
    E = torch.empty(1, dtype=torch.float64, device=DEV)
    F = torch.empty((N, 3), dtype=torch.float32, device=DEV)

    def step():
        m.neighbors(pos, None, box, 1, out=nl)
        m.energy_forces(z, pos, nl, None, box, 1, out=(E, F, None))

    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream(DEV).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    gen = torch.Generator(device="cpu").manual_seed(11)
    for _ in range(3):
        pos.add_((torch.rand(pos.shape, generator=gen) - 0.5).to(DEV) * 0.02)
        g.replay()
        torch.cuda.synchronize()
        Eg, Fg = E.clone(), F.clone()
        m.check_status("graph replay")
        nl2 = m.neighbors(pos, None, box, 1)
        E2, F2, _ = m.energy_forces(z, pos, nl2, None, box, 1)
        torch.cuda.synchronize()
        assert torch.equal(Eg, E2) and torch.equal(Fg, F2)
