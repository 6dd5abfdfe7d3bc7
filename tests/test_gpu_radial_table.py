"""GPU checks of the tabulated radial functions (radial_table = n > 0): the
interpolated model against the FP64 oracle of the exact model, at the
standard tolerances for n = 4096; the interpolation error shrinks as n grows;
forces are the exact derivatives of the interpolated energy; the tables follow
the weights; weight gradients are refused."""
import functools

import numpy as np
import pytest
import torch

from oracle.neighbors import neighbor_pairs
from paper_2402_17660_gb300 import _lib, synth
from paper_2402_17660_gb300.tnet import TensorNet

from .gpu_helpers import (DEV, E_TOL, F_TOL, RC, energy_errors, force_error, gpu_energy_forces, gpu_pairs,
                          margin_ok, oracle_energy_forces, to_dev)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

SHAPE = synth.ModelShape()
W = synth.init_weights(SHAPE, seed=0)
NT = 4096
BF16_TOL = 1e-2


def _model(sys, n=NT, shape=SHAPE, weights=W, precision=0, **kw):
    i, _ = neighbor_pairs(sys.pos, sys.batch, sys.box, RC)
    return TensorNet(weights, F=shape.F, K=shape.K, L=shape.L, max_z=shape.max_z, cutoff_upper=shape.cutoff_upper,
                     max_atoms=sys.n_atoms, max_systems=sys.n_systems, max_pairs=int(len(i) * 1.25) + 64,
                     precision=precision, device=DEV, radial_table=n, **kw)


@functools.lru_cache(maxsize=None)
def _oracle(name):
    s = synth.workload(name)
    return oracle_energy_forces(W, s)


def _errors(sys, m, ref=None, shape=SHAPE, weights=W):
    E, F = gpu_energy_forces(m, sys)
    Es, Ei, Fo = ref if ref is not None else oracle_energy_forces(weights, sys, shape)
    return energy_errors(E, Es, Ei, sys.batch).max(), force_error(F, Fo)


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("name", ["molecule32", "water3000"])
def test_table_matches_oracle(name, precision):
    s = synth.workload(name)
    e, f = _errors(s, _model(s, precision=precision), _oracle(name))
    print(f"{name} table n={NT} precision {precision}: rel energy err {e:.2e}, rel RMS force err {f:.2e}")
    assert e <= E_TOL and f <= F_TOL


def test_table_bf16_mode():
    s = synth.workload("water3000")
    e, f = _errors(s, _model(s, precision=1), _oracle("water3000"))
    print(f"water3000 table BF16: rel energy err {e:.2e}, rel RMS force err {f:.2e}")
    assert e <= BF16_TOL and f <= BF16_TOL


def _small_box():
    for seed in range(300, 340):
        c = synth.random_cluster(30, seed=seed, side=10.5, min_dist=1.2)
        c.box = (np.eye(3) * 10.5)[None].astype(np.float32)
        if margin_ok(c):
            return c
    raise RuntimeError


@pytest.mark.parametrize("case", ["small_box", "batch", "triclinic", "sparse"])
def test_table_cases(case):
    if case == "small_box":
        s = _small_box()
    elif case == "batch":
        s = synth.molecule_batch(24, seed=3)
    elif case == "triclinic":
        s = synth.triclinic_water(10, 31.04, seed=5)
    else:   # an isolated atom and a pair close to the cutoff
        s = synth.System("sparse", np.array([1, 6, 8, 7], np.int32),
                         np.array([[0, 0, 0], [20, 0, 0], [20, 4.9, 0], [0, 0, 30]], np.float32),
                         np.zeros(4, np.int32), None, 1)
    e, f = _errors(s, _model(s))
    print(f"{case}: rel energy err {e:.2e}, rel RMS force err {f:.2e}")
    assert e <= E_TOL and f <= F_TOL


@pytest.mark.parametrize("L", [0, 1, 3])
def test_table_layer_counts(L):
    shape = synth.ModelShape(L=L)
    w = synth.init_weights(shape, seed=4)
    s = synth.workload("molecule32")
    e, f = _errors(s, _model(s, shape=shape, weights=w), shape=shape, weights=w)
    print(f"L={L}: rel energy err {e:.2e}, rel RMS force err {f:.2e}")
    assert e <= E_TOL and f <= F_TOL


def test_table_resolution():
    """Cubic Hermite error falls as h^4 (values) and h^3 (derivatives)."""
    s = synth.workload("water3000")
    ref = _oracle("water3000")
    errs = {n: _errors(s, _model(s, n=n), ref) for n in (256, 1024, 4096)}
    for n, (e, f) in errs.items():
        print(f"n={n}: rel energy err {e:.2e}, rel RMS force err {f:.2e}")
    assert errs[256][1] <= BF16_TOL
    assert errs[4096][1] <= errs[256][1] and errs[4096][1] <= F_TOL


def test_table_forces_are_derivatives_of_interpolated_energy():
    """A coarse table (n = 256, interpolation error well above FP32 rounding):
    a central difference of its energy along the force field equals -sum F.dx."""
    s = synth.workload("water3000")
    m = _model(s, n=256)
    E0, F0 = gpu_energy_forces(m, s)
    v = F0.astype(np.float64) / np.sqrt(np.mean(np.sum(F0.astype(np.float64) ** 2, 1)))
    h = 1e-3
    sp = synth.System(s.name, s.z, (s.pos + h * v).astype(np.float32), s.batch, s.box, 1)
    sm = synth.System(s.name, s.z, (s.pos - h * v).astype(np.float32), s.batch, s.box, 1)
    dp = sp.pos.astype(np.float64) - sm.pos.astype(np.float64)
    Ep, _ = gpu_energy_forces(m, sp)
    Em, _ = gpu_energy_forces(m, sm)
    fd = Ep[0] - Em[0]
    an = -np.sum(F0.astype(np.float64) * dp)
    print(f"table n=256: FD {fd:.6e} analytic {an:.6e} rel {abs(fd - an) / abs(an):.2e}")
    assert abs(fd - an) <= 1e-3 * abs(an)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_table_recompute_bitwise_equal(precision):
    s = synth.workload("water3000")
    out = []
    for rec in (False, True):
        m = _model(s, precision=precision, recompute_edges=rec)
        out.append(gpu_energy_forces(m, s))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_table_follows_weights():
    s = synth.workload("molecule32")
    m = _model(s)
    w2 = synth.init_weights(SHAPE, seed=9)
    m.set_weights(w2)
    e, f = _errors(s, m, weights=w2)
    assert e <= E_TOL and f <= F_TOL


def test_table_weight_gradients_unsupported():
    s = synth.workload("molecule32")
    m = _model(s)
    z, pos, batch, box = to_dev(s)
    nl = gpu_pairs(m, s)
    with pytest.raises(_lib.TnetError) as ex:
        m.energy_forces(z, pos, nl, None, box, 1, forces=True, grad_weights=True)
    assert ex.value.code == 9


def test_table_md_matches_exact_model():
    """Ten MD steps with the tables against ten with the exact radial functions
    from the same state: the trajectories agree to the interpolation error."""
    wm = synth.md_weights(SHAPE, seed=0)
    s = synth.workload("water3000")
    z, pos, _, box = to_dev(s)
    vel = torch.from_numpy(synth.maxwell_boltzmann(s, 300.0, seed=1)).to(DEV)
    inv_m = torch.from_numpy(1.0 / s.masses()).to(DEV)
    res = []
    for n in (0, NT):
        m = TensorNet(wm, max_atoms=s.n_atoms, max_pairs=300000, device=DEV, radial_table=n)
        p, v = pos.clone(), vel.clone()
        m.reset_status()
        ek, ep = m.md(z, inv_m, p, v, box, 0.5, 1.0, 10, 10)
        torch.cuda.synchronize()
        m.check_status("md")
        res.append((p.cpu().numpy(), ep.cpu().numpy()))
    dx = np.abs(res[0][0] - res[1][0]).max()
    de = np.abs(res[0][1] - res[1][1]).max() / np.abs(res[0][1]).max()
    print(f"table MD vs exact after 10 steps: max |dx| {dx:.2e} A, max rel dE_pot {de:.2e}")
    assert dx <= 1e-4 and de <= 1e-5
