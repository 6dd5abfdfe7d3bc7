"""The forms of the message kernels and their adjoint (the message_kernel
tuning knob) compute the same sums (TensorNet's messages, Sec. 2.1.1): one
warp per row with four channels per lane (forms 0 and 3, the adjoint at two
or three blocks per SM), or one thread per channel with one or four rows per
block (forms 1 and 4).
Every form is held to the FP64 oracle for energies, forces and every weight
gradient on a list with skin entries, and the forms agree with each other
within rounding in all three precisions."""
import numpy as np
import pytest
import torch

from oracle.tensornet import TensorNet as Oracle
from paper_2402_17660_gb300 import synth
from paper_2402_17660_gb300.tnet import TensorNet, unpack_weights

from .gpu_helpers import DEV, E_TOL, F_MAX_TOL, F_TOL, energy_errors, force_errors, gpu_pairs, margin_ok, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

SHAPE = synth.ModelShape()
W = synth.init_weights(SHAPE, seed=0)
KNOB = 6           # index of the message_kernel knob
FORMS = (0, 1, 3, 4)


def _model(sys, precision, max_pairs):
    return TensorNet(W, F=SHAPE.F, K=SHAPE.K, L=SHAPE.L, max_z=SHAPE.max_z, max_atoms=sys.n_atoms,
                     max_systems=sys.n_systems, max_pairs=max_pairs, precision=precision, device=DEV)


def _run(m, sys, nl, form, grads=True):
    knobs = m.get_tuning()
    knobs[KNOB] = form
    m.set_tuning(knobs)
    z, pos, batch, box = to_dev(sys)
    m.reset_status()
    E, F, G = m.energy_forces(z, pos, nl, batch if sys.n_systems > 1 else None, box, sys.n_systems,
                              forces=True, grad_weights=grads)
    torch.cuda.synchronize()
    m.check_status(f"energy_forces, message form {form}")
    Gd = unpack_weights(G.cpu().numpy(), SHAPE.F, SHAPE.K, SHAPE.L, SHAPE.max_z) if grads else None
    return E.cpu().numpy(), F.cpu().numpy(), Gd


def _periodic_batch():
    parts = [synth.random_cluster(20, seed=900 + k, side=12.5, min_dist=1.2) for k in range(3)]
    s = synth.System("pbcbatch3", np.concatenate([p.z for p in parts]), np.concatenate([p.pos for p in parts]),
                     np.repeat(np.arange(3, dtype=np.int32), 20),
                     np.tile((np.eye(3) * 12.5)[None], (3, 1, 1)).astype(np.float32), 3)
    assert margin_ok(s)
    return s


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("form", FORMS)
def test_form_against_oracle_with_weight_gradients(form, precision):
    """A periodic batch of three small boxes on a list with a 1 A skin (so the
    rows hold entries beyond the cutoff, which every form must skip)."""
    s = _periodic_batch()
    m = _model(s, precision, 20000)
    nl = gpu_pairs(m, s, cutoff=6.0)
    E, F, G = _run(m, s, nl, form)
    o = Oracle(W, F=SHAPE.F, K=SHAPE.K, L=SHAPE.L)
    Es, Ei, Fo, Go = o.energy_forces(s.z, s.pos, s.batch, s.box, n_systems=s.n_systems, want_weights=True)
    assert np.all(energy_errors(E, Es, Ei, s.batch) <= E_TOL)
    f_err, f_max = force_errors(F, Fo)
    assert f_err <= F_TOL and f_max <= F_MAX_TOL, (f_err, f_max)
    for k, ref in Go.items():
        rel = np.sqrt(np.mean((G[k].astype(np.float64) - ref) ** 2)) / max(np.sqrt(np.mean(ref ** 2)), 1e-30)
        assert rel <= F_TOL, (form, precision, k, rel)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_forms_agree_on_water3000(precision):
    s = synth.workload("water3000")
    m = _model(s, precision, 250000)
    nl = gpu_pairs(m, s)
    ref = _run(m, s, nl, 3)
    # BF16 mode rounds the message adjoint's outputs to bf16 for its GEMMs, so a
    # reassociated sum may move an operand by one bf16 ulp
    e_tol, f_tol, g_tol = (1e-6, 1e-5, 1e-4) if precision != 1 else (1e-4, 2e-3, 2e-2)
    for form in FORMS:
        E, F, G = _run(m, s, nl, form)
        assert abs(E[0] - ref[0][0]) <= e_tol * abs(ref[0][0]), (form, E, ref[0])
        f_err, _ = force_errors(F, ref[1])
        assert f_err <= f_tol, (form, f_err)
        for k in ref[2]:
            r = ref[2][k].astype(np.float64)
            rel = np.sqrt(np.mean((G[k] - r) ** 2)) / max(np.sqrt(np.mean(r ** 2)), 1e-30)
            assert rel <= g_tol, (form, k, rel)

