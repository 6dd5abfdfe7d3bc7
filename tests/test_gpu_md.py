"""GPU checks of tnet_md_step: five steps follow a velocity-Verlet
trajectory driven by the FP64 oracle's forces (stored in tests/golden by
make_oracle_refs.py, which calls only the oracle); one step equals a
hand-assembled velocity Verlet step built from tnet_energy_forces; graph
replays equal the eager path bit for bit; the total energy is conserved over
a short run."""
import os

import numpy as np
import pytest
import torch

from paper_2402_17660_gb300 import synth

from .gpu_helpers import DEV, gpu_energy_forces, gpu_pairs, make_model, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

W = synth.md_weights(synth.ModelShape(), seed=0)
ACC = synth.EV_PER_AMU_A2_FS2


def _state(sys):
    z, pos, _, box = to_dev(sys)
    vel = torch.from_numpy(synth.maxwell_boltzmann(sys, 300.0, seed=1)).to(DEV)
    inv_m = torch.from_numpy(1.0 / sys.masses()).to(DEV)
    return z, pos, vel, inv_m, box


@pytest.mark.parametrize("name", ["water3000", "triclinic"])
def test_one_step_matches_velocity_verlet(name):
    s = synth.workload(name) if name != "triclinic" else synth.triclinic_water(6, 18.6, seed=5, radii=(5.0, 6.0))
    m = make_model(W, s, max_pairs=300000)
    z, pos, vel, inv_m, box = _state(s)
    dt = 0.5
    E0, F0 = gpu_energy_forces(m, s)
    p1, v1 = pos.clone(), vel.clone()
    m.reset_status()
    ek, ep = m.md(z, inv_m, p1, v1, box, dt, 1.0, 20, 1)
    torch.cuda.synchronize()
    m.check_status("md")
    F0t = torch.from_numpy(F0).to(DEV)
    vh = vel + 0.5 * dt * ACC * F0t * inv_m[:, None]
    x1 = pos + dt * vh
    assert torch.allclose(p1, x1, rtol=0, atol=1e-5)
    s1 = synth.System(s.name, s.z, x1.cpu().numpy(), s.batch, s.box, 1)
    E1, F1 = gpu_energy_forces(m, s1, nl=gpu_pairs(m, s1, cutoff=6.0))
    v_ref = vh + 0.5 * dt * ACC * torch.from_numpy(F1).to(DEV) * inv_m[:, None]
    assert torch.allclose(v1, v_ref, rtol=0, atol=1e-5)
    assert abs(ep[0].item() - E1[0]) <= 1e-5 * abs(E1[0]) + 1e-3
    ke = 0.5 * np.sum(np.sum(v1.cpu().numpy().astype(np.float64) ** 2, 1) / (1.0 / s.masses())) / ACC
    assert abs(ek[0].item() - ke) <= 1e-6 * ke


@pytest.mark.parametrize("prec", [0, 2])
def test_md_follows_the_oracle_trajectory(prec):
    """Water3000, Maxwell-Boltzmann velocities at 300 K, 0.5 fs steps, list at
    cutoff + 1 A skin: after five steps of tnet_md_step (FP32 state) every
    position is within 1e-5 A and every velocity within 1e-4 of the RMS
    velocity of the FP64 oracle's trajectory; per-step potential energies
    within 1e-5 relative, kinetic energies within 1e-6."""
    d = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_md_water3000.npz"))
    wv = np.concatenate([np.asarray(W[k], np.float64).ravel() for k, _ in synth.param_spec(synth.ModelShape())])
    assert np.allclose([wv.sum(), (wv * wv).sum()], d["weights_checksum"], rtol=1e-13, atol=0)
    s = synth.System("water3000", d["z"].astype(np.int32), d["pos0"], np.zeros(len(d["z"]), np.int32), d["box"], 1)
    from paper_2402_17660_gb300.tnet import TensorNet
    m = TensorNet(W, max_atoms=s.n_atoms, max_systems=1, max_pairs=300000, precision=prec, device=DEV)
    z, pos, _, box = to_dev(s)
    vel = torch.from_numpy(d["vel0"]).to(DEV)
    inv_m = torch.from_numpy(1.0 / s.masses()).to(DEV)
    n = int(d["steps"])
    m.reset_status()
    ek, ep = m.md(z, inv_m, pos, vel, box, float(d["dt"]), 1.0, 20, n)
    torch.cuda.synchronize()
    m.check_status("md")
    dx = np.abs(pos.cpu().numpy().astype(np.float64) - d["pos"]).max()
    v_rms = np.sqrt(np.mean(np.sum(d["vel"] ** 2, 1)))
    dv = np.sqrt(np.sum((vel.cpu().numpy().astype(np.float64) - d["vel"]) ** 2, 1)).max() / v_rms
    de = np.abs(ep.cpu().numpy() - d["e_pot"]).max() / np.abs(d["e_pot"]).max()
    dk = np.abs(ek.cpu().numpy() - d["e_kin"]).max() / np.abs(d["e_kin"]).max()
    print(f"md vs oracle (precision {prec}): max |dx| {dx:.2e} A, max |dv| {dv:.2e} of RMS v, E_pot {de:.2e}, "
          f"E_kin {dk:.2e}")
    assert dx <= 1e-5 and dv <= 1e-4 and de <= 1e-5 and dk <= 1e-6


def test_graph_replay_equals_eager():
    s = synth.workload("water3000")
    m = make_model(W, s, max_pairs=300000)
    z, pos, vel, inv_m, box = _state(s)
    pa, va = pos.clone(), vel.clone()
    pb, vb = pos.clone(), vel.clone()
    m.reset_status()
    eka, epa = m.md(z, inv_m, pa, va, box, 0.5, 1.0, 10, 20)   # two graph replays
    ekb, epb = m.md(z, inv_m, pb, vb, box, 0.5, 1.0, 10, 5)    # eager path (5 < 10)
    ekb2, epb2 = m.md(z, inv_m, pb, vb, box, 0.5, 1.0, 10, 5)
    torch.cuda.synchronize()
    m.check_status("md")
    # the eager run rebuilt at steps 0 and 5 of each call; compare with a
    # replayed run that rebuilds at the same steps instead
    pc, vc = pos.clone(), vel.clone()
    ekc, epc = m.md(z, inv_m, pc, vc, box, 0.5, 1.0, 5, 10)     # graph of 5 steps, replayed twice
    torch.cuda.synchronize()
    assert torch.equal(pc, pb) and torch.equal(vc, vb)
    assert torch.equal(epc[:5], epb) and torch.equal(epc[5:], epb2)
    assert np.isfinite(epa.cpu().numpy()).all() and np.isfinite(eka.cpu().numpy()).all()


def test_energy_conservation_short_run():
    s = synth.workload("water3000")
    m = make_model(W, s, max_pairs=300000)
    z, pos, vel, inv_m, box = _state(s)
    m.reset_status()
    ek, ep = m.md(z, inv_m, pos, vel, box, 0.25, 1.0, 20, 200)
    torch.cuda.synchronize()
    m.check_status("md")
    et = (ek + ep).cpu().numpy()
    ke = ek.cpu().numpy()
    drift = abs(et[-1] - et[0]) / s.n_atoms
    fluct = np.std(ke) / s.n_atoms
    print(f"E_tot drift per atom over 50 fs: {drift:.3e} eV; KE fluctuation per atom {fluct:.3e} eV")
    assert drift < max(0.05 * np.std(ke), 1e-3 * s.n_atoms) / s.n_atoms


def test_triggered_rebuilds_make_the_trajectory_schedule_independent():
    """A thin skin forces displacement-triggered rebuilds between the
    periodic ones; every list then holds all pairs within the cutoff, and
    only active pairs enter the sums, so the trajectory equals the one with
    a fresh cutoff list in every step, bit for bit."""
    s = synth.workload("water3000")
    m = make_model(W, s, max_pairs=300000)
    z, pos, vel, inv_m, box = _state(s)
    pa, va = pos.clone(), vel.clone()
    pb, vb = pos.clone(), vel.clone()
    m.reset_status()
    eka, epa = m.md(z, inv_m, pa, va, box, 0.5, 0.2, 20, 40)
    n_a = m.md_rebuilds()
    ekb, epb = m.md(z, inv_m, pb, vb, box, 0.5, 0.0, 1, 40)
    n_b = m.md_rebuilds()
    torch.cuda.synchronize()
    m.check_status("md")
    assert n_b == 41                   # the initial build plus one per step
    assert 3 < n_a < 41                # periodic (2) + initial + triggered ones
    assert torch.equal(pa, pb) and torch.equal(va, vb)
    assert torch.equal(epa, epb) and torch.equal(eka, ekb)


def test_md_neighbor_list_is_the_list_at_the_last_rebuild():
    """With a rebuild in every step, the list md() keeps equals a fresh
    tnet_neighbors call at cutoff + skin on the final positions."""
    s = synth.workload("water3000")
    m = make_model(W, s, max_pairs=300000)
    z, pos, vel, inv_m, box = _state(s)
    m.reset_status()
    m.md(z, inv_m, pos, vel, box, 0.5, 1.0, 1, 3)
    torch.cuda.synchronize()
    m.check_status("md")
    a = m.md_neighbor_list(s.n_atoms)
    b = m.neighbors(pos, None, box, 1, cutoff=6.0)
    torch.cuda.synchronize()
    n = int(b.n_pairs.item())
    assert int(a.n_pairs.item()) == n
    assert torch.equal(a.row_ptr, b.row_ptr) and torch.equal(a.col[:n], b.col[:n])

