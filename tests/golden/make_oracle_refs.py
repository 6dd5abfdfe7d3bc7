"""Writes the stored FP64 oracle results that the full-size GPU parity tests
compare against: energies and forces of the ~24,000-atom solvated box and of
the 512-molecule batch, and a five-step velocity-Verlet trajectory of the
3,000-atom water box driven by the oracle's forces.

Only the oracle (`oracle/`) and the seeded input generators (`synth`) are
called.  Each file also stores the inputs it was computed from (atomic
numbers, float32 positions, box, batch, initial velocities), so a test runs
the CUDA path on exactly these inputs, whatever machine regenerates them, and
a checksum of the weights, which the test recomputes.

Run from the repository root:  python tests/golden/make_oracle_refs.py [name ...]
(names: solvated24k batch512 md_water3000; each takes a few minutes and, for
the solvated box, about 30 GB of host memory).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.tensornet import TensorNet as Oracle  # noqa: E402
from paper_2402_17660_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
MD_STEPS = 5
MD_DT = 0.5          # fs
MD_T = 300.0         # K, Maxwell-Boltzmann initial velocities (seed 1)


def weights_checksum(W: dict) -> np.ndarray:
    """Sum and sum of squares of every weight (float64), in blob order."""
    v = np.concatenate([np.asarray(W[k], np.float64).ravel() for k, _ in synth.param_spec(synth.ModelShape())])
    return np.array([v.sum(), (v * v).sum()])


def energy_forces_ref(name: str) -> None:
    s = synth.workload(name)
    W = synth.init_weights(synth.ModelShape(), seed=0)
    t0 = time.time()
    Es, Ei, Fo, _ = Oracle(W).energy_forces(s.z, s.pos, s.batch, s.box, n_systems=s.n_systems)
    dt = time.time() - t0
    abs_ei = np.bincount(s.batch, weights=np.abs(Ei), minlength=s.n_systems)
    out = os.path.join(HERE, f"oracle_{name}.npz")
    np.savez_compressed(out, z=s.z.astype(np.int8), pos=s.pos.astype(np.float32),
                        batch=s.batch.astype(np.int32), n_systems=np.int32(s.n_systems),
                        box=np.zeros((0, 3, 3), np.float32) if s.box is None else s.box.astype(np.float32),
                        energy=Es.astype(np.float64), abs_ei=abs_ei.astype(np.float64),
                        forces=Fo.astype(np.float32), weights_checksum=weights_checksum(W),
                        seconds=np.float64(dt))
    print(f"{name}: N={s.n_atoms} oracle {dt:.1f} s -> {out}")


def md_ref(name: str = "water3000") -> None:
    """Velocity Verlet in FP64 with the oracle's forces: v += dt/2 a;
    x += dt v; forces at x; v += dt/2 a, with a = F / m in A/fs^2."""
    s = synth.workload(name)
    W = synth.md_weights(synth.ModelShape(), seed=0)
    o = Oracle(W)
    v0 = synth.maxwell_boltzmann(s, MD_T, seed=1)
    inv_m = 1.0 / s.masses().astype(np.float64)
    acc = synth.EV_PER_AMU_A2_FS2
    x = s.pos.astype(np.float64)
    v = v0.astype(np.float64)
    t0 = time.time()
    Es, _, F, _ = o.energy_forces(s.z, x, s.batch, s.box)
    xs, vs, ep, ek = [], [], [], []
    for _ in range(MD_STEPS):
        v = v + 0.5 * MD_DT * acc * F * inv_m[:, None]
        x = x + MD_DT * v
        Es, _, F, _ = o.energy_forces(s.z, x, s.batch, s.box)
        v = v + 0.5 * MD_DT * acc * F * inv_m[:, None]
        xs.append(x.copy())
        vs.append(v.copy())
        ep.append(Es[0])
        ek.append(0.5 * np.sum(np.sum(v * v, 1) / inv_m) / acc)
    dt = time.time() - t0
    out = os.path.join(HERE, f"oracle_md_{name}.npz")
    np.savez_compressed(out, z=s.z.astype(np.int8), pos0=s.pos.astype(np.float32), vel0=v0.astype(np.float32),
                        box=s.box.astype(np.float32), dt=np.float64(MD_DT), steps=np.int32(MD_STEPS),
                        pos=np.array(xs[-1]), vel=np.array(vs[-1]), e_pot=np.array(ep), e_kin=np.array(ek),
                        weights_checksum=weights_checksum(W), seconds=np.float64(dt))
    print(f"md {name}: {MD_STEPS} steps, oracle {dt:.1f} s -> {out}")


def main(names: list[str]) -> None:
    for n in names or ["md_water3000", "batch512", "solvated24k"]:
        if n.startswith("md_"):
            md_ref(n[3:])
        else:
            energy_forces_ref(n)


if __name__ == "__main__":
    main(sys.argv[1:])
