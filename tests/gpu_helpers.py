"""Shared helpers of the GPU parity tests: run the CUDA path (through the
C ABI) and the FP64 oracle on the same seeded inputs and compare."""
import numpy as np
import torch

from oracle.neighbors import minimum_image, neighbor_pairs
from oracle.tensornet import TensorNet as Oracle
from paper_2402_17660_gb300 import synth
from paper_2402_17660_gb300.tnet import TensorNet

RC = 5.0
E_TOL = 1e-5   # |dE_s| <= E_TOL * max(|E_s|, sum_i |E_i|)
F_TOL = 1e-4   # RMS_i |dF_i| <= F_TOL * RMS_i |F_i|
F_MAX_TOL = 2e-3   # max_i |dF_i| <= F_MAX_TOL * RMS_i |F_i| (the worst atom)
BF16_E_TOL = 1e-2
BF16_F_TOL = 1e-2
BF16_F_MAX_TOL = 1e-1

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def to_dev(sys: synth.System):
    pos = torch.from_numpy(np.ascontiguousarray(sys.pos)).to(DEV)
    z = torch.from_numpy(np.ascontiguousarray(sys.z)).to(DEV)
    batch = torch.from_numpy(np.ascontiguousarray(sys.batch)).to(DEV)
    box = None if sys.box is None else torch.from_numpy(np.ascontiguousarray(sys.box)).to(DEV)
    return z, pos, batch, box


def make_model(W, sys, max_pairs=None, shape=synth.ModelShape(), cutoff=RC):
    if max_pairs is None:
        i, _ = neighbor_pairs(sys.pos, sys.batch, sys.box, cutoff) if sys.n_atoms <= 30000 else (None, None)
        max_pairs = int(len(i) * 1.25) + 64 if i is not None else 120 * sys.n_atoms
    return TensorNet(W, F=shape.F, K=shape.K, L=shape.L, max_z=shape.max_z, cutoff_upper=shape.cutoff_upper,
                     max_atoms=max(sys.n_atoms, 1), max_systems=sys.n_systems, max_pairs=max_pairs, device=DEV)


def gpu_pairs(m, sys, cutoff=RC, cap=None):
    z, pos, batch, box = to_dev(sys)
    m.reset_status()
    nl = m.neighbors(pos, batch if sys.n_systems > 1 else None, box, sys.n_systems, cutoff=cutoff, cap=cap)
    torch.cuda.synchronize()
    return nl


def csr_to_pairs(nl):
    rp = nl.row_ptr.cpu().numpy().astype(np.int64)
    n = int(nl.n_pairs.item())
    col = nl.col[:n].cpu().numpy().astype(np.int64)
    i = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return i, col


def margin_ok(sys, cutoff=RC, margin=1e-4):
    i, j = neighbor_pairs(sys.pos, sys.batch, sys.box, cutoff + 2 * margin)
    r = sys.pos.astype(np.float64)[i] - sys.pos.astype(np.float64)[j]
    if sys.box is not None:
        r = np.concatenate([minimum_image(r[sys.batch[i] == s], sys.box[s]) for s in range(sys.n_systems)]) \
            if sys.n_systems > 1 else minimum_image(r, sys.box[0])
    d = np.linalg.norm(r, axis=1)
    return bool(np.all(np.abs(d - cutoff) >= margin))


def gpu_energy_forces(m, sys, nl=None, seed=None, cutoff=RC):
    z, pos, batch, box = to_dev(sys)
    if nl is None:
        nl = gpu_pairs(m, sys, cutoff)
    m.reset_status()
    sd = None if seed is None else torch.tensor(seed, dtype=torch.float32, device=DEV)
    E, F, _ = m.energy_forces(z, pos, nl, batch if sys.n_systems > 1 else None, box, sys.n_systems,
                              forces=True, seed=sd)
    torch.cuda.synchronize()
    m.check_status("energy_forces")
    return E.cpu().numpy(), F.cpu().numpy()


def oracle_energy_forces(W, sys, shape=synth.ModelShape(), seed=None):
    o = Oracle(W, F=shape.F, K=shape.K, L=shape.L, rc=shape.cutoff_upper)
    Es, Ei, Fo, _ = o.energy_forces(sys.z, sys.pos, sys.batch, sys.box, n_systems=sys.n_systems, seed=seed)
    return Es, Ei, Fo


def energy_errors(E, Es, Ei, batch):
    scale = np.maximum(np.abs(Es), np.bincount(batch, weights=np.abs(Ei), minlength=len(Es)))
    return np.abs(E - Es) / scale


def force_error(F, Fo):
    """RMS_i |F_i - Fo_i| / RMS_i |Fo_i|."""
    return np.sqrt(np.mean(np.sum((F - Fo) ** 2, 1))) / np.sqrt(np.mean(np.sum(Fo ** 2, 1)))


def force_errors(F, Fo):
    """(RMS_i |dF_i|, max_i |dF_i|), both relative to RMS_i |Fo_i|."""
    F = np.asarray(F, np.float64)
    Fo = np.asarray(Fo, np.float64)
    d = np.sqrt(np.sum((F - Fo) ** 2, 1))
    rms = np.sqrt(np.mean(np.sum(Fo ** 2, 1)))
    return float(np.sqrt(np.mean(d * d)) / rms), float(d.max() / rms)
