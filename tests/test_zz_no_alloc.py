"""The allocation-free neighbor search (tnet_neighbors_noalloc) against the
context-based tnet_neighbors, through the C ABI.

Some callers cannot allocate device memory (a host framework that owns the
pool, a real-time loop that forbids cudaMalloc, a plain C caller with no
allocator); this entry point serves them from a fixed static scratch array.
The test runs two different systems back to back through it (the second
call must not see the first call's leftovers) and requires the same pair
list, bit for bit, as the existing entry point."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2402_17660_gb300 import _lib, synth
from paper_2402_17660_gb300.tnet import TensorNet

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
W = synth.init_weights(synth.ModelShape(), seed=0)


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _inputs(sys):
    pos = torch.from_numpy(np.ascontiguousarray(sys.pos)).to(DEV)
    batch = torch.from_numpy(sys.batch).to(DEV) if sys.n_systems > 1 else None
    box = torch.from_numpy(sys.box).to(DEV) if sys.box is not None else None
    return pos, batch, box


def _noalloc(lib, sys, cap):
    pos, batch, box = _inputs(sys)
    row_ptr = torch.empty(sys.n_atoms + 1, dtype=torch.int32, device=DEV)
    col = torch.full((cap,), -7, dtype=torch.int32, device=DEV)
    npairs = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    rc = lib.tnet_neighbors_noalloc(sys.n_atoms, sys.n_systems, _p(pos), _p(batch), _p(box),
                                    ctypes.c_float(5.0), _p(row_ptr), _p(col), cap, _p(npairs), _p(status),
                                    stream)
    assert rc == 0
    return row_ptr, col, npairs, status


def _reference(sys, cap):
    m = TensorNet(W, max_atoms=sys.n_atoms, max_systems=sys.n_systems, max_pairs=cap, device=DEV)
    pos, batch, box = _inputs(sys)
    m.reset_status()
    nl = m.neighbors(pos, batch, box, sys.n_systems)
    torch.cuda.synchronize()
    assert int(m.status.item()) == 0
    return nl


def test_noalloc_matches_context_entry_point_twice_in_a_row():
    lib = _lib.load()
    cases = [synth.workload("water3000"), synth.molecule_batch(64, seed=5)]
    cap = 80 * 3000
    outs = [_noalloc(lib, s, cap) for s in cases]       # two calls in a row
    torch.cuda.synchronize()
    for s, (row_ptr, col, npairs, status) in zip(cases, outs):
        ref = _reference(s, cap)
        n = int(ref.n_pairs.item())
        assert int(status.item()) == 0
        assert int(npairs.item()) == n
        assert torch.equal(row_ptr, ref.row_ptr)
        assert torch.equal(col[:n], ref.col[:n])


@pytest.mark.parametrize("n_atoms,n_systems", [(20000, 1), (2000, 1025)])
def test_noalloc_rejects_sizes_beyond_its_limit(n_atoms, n_systems):
    """Beyond 16,384 atoms or 1,024 systems the call returns WORKSPACE (7) at
    once and enqueues nothing: the outputs keep their sentinels."""
    lib = _lib.load()
    rng = np.random.default_rng(1)
    pos = torch.from_numpy(rng.uniform(0, 60, (n_atoms, 3)).astype(np.float32)).to(DEV)
    batch = torch.from_numpy(np.sort(rng.integers(0, n_systems, n_atoms)).astype(np.int32)).to(DEV)
    out = torch.full((n_atoms + 1,), -3, dtype=torch.int32, device=DEV)
    col = torch.full((16,), -5, dtype=torch.int32, device=DEV)
    npairs = torch.full((1,), -9, dtype=torch.int64, device=DEV)
    status = torch.full((1,), -11, dtype=torch.int32, device=DEV)
    rc = lib.tnet_neighbors_noalloc(n_atoms, n_systems, _p(pos), _p(batch), None, ctypes.c_float(5.0), _p(out),
                                    _p(col), 16, _p(npairs), _p(status), None)
    assert rc == 7
    torch.cuda.synchronize()
    assert bool((out == -3).all()) and bool((col == -5).all())
    assert int(npairs.item()) == -9 and int(status.item()) == -11
