"""Host-side checks of the C-ABI library (no GPU needed): the library loads,
exports every function include/tnet.h declares, reports shapes and workspace
sizes, and the Python blob layout agrees with the header and the
generators."""
import ctypes
import os

import numpy as np
import pytest
import torch

from paper_2402_17660_gb300 import _lib, synth, tnet


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _lib.header_functions()
    assert {"tnet_neighbors", "tnet_energy_forces", "tnet_md_step", "tnet_create"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_weights_count_matches_layouts(lib):
    for F, K, L in ((128, 32, 2), (64, 8, 0), (128, 32, 1), (256, 64, 3)):
        d = _lib.ModelDesc(F, K, L, 100, 5.0, 0.0, 0)
        n = lib.tnet_weights_count(ctypes.byref(d))
        spec = synth.param_spec(synth.ModelShape(F=F, K=K, L=L))
        assert n == sum(int(np.prod(s)) for _, s in spec)
        assert [(a, tuple(b)) for a, b in tnet.blob_layout(F, K, L, 100)] == [(a, tuple(b)) for a, b in spec]


def test_invalid_shapes_rejected(lib):
    for bad in ((100, 32, 2), (128, 7, 2), (128, 32, 9), (128, 32, -1)):
        d = _lib.ModelDesc(*bad, 100, 5.0, 0.0, 0)
        assert lib.tnet_weights_count(ctypes.byref(d)) == -1
    d = _lib.ModelDesc(128, 32, 2, 100, 5.0, 6.0, 0)
    assert lib.tnet_weights_count(ctypes.byref(d)) == -1


def test_workspace_bytes(lib):
    d = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0)
    a = lib.tnet_workspace_bytes(ctypes.byref(d), 1000, 1, 100000)
    b = lib.tnet_workspace_bytes(ctypes.byref(d), 2000, 1, 200000)
    assert 0 < a < b
    assert lib.tnet_workspace_bytes(ctypes.byref(d), 0, 1, 10) == -1


def test_recompute_edges_shrinks_workspace(lib):
    keep = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0)
    rec = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 1)
    a = lib.tnet_workspace_bytes(ctypes.byref(keep), 3000, 1, 160000)
    b = lib.tnet_workspace_bytes(ctypes.byref(rec), 3000, 1, 160000)
    # one layer's radial-MLP activations: 9 F floats per undirected pair (a1,
    # h1, a2, h2, a3; the filter g = phi SiLU(a3) is never stored)
    assert a - b >= 9 * 128 * 4 * 80000
    one = _lib.ModelDesc(128, 32, 1, 100, 5.0, 0.0, 0, 0)
    one_r = _lib.ModelDesc(128, 32, 1, 100, 5.0, 0.0, 0, 1)
    assert lib.tnet_workspace_bytes(ctypes.byref(one), 3000, 1, 160000) == \
        lib.tnet_workspace_bytes(ctypes.byref(one_r), 3000, 1, 160000)
    bad = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 2)
    assert lib.tnet_workspace_bytes(ctypes.byref(bad), 3000, 1, 160000) == -1


def test_create_rejects_bad_workspace(lib):
    d = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0)
    ctx = ctypes.c_void_p()
    rc = lib.tnet_create(ctypes.byref(ctx), ctypes.byref(d), 100, 1, 1000, None, 0)
    assert rc == 7 and not ctx.value
    rc = lib.tnet_create(ctypes.byref(ctx), ctypes.byref(d), 100, 1, 1000, ctypes.c_void_p(0x1001), 1 << 40)
    assert rc == 7


def test_null_context_rejected(lib):
    assert lib.tnet_neighbors(None, 10, 1, None, None, None, ctypes.c_float(5.0), None, None, 0, None,
                              None, None) == 1
    assert lib.tnet_energy_forces(None, None, 1, 1, None, None, None, None, None, None, None, None, None,
                                  None, None, None) == 1
    assert lib.tnet_md_step(None, None, 1, None, None, None, None, None, ctypes.c_float(0.5),
                            ctypes.c_float(1.0), 20, 10, None, None, None, None) == 1
    assert lib.tnet_status_string(2).decode() == "pair capacity exceeded"


def test_pack_unpack_roundtrip():
    W = synth.init_weights(synth.ModelShape(F=64, K=8, L=1), seed=3)
    blob = tnet.pack_weights(W, 64, 8, 1, 100)
    back = tnet.unpack_weights(blob, 64, 8, 1, 100)
    for k in W:
        assert np.array_equal(back[k], W[k])


def test_tuning_knobs_exported(lib):
    from paper_2402_17660_gb300 import tnet
    knobs = tnet.tuning_knobs(lib)
    assert len(knobs) == lib.tnet_tuning_knobs() >= 4
    for name, cands in knobs:
        assert name and len(cands) >= 2 and all(c >= 0 for c in cands) and len(set(cands)) == len(cands)
    assert lib.tnet_tuning_name(99) is None
    assert lib.tnet_set_tuning(None, None, 0) == 1


def test_radial_table_workspace(lib):
    """Table mode keeps the tables (2 (L+1) n 3F floats) and per-pair f, g and
    their d-derivatives, but none of the per-pair radial-MLP activations."""
    plain = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0, 0)
    tab = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0, 4096)
    a = lib.tnet_workspace_bytes(ctypes.byref(plain), 3000, 1, 160000)
    b = lib.tnet_workspace_bytes(ctypes.byref(tab), 3000, 1, 160000)
    assert 0 < b < a
    for n in (1, 255, 16385, -4):
        bad = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0, n)
        assert lib.tnet_workspace_bytes(ctypes.byref(bad), 3000, 1, 160000) == -1
    for n in (256, 16384):
        ok = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0, n)
        assert lib.tnet_workspace_bytes(ctypes.byref(ok), 3000, 1, 160000) > 0
    assert lib.tnet_radial_tables(None, None, None) == 1


def test_plain_c_client(lib, tmp_path):
    """include/tnet.h is a C99 header: a C program includes it, links
    libtnet.so and calls the host-side entry points (no GPU needed)."""
    import shutil
    import subprocess
    from paper_2402_17660_gb300 import build as _build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(r'''
#include <stdio.h>
#include "tnet.h"
int main(void) {
    tnet_model_desc d = {128, 32, 2, 100, 5.0f, 0.0f, 0, 0, 0};
    int64_t nw = tnet_weights_count(&d);
    int64_t ws = tnet_workspace_bytes(&d, 3000, 1, 160000);
    tnet_model_desc bad = d;
    bad.radial_table = 100;
    printf("%lld %lld %lld %d %s\n", (long long)nw, (long long)ws,
           (long long)tnet_workspace_bytes(&bad, 3000, 1, 160000), tnet_tuning_knobs(),
           tnet_status_string(TNET_ERR_CAPACITY));
    return (nw > 0 && ws > 0) ? 0 : 1;
}
''')
    exe = tmp_path / "client"
    libdir = os.path.dirname(_build.LIB)
    root = os.path.dirname(os.path.dirname(os.path.abspath(_build.__file__)))
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", str(src), "-I", os.path.join(root, "include"),
                    "-L", libdir, "-ltnet", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    d = _lib.ModelDesc(128, 32, 2, 100, 5.0, 0.0, 0, 0, 0)
    assert int(out[0]) == lib.tnet_weights_count(ctypes.byref(d))
    assert int(out[1]) == lib.tnet_workspace_bytes(ctypes.byref(d), 3000, 1, 160000)
    assert int(out[2]) == -1 and int(out[3]) == lib.tnet_tuning_knobs()


def test_missing_library_fails_loudly(tmp_path):
    """There is no CPU fallback: asking for a library that is not there (and
    not building it) raises instead of returning a stand-in."""
    from paper_2402_17660_gb300 import _lib
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(str(tmp_path / "libtnet.so"), build_if_missing=False)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_model_without_a_gpu_raises():
    """Without a CUDA device the model cannot be built: nothing falls back to
    the host."""
    from paper_2402_17660_gb300 import synth
    from paper_2402_17660_gb300.tnet import TensorNet
    W = synth.init_weights(synth.ModelShape(), seed=0)
    with pytest.raises(Exception):
        TensorNet(W, max_atoms=10, max_systems=1, max_pairs=100)
