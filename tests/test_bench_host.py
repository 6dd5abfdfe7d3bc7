"""Host-side logic of bench.py (no GPU): the source revision that guards the
stored DRAM-traffic figures, and the algorithmic work model the roofline line
divides by."""
import json
import os

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_2402_17660_gb300", "csrc")


def test_definition_is_the_whole_function():
    text = open(os.path.join(CSRC, "model.cu")).read()
    body = bench._definition(text, "k_message_bwd")
    assert body.startswith("__global__") and body.endswith("}")
    assert body.count("{") == body.count("}")
    assert "k_message_bwd(" in body and "k_node_norm_bwd" not in body
    helper = bench._definition(text, "tab_slope")
    assert helper.startswith("__device__") and "inv_h" in helper
    with pytest.raises(KeyError):
        bench._definition(text, "no_such_kernel")


def test_revision_follows_only_its_own_source(tmp_path, monkeypatch):
    d = tmp_path / "paper_2402_17660_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "a.cu").write_text("__global__ void k_one(int *x) { x[0] = 1; }\n"
                            "__global__ void k_two(int *x) { if (x) { x[1] = 2; } }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    one, two = bench.kernel_revision(["a.cu:k_one"]), bench.kernel_revision(["a.cu:k_two"])
    (d / "a.cu").write_text("__global__ void k_one(int *x) { x[0] = 1; }\n"
                            "__global__ void k_two(int *x) { if (x) { x[1] = 3; } }\n")
    assert bench.kernel_revision(["a.cu:k_one"]) == one
    assert bench.kernel_revision(["a.cu:k_two"]) != two


def test_stored_traffic_entries_resolve():
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, e in t.items():
        workload, precision, tag = key.split(":")[:3]
        assert e["bytes_per_launch"] > 0
        bench.kernel_revision(e.get("rev_files"))   # every named definition exists


def test_table_mode_work_model():
    """With tabulated radial functions the message adjoint writes no dE/da3 and
    reads no a3 from HBM, so its algorithmic bytes fall; the per-pair MLP
    stages have no table-mode work model (they do not run)."""
    nu, N, E, F, K = 81048, 3000, 162096, 128, 32
    fx, bx, ex = bench.stage_work("message_bwd", nu, N, E, F, K, "tf32x3")
    ft, bt, et = bench.stage_work("message_bwd", nu, N, E, F, K, "tf32x3", table=2048)
    assert ex == et == "hbm" and bt < bx
    node = 4.0 * 9 * N * F
    assert bt == 4 * node + 8.0 * E + 2047 * 3 * F * 16.0 + 2 * 4.0 * nu
    for tag in ("mlp1", "mlp2", "mlp3", "mlp1_bwd", "mlp2_bwd", "mlp3_bwd"):
        assert bench.stage_work(tag, nu, N, E, F, K, "tf32x3", table=2048) is None


def test_operand_copies_only_in_bf16_mode():
    """The 3xTF32 mode splits its operands in shared memory and writes no
    copies: its message adjoint moves the FP32 path's bytes; BF16 adds 2 B per
    copied element (dE/dY) and writes dE/da3 only as its bf16 copy."""
    nu, N, E, F, K = 81048, 3000, 162096, 128, 32
    b32 = bench.stage_work("message_bwd", nu, N, E, F, K, "fp32")[1]
    bx3 = bench.stage_work("message_bwd", nu, N, E, F, K, "tf32x3")[1]
    bbf = bench.stage_work("message_bwd", nu, N, E, F, K, "bf16")[1]
    assert b32 == bx3
    assert bbf == b32 + 2.0 * 9 * N * F - 2.0 * 3 * F * nu


def test_cpu_baseline_times_the_sample_on_one_thread_too():
    """The CPU baseline record states how the oracle uses the host cores and
    times the same sample again in a child process on one thread."""
    from paper_2402_17660_gb300 import synth
    W = synth.init_weights(synth.ModelShape(), seed=0)    # the shape the oracle timing assumes
    s = synth.random_cluster(12, seed=3)
    rec, ref = bench.cpu_baseline(s, W)
    assert rec["kind"] == "oracle" and rec["measured_on_full_workload"] and ref is not None
    assert "threads" in rec
    st = rec["single_thread"]
    assert st is not None and st["cores"] == 1 and st["value"] > 0 and st["seconds_per_sample_eval"] > 0


def test_stage_roofline_reproduces_a_measured_line():
    """The roofline helper on the numbers of a water96k bench line (message
    adjoint: 4.1743 ms per launch) gives that line's HBM fraction; a 3xTF32
    GEMM stage is bound by the tensor roof (a third of the TF32 rate)."""
    peaks = {"hbm_gbs": 6685.8, "bf16_tflops": 1991.1}
    nu, N, E = 2585414, 96000, 5170828
    r = bench.stage_roofline("message_bwd", 4.174331029256185, nu, N, E, 128, 32, "tf32x3", 0, False, peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["algorithmic_bytes_per_launch"] - 9784255400.0) < 1.0
    assert abs(r["frac"] - 0.3505803042423122) < 1e-12
    g = bench.stage_roofline("mlp3", 2.18, nu, N, E, 128, 32, "tf32x3", 0, False, peaks)
    assert g["bound"] == "tensor" and abs(g["peak"] - 1991.1 / 6) < 1e-9
    assert abs(g["achieved"] - 2.0 * nu * 256 * 384 / 2.18e-3 / 1e12) < 1e-9
