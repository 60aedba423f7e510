"""Host logic of the benchmark's roofline report (CPU): the per-kernel
algorithmic-byte models, the extraction of a kernel's source text and the
rule that a stored DRAM-traffic figure is reported only while the kernel's
source is the one it was measured on."""
import hashlib
import json
import os

import bench

# counts of the 4096 x 4096 headline grid (one build)
N_V, A = 16_777_216, 67_092_480
STATS = {"T": 16_777_215, "lr_n": 17_547_804, "c1": 2_097_526, "E2": 14_763_947}


def test_byte_models_are_positive_and_match_their_formulas():
    names = ["k_r1_choose", "k_r1_resolve", "k_r1_label", "k_build_list", "k_run_flags", "k_row_starts",
             "k_prune_leaves", "k_pairs_succ", "k_lr_walk1", "k_lr_final1",
             "k_parent_from_rank", "k_parent_from_owner"]
    for nm in names:
        b = bench.kernel_bytes(nm, N_V, A, STATS, 4)
        assert b is not None and b > 0, nm
    # the list build: offsets, every column (read once, 4 bytes), C1 of both
    # ends of the arcs kept (2 x 4 bytes over half the arcs), the row labels,
    # and a 12-byte entry per inter-component edge
    want = (N_V + 1) * 4 + 4 * A + 4 * N_V + 2 * A + 12 * STATS["E2"]
    assert bench.kernel_bytes("k_build_list", N_V, A, STATS, 4) == want
    # the top list-ranking level: successor read and packed 4-byte record
    # written per element, three words per splitter (K = 16)
    N = STATS["lr_n"]
    assert bench.kernel_bytes("k_lr_walk1", N_V, A, STATS, 4) == 8 * N + 12 * ((N + 15) // 16)
    # a kernel without a model has none
    assert bench.kernel_bytes("k_not_a_kernel", N_V, A, STATS, 4) is None


def test_function_source_takes_the_whole_balanced_body(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("// lead\n__global__ void k_a(int x) {\n  if (x) { x = 1; }\n  { }\n}\n"
                   "__global__ void k_b() {}\n")
    a = bench._function_source(str(src), "k_a")
    assert a.startswith("__global__ void k_a(") and a.endswith("}") and "k_b" not in a
    assert a.count("{") == a.count("}")
    assert bench._function_source(str(src), "k_missing") is None


def test_traffic_is_reported_only_for_the_measured_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2603_11645_gb300" / "csrc"
    csrc.mkdir(parents=True)
    kfile = csrc / "x.cu"
    kfile.write_text("__global__ void k_x(int* p) {\n  p[0] = 1;\n}\n")
    text = bench._function_source(str(kfile), "k_x")
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"file": "paper_2603_11645_gb300/csrc/x.cu", "function": "k_x",
             "sha256": hashlib.sha256(text.encode()).hexdigest(), "bytes_per_unit": 2.5}
    (prof / "traffic.json").write_text(json.dumps({"k_x": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k_x", 1000) == 2500          # scaled to the units
    assert bench.traffic_for("k_other", 1000) is None      # never measured
    kfile.write_text("__global__ void k_x(int* p) {\n  p[0] = 2;\n}\n")
    assert bench.traffic_for("k_x", 1000) is None          # source changed since


def test_committed_traffic_records_name_existing_kernels():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as f:
        d = json.load(f)
    assert d, "no traffic records"
    for key, e in d.items():
        src = bench._function_source(os.path.join(bench.ROOT, e["file"]), e["function"])
        assert src is not None, key
        assert e["bytes_per_unit"] > 0 and e["read_bytes"] + e["write_bytes"] > 0


def test_roofline_entry_for_the_headline_kernel():
    """The roofline object as the bench builds it from live stage times:
    achieved = algorithmic bytes / mean launch time, frac against the peak,
    and the committed traffic converted to a bandwidth fraction."""
    kern = {"k_r1_resolve": [0.48, 0.50], "k_pairs_succ": [0.44, 0.44]}
    r = bench.roofline_entry("k_r1_resolve", kern, N_V, A, STATS, 6786.2, "measured", 3.5 * 2, 1)
    byts = bench.kernel_bytes("k_r1_resolve", N_V, A, STATS, 4)
    assert r["kernel"] == "k_r1_resolve" and r["algorithmic_bytes"] == int(byts)
    assert r["launch_ms"] == 0.49
    assert abs(r["achieved"] - byts / 0.49e-3 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 6786.2) < 1e-4
    assert r["traffic"] == bench.traffic_for("k_r1_resolve", STATS["T"])
    if r["traffic"]:
        assert abs(r["traffic_frac"] - r["traffic"] / 0.49e-3 / 1e9 / 6786.2) < 1e-4
    assert r["share_of_step"] == round(0.98 / 7.0, 3)
    assert bench.roofline_entry(None, kern, N_V, A, STATS, 1.0, "", 1.0, 1) is None
    assert bench.roofline_entry("k_unknown", {"k_unknown": [1.0]}, N_V, A, STATS, 1.0, "", 1.0, 1) is None


def test_reference_arm_line_keeps_the_contract():
    """`bench.py --impl reference` (the CPU oracle on a bounded sample): one
    JSON object with the bench's metric and unit, impl = reference, a
    cpu_baseline describing the run and an e2e entry without host copies;
    ranks other than 0 do no work."""
    import argparse
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2) is None
    line = bench.run_reference(args, 0, 1)
    json.dumps(line)  # serialisable as the printed line
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "edges/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 == e2e["d2h_bytes_per_step"]
