"""Host-side logic of bench.py (no GPU): the algorithmic bytes and propagator flops per site of a
coupled step that the step-level roofline fractions divide by, the peaks they are fractions of,
the rule that ties the reported DRAM traffic to the kernel source it was captured on, and the
workload description of the JSON line."""
import bench


def test_step_bytes_per_site():
    # 128^3 workload: N = 64, 4 inversion iterations of 2 density evaluations, 8 Jacobi sweeps, LB
    assert bench.step_bytes_per_site(64, 4, 8, 1) == 8 * (8 * 64 + 64) + 24 + 44 + 40 * 8 + 180
    assert bench.step_bytes_per_site(64, 4, 8, 1, es=8) == 2 * bench.step_bytes_per_site(64, 4, 8, 1)
    assert bench.step_bytes_per_site(64, 4, 8, 0) == bench.step_bytes_per_site(64, 4, 8, 1) - 180
    assert bench.step_bytes_per_site(16, 6, 8, 1, evals_per_iter=1) == 6 * (8 * 16 + 64) + 24 + 44 + 320 + 180


def test_step_prop_flops_per_site():
    assert bench.step_prop_flops_per_site(64, 4) == 2 * 4 * 28 * 64
    assert bench.step_prop_flops_per_site(10, 1, evals_per_iter=1) == 280


def test_peaks_come_from_the_measured_file():
    import json
    import os
    d = json.load(open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")))
    assert bench.peaks() == (float(d["hbm_gbs"]), "measured")
    assert bench.bf16_peak() == (float(d["bf16_tflops"]), "measured burst")


def test_traffic_record_applies_only_to_the_source_it_was_taken_on(tmp_path):
    """The DRAM traffic per contour step is reported only while the sweep's source is the one the
    committed ncu capture ran (hash match) and for the same chain length."""
    import json
    import os
    src = os.path.join(bench.ROOT, "paper_1204_2088_gb300", "csrc", "dscf_pers.cu")
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["prop_sweep"]
    assert bench.ncu_traffic(src, rec["N"]) == rec["dram_bytes_per_contour_step"]
    assert bench.ncu_traffic(src, rec["N"] + 1) is None
    changed = tmp_path / "dscf_pers.cu"
    changed.write_bytes(open(src, "rb").read() + b"\n")
    assert bench.ncu_traffic(str(changed), rec["N"]) is None


def test_workload_config_names_the_workload():
    from paper_1204_2088_gb300 import inputs
    c = bench.workload_config(inputs.workload("melt128"))
    assert c["workload"].startswith("melt128: AB diblock melt, 128x128x128 periodic, N=64, nA=19, chi N=25,")
    assert c["grid"] == [128, 128, 128] and c["N"] == 64 and c["hydro"] == 1
    assert "l2" in c
