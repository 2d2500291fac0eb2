"""Host logic of the benchmark's roofline figures (no GPU).

The algorithmic byte model behind `roofline.achieved` and the whole-step
bandwidth, and the lookup of the recorded DRAM traffic, checked against
counts written out by hand for small cases.
"""
import bench


N, D, B = 1000, 30, 4


def test_cycle_steps_split_a_restarted_solve():
    assert bench.cycle_steps(7, 50) == [7]
    assert bench.cycle_steps(50, 50) == [50]
    assert bench.cycle_steps(60, 50) == [50, 10]
    assert bench.cycle_steps(100, 50) == [50, 50]


def test_step_bytes_follow_the_update_and_sketch_reads():
    # three steps j = 0, 1, 2 in one cycle
    k = 3
    assert bench.phase_bytes("apply", N, D, k, B) == 3 * 2 * N * B
    # step j reads W, writes S(W), reads Q_0..Q_j for the fused dots
    assert bench.phase_bytes("sketch", N, D, k, B) == sum(N * B + D * B + (j + 1) * D * B for j in range(3))
    # step j reads W and V_0..V_j, writes V_{j+1}, and the same for the sketched column
    assert bench.phase_bytes("update", N, D, k, B) == (3 + 4 + 5) * (N + D) * B
    assert bench.phase_bytes("assemble", N, D, k, B) == 4 * N * B
    assert bench.phase_bytes("init", N, D, k, B) == 3 * N * B
    assert bench.phase_bytes("tikhonov", N, D, k, B) == 0.0


def test_restarted_cycles_restart_the_step_index():
    # 5 steps in cycles of at most 3: j = 0, 1, 2 then j = 0, 1
    upd = bench.phase_bytes("update", N, D, 5, B, m=3)
    assert upd == ((3 + 4 + 5) + (3 + 4)) * (N + D) * B
    # one restart: X += V y over the first cycle's 3 + 1 tensors and the residual's 4 passes
    assert bench.phase_bytes("init", N, D, 5, B, m=3) == 3 * N * B + (3 + 1) * N * B + 4 * N * B
    assert bench.phase_bytes("assemble", N, D, 5, B, m=3) == (2 + 1) * N * B


def test_recorded_traffic_scales_the_ratio_and_drops_stale_lines(tmp_path, monkeypatch):
    sha = bench.source_sha("update")
    f = tmp_path / "traffic.txt"
    f.write_text("# comment\n"
                 f"phase=update workload=w1 dram_ratio=0.5 source_sha={sha}\n"
                 "phase=apply workload=w1 dram_ratio=0.7 source_sha=0000000000000000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic("update", "w1", 1000.0) == 500
    assert bench.recorded_traffic("update", "w2", 1000.0) is None      # no line for this workload
    assert bench.recorded_traffic("apply", "w1", 1000.0) is None       # kernel changed since the capture


def test_committed_traffic_lines_are_current_for_the_reported_groups():
    # the dominant groups of the two rooflines the benchmark reports
    assert bench.recorded_traffic("update", bench.WORKLOAD + "_lockstep16", 1.0) is not None
    assert bench.recorded_traffic("sketch", bench.WORKLOAD, 1.0) is not None
