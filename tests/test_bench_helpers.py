"""bench.py's roofline helpers (no GPU): the algorithmic bytes of one
residual, and the DRAM traffic record, which is reported only for the
captured workload and only while the kernel sources match the capture."""
import os
import types

import bench


def test_spmv_bytes_counts_values_indices_and_vectors_once():
    s = types.SimpleNamespace(nnz=10, n=7, m=5)
    # 10 entries x (4 B value + 4 B index) + x (7 x 4 B) + b and r (2 x 5 x 4 B)
    assert bench.spmv_bytes(s, 4, 4) == 10 * 8 + 7 * 4 + 2 * 5 * 4
    assert bench.spmv_bytes(s, 8, 8) == 10 * 12 + 7 * 8 + 2 * 5 * 8


def test_traffic_record_matches_the_committed_kernels():
    s = types.SimpleNamespace(m=1 << 20, n=1 << 20, nnz=9692830)
    t32 = bench.profiled_traffic("k_residual<float,float>", s)
    t64 = bench.profiled_traffic("k_residual<double,float>", s)
    assert t32 is not None and t64 is not None
    # within 10% of the algorithmic bytes: no re-reads
    assert 1.0 <= t32 / bench.spmv_bytes(s, 4, 4) <= 1.1
    assert 1.0 <= t64 / bench.spmv_bytes(s, 4, 8) <= 1.1


def test_traffic_record_is_dropped_for_other_workloads_or_changed_sources(tmp_path, monkeypatch):
    s = types.SimpleNamespace(m=1 << 20, nnz=9692830)
    assert bench.profiled_traffic("k_residual<float,float>", types.SimpleNamespace(m=1 << 18, nnz=5)) is None
    src = open(os.path.join(bench.ROOT, bench.KERNEL_SOURCES[0])).read()
    marker = bench.RESIDUAL_REGION[0]
    # a change outside the residual kernel's region keeps the record ...
    outside = tmp_path / "outside.cu"
    outside.write_text(src + "\n// changed elsewhere\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", (str(outside), bench.KERNEL_SOURCES[1]))
    assert bench.profiled_traffic("k_residual<float,float>", s) is not None
    # ... a change inside it drops the record
    inside = tmp_path / "inside.cu"
    inside.write_text(src.replace(marker, marker + "\n// changed"))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", (str(inside), bench.KERNEL_SOURCES[1]))
    assert bench.profiled_traffic("k_residual<float,float>", s) is None


def test_block_residual_traffic_record_matches_the_committed_kernel():
    s = types.SimpleNamespace(m=1 << 20, n=1 << 20, nnz=9692830)
    t32 = bench.profiled_traffic("k_mres<float,float,16>", s)
    t64 = bench.profiled_traffic("k_mres<double,float,16>", s)
    assert t32 is not None and t64 is not None
    # X's random row gathers re-read part of X (67 / 134 MB against L2)
    assert 1.0 <= t32 / bench.mres_bytes(s, 16, 4, 4) <= 1.6
    assert 1.0 <= t64 / bench.mres_bytes(s, 16, 4, 8) <= 2.0
    assert bench.profiled_traffic("k_mres<float,float,8>", s) is None
