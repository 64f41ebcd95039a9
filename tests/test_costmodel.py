"""Host logic of the measurement: the DRAM-traffic table lookup (valid only for the sources it was taken
from) and the per-launch work figures of the cost model."""
import os

from paper_2402_04514_gb300 import assembly, costmodel


def test_traffic_table_lookup(tmp_path):
    dg = costmodel.library_source_digest()
    assert len(dg) == 16
    t = tmp_path / "traffic.txt"
    t.write_text("# comment\n"
                 f"high 1000 300 100 {dg}\n"
                 f"high 1000 600 200 {dg} mixed\n"
                 "edge 1000 50 50 0123456789abcdef\n")
    assert costmodel.measured_traffic(str(t), "high", 4000) == 1600.0
    assert costmodel.measured_traffic(str(t), "high", 4000, "mixed") == 3200.0
    assert costmodel.measured_traffic(str(t), "edge", 4000) is None  # taken from other sources
    assert costmodel.measured_traffic(str(t), "low", 4000) is None
    assert costmodel.measured_traffic(str(tmp_path / "missing.txt"), "high", 4000) is None


def test_committed_traffic_table_parses():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "dram_traffic_q2_512_four_quadrant.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert rows and all(len(r) == 6 and r[5] in ("fp64", "mixed") and len(r[4]) == 16 for r in rows)
    assert {r[0] for r in rows} == {"high", "edge", "low"}


def test_work_figures_are_positive_and_scale_with_the_mesh():
    small = costmodel.Counts.of(assembly.assemble_2d(8, 8, 2))
    large = costmodel.Counts.of(assembly.assemble_2d(16, 16, 2))
    for fn in (costmodel.bytes_per_launch, costmodel.flops_per_launch):
        a, b = fn(small), fn(large)
        for k in ("prim", "edge", "low", "high", "limit2", "final"):
            assert a[k] > 0 and 3.0 < b[k] / a[k] < 5.0, (fn.__name__, k)
