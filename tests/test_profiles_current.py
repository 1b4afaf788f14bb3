"""The DRAM traffic recorded from ncu captures (profiles/ncu_traffic.txt) belongs to the kernels as
they are now: bench.py reports a kernel's recorded traffic only while the hash of its definition
matches, so a stale line would silently turn its roofline traffic into null.  A kernel changed on
purpose needs a new capture, or its line removed.  Host-only."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def recorded_lines():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")) as f:
        for ln in f:
            if ln.startswith("kernel="):
                yield dict(p.split("=", 1) for p in ln.split())


def test_recorded_traffic_matches_the_current_kernels():
    lines = list(recorded_lines())
    assert lines
    for kv in lines:
        assert bench.kernel_source_sha(kv["kernel"]) == kv["source_sha"], (
            "%s changed since its ncu capture: capture it again or drop its line" % kv["kernel"])
        assert float(kv["dram_bytes_per_launch"]) > 0


def test_the_benchmark_step_kernels_have_recorded_traffic():
    """The FP64 pair form's three step kernels (the benchmark's default), the dominant pass 2 among
    them, carry ncu traffic scaled to the full configuration-3 launch."""
    nb = 116920848
    for k in bench.FLOPS_BOND_PAIRS:
        t = bench.recorded_traffic(k, nb)
        assert t is not None and t > nb  # more than a byte per directed bond
