"""The stored accepted pools of the 256-experiment batched workload are the oracle's: the
three cheapest experiments are re-derived here with the FP64 oracle (every one of their 1e5
draws scored, the K = 1000 smallest (M, draw index) kept) and must reproduce their stored
lines exactly, and the file covers all 256 experiments with the workload's shapes."""
import importlib.util
from pathlib import Path

GOLDEN = Path(__file__).resolve().parent / "golden"


def _maker():
    spec = importlib.util.spec_from_file_location("make_batched_golden", GOLDEN / "make_batched_golden.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_batched_golden_lines_are_the_oracles():
    m = _maker()
    stored = m.read_lines()
    wls = m.batched_workloads(256)
    assert sorted(stored) == list(range(256))
    for e, w in enumerate(wls):
        f = stored[e].split()
        assert (int(f[1]), int(f[2]), f[3], int(f[4])) == (w.n, w.d, w.whiten, 1000)
    for e in sorted(range(256), key=lambda e: wls[e].n * wls[e].d)[:3]:
        assert m.line_of(e, wls[e]) == stored[e]
