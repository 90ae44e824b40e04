"""Writes batched_256_accepted.txt: the FP64 oracle's accepted pool of every experiment of
the 256-experiment batched workload (n log-uniform on [50, 2000], n1 = n // 2, d uniform on
{10..500}, 1e5 Philox draws from draw 0, q = 0.01, so K = 1000 per experiment).

The accepted set is the K draws with the smallest (M, draw index) (Sec. 2.2, "Choosing
stringency"). Each experiment's line records the set by a SHA-256 of its keys (ascending
draw index, little-endian uint64), the smallest and largest key, the sum of the keys and the
largest accepted M, so the GPU test can compare the whole set without storing it.

Only the oracle and the seeded input generators are used. Run from the repository root:

    python tests/golden/make_batched_golden.py            # all 256 experiments
    python tests/golden/make_batched_golden.py --check 3  # re-derive the 3 cheapest lines

It takes about four minutes on 16 host cores (the oracle scores 2.8e12 multiply-adds).
"""
from __future__ import annotations

import argparse
import hashlib
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_2501_07642_b300.workloads import batched_workloads  # noqa: E402

OUT = Path(__file__).resolve().parent / "batched_256_accepted.txt"
HEADER = "# e n d whiten K sha256(keys,<u8) min_key max_key sum_keys max_M64"


def keys_digest(keys: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(keys, dtype="<u8").tobytes()).hexdigest()


def line_of(e: int, w) -> str:
    X = w.covariates()
    Zc, *_ = O.prep(X, w.whiten, w.ridge)
    keys, m64 = O.select(Zc, w.n1, w.philox_seed, 0, w.draws, q=w.q)
    return (f"{e} {w.n} {w.d} {w.whiten} {len(keys)} {keys_digest(keys)} {int(keys.min())} {int(keys.max())} "
            f"{int(keys.astype(np.uint64).sum())} {float(m64.max()):.17g}")


def read_lines() -> dict[int, str]:
    out = {}
    for ln in OUT.read_text().splitlines():
        if ln and not ln.startswith("#"):
            out[int(ln.split()[0])] = ln
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", type=int, default=0, help="re-derive the N cheapest experiments and compare")
    args = ap.parse_args()
    wls = batched_workloads(256)
    if args.check:
        stored = read_lines()
        cheapest = sorted(range(256), key=lambda e: wls[e].n * wls[e].d)[: args.check]
        for e in cheapest:
            got = line_of(e, wls[e])
            if got != stored[e]:
                raise SystemExit(f"experiment {e}: stored\n  {stored[e]}\nre-derived\n  {got}")
        print(f"{len(cheapest)} lines re-derived identically")
        return
    lines = [HEADER]
    for e, w in enumerate(wls):
        lines.append(line_of(e, w))
        print(lines[-1], flush=True)
    OUT.write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
