"""The random-gather ceiling of the current GPU for the access patterns of the solver's two
sparse products, measured with pdlp_gather_bench (a synthetic SELL-32 product, one gather
per entry) for each gather method and pattern.  Usage:

    python -m paper_2501_07018_gb300.gather_ceiling [--nnz N]

Prints one line per case: method, element size, gathered-vector length, entries per row,
column pattern, microseconds per launch and gathered entries per second.
"""
from __future__ import annotations

import argparse
import json

from . import binding

# (method, element bytes, vector length, entries per row, degree exponent (0 = uniform))
CASES = [
    ("lsu", 8, 2_000_000, 24, 0.0), ("lsu", 8, 2_000_000, 10, 0.0), ("lsu", 8, 2_000_000, 8, 0.0),
    ("lsu", 8, 5_000_000, 24, 0.0), ("lsu", 8, 5_000_000, 25, 2.08),
    ("lsu", 4, 2_000_000, 10, 0.0), ("lsu", 4, 5_000_000, 25, 2.08),
    ("tma", 8, 2_000_000, 24, 0.0), ("tma", 8, 2_000_000, 8, 0.0), ("tma", 8, 5_000_000, 24, 2.08),
    ("hybrid", 8, 2_000_000, 24, 0.0), ("hybrid", 8, 5_000_000, 24, 2.08),
]


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nnz", type=int, default=50_000_000)
    ap.add_argument("--json", action="store_true", help="one JSON object per line")
    args = ap.parse_args()
    for method, eb, table, row_len, deg in CASES:
        r = binding.gather_bench(method, eb, table, row_len, args.nnz, deg, reps=10)
        pattern = f"power-law degrees s={deg}" if deg > 0 else "uniform"
        if args.json:
            print(json.dumps(dict(method=method, elem_bytes=eb, table_len=table, row_len=row_len,
                                  pattern=pattern, **r)))
        else:
            print(f"{method:6s} {eb}B  vector {table:>9d}  row {row_len:2d}  {pattern:24s}"
                  f" {r['us']:8.1f} us  {r['entries_per_s'] / 1e9:6.1f} G entries/s"
                  f"  |y - y_lsu| {r['max_diff_vs_lsu']:.1e}", flush=True)


if __name__ == "__main__":
    main()
