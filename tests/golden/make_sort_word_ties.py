"""Writes sort_word_ties.txt: cells of the 128 x 128 x 256 grid (all 256 SDs
live, ranks 0..255) whose step-0 sort keys (seed 0) hold two keys with equal
top 24 bits, ordered against their ranks by the full keys, at sorted
positions 2l + 1 and 2l + 2 (so they sit in different pairs).  Only the
oracle's sort key is called.

    python tests/golden/make_sort_word_ties.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

SEED, STEP, N, CELLS = 0, 0, 256, 128 * 128


def tie_positions(cell):
    """Sorted positions p (odd) where keys at p and p + 1 share their top 24
    bits and the full keys order them against their ranks."""
    keys = [O.sort_key(SEED, r, cell, STEP) for r in range(N)]
    order = sorted(range(N), key=lambda r: (keys[r], r))
    out = []
    for p in range(N - 1):
        a, b = order[p], order[p + 1]
        if keys[a] >> 40 == keys[b] >> 40 and a > b and p % 2 == 1:
            out.append(p)
    return out


def main():
    O.build()
    rows = []
    for c in range(CELLS):
        for p in tie_positions(c):
            rows.append((c, p))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sort_word_ties.txt")
    with open(path, "w") as f:
        f.write("# cell sorted_position: 24-bit key ties ordered against rank, across a pair boundary\n")
        f.write(f"# seed {SEED} step {STEP} sd_per_cell {N} cells {CELLS}; written by make_sort_word_ties.py\n")
        for c, p in rows:
            f.write(f"{c} {p}\n")
    print(len(rows), "rows")


if __name__ == "__main__":
    main()
