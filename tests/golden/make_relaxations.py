"""Write tests/golden/relaxations.txt: the oracle's counts on the benchmark
graphs (sequential Dijkstra from source 0): reached vertices, reached arcs
and successful relaxations U, i.e. arcs that strictly lowered a tentative
distance.  The benchmark's algorithmic bytes are 8(n+1) + 8m + 8n + 16 U
(row pointers, column and weight arrays, the distance write, one heap word
written and read per successful relaxation).  Calls only oracle/ and gen/.

    python tests/golden/make_relaxations.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = [
    ("banded_n2e20", lambda: gen.banded(1 << 20, 64, 512, 1, 65535, 1)),
    ("banded_n2e19", lambda: gen.banded(1 << 19, 64, 512, 1, 65535, 1)),
    ("banded_n2e18", lambda: gen.banded(1 << 18, 64, 512, 1, 65535, 1)),
    ("grid64", lambda: gen.grid(64, 64, 1, 100, 0)),
]


def main():
    lines = ["# name n m reached reached_arcs successful_relaxations (oracle Dijkstra from source 0;",
             "# written by tests/golden/make_relaxations.py)"]
    for name, make in WORKLOADS:
        g = make()
        d, settled, scanned, U = oracle.dijkstra_counts(g, 0)
        lines.append(f"{name} {g.n} {g.m} {settled} {scanned} {U}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "relaxations.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
