"""Write the exact SAW counts used by the tests, from the oracle's enumerator only.

    python tests/golden/make_golden.py

Produces tests/golden/saw_counts_d2.txt (n <= 16) and saw_counts_d3.txt (n <= 11).
The enumerator itself is pinned by closed forms, an independent brute force and
the published leading terms (tests/test_oracle_pins.py).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402


def main():
    for d, nmax in ((2, 16), (3, 11)):
        c = oracle.enumerate_cn(d, nmax)
        path = os.path.join(HERE, "saw_counts_d%d.txt" % d)
        with open(path, "w") as f:
            f.write("# c_n, n = 0..%d, d = %d: exact counts of n-step self-avoiding walks\n" % (nmax, d))
            f.write("# written by tests/golden/make_golden.py from oracle.enumerate_cn\n")
            for n, v in enumerate(c):
                f.write("%d %d\n" % (n, int(v)))
        print(path)


if __name__ == "__main__":
    main()
