"""Writes the stored fixtures under tests/golden/ from the CPU oracle alone.

    python tests/golden/make_golden.py

reps_n16384_nr128_seed2.txt : oracle.sample_reps(16384, 128, seed=2), the
    representative set of the 16384-point, 128-representative workload
    (Section 4 sampling, fixed-size reading with SplitMix64).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    r = oracle.sample_reps(16384, 128, 2)
    with open(os.path.join(HERE, "reps_n16384_nr128_seed2.txt"), "w") as f:
        f.write("# oracle.sample_reps(16384, 128, seed=2); SplitMix64 + partial Fisher-Yates (Section 4)\n")
        for v in r:
            f.write(f"{int(v)}\n")


if __name__ == "__main__":
    main()
