"""Writes config1_map.txt: the FP64 oracle's map of config 1 (Algorithm 5;
4 sites x 3 channels, 16x16 scans), the reference the benchmark's precision
report compares every GPU precision with.  Calls only oracle/ and synth/.

    python tests/golden/make_config1_map.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import bip as obip  # noqa: E402


def main():
    sp = synth.make_specimen(synth.config1())
    m = obip.bip_map(obip.make_problem(sp)).map
    path = os.path.join(HERE, "config1_map.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle map of config 1 (Algorithm 5), scans in raster order, written by make_config1_map.py\n")
        for v in m:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
