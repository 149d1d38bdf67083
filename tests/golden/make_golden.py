"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Calls only ``oracle`` (and the seeded input layout); nothing here comes from
the CUDA path.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2404_04994_gb300 import inputs  # noqa: E402


def main():
    g = json.load(open(os.path.join(HERE, "paper_examples.json")))["example_model"]
    ras = inputs.raster(2, 0, 1, np.zeros(2), lo=g["lo"], hi=g["hi"],
                        W=g["pixels"], H=g["pixels"])
    out = oracle.ground_state(np.array(g["cdd"]), np.array(g["cgd"]), raster=ras)
    np.savetxt(os.path.join(HERE, "example_model_open_map.txt"),
               out["n"][:, :2].reshape(100, 200), fmt="%d")


if __name__ == "__main__":
    main()
