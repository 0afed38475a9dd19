"""Error of each field of the FP32 split-precision run against the FP64 oracle.

Runs the dam break at a given dp for a number of steps on the GPU
(SPH_FP32_SPLIT and SPH_FP64) and with the oracle on the host cores from the
same initial state, then prints one JSON line with the max and RMS error of
position (in units of dp), velocity (relative to max|v| + g t) and density
(relative), for both GPU forms.  Test infrastructure: not collected by pytest.

    python tests/report_split_precision.py --dp 0.0025 --steps 200

The same comparison, with its bars asserted, is the gpu test
tests/test_gpu_northstar.py::test_split_precision_5m_200_steps.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dp", type=float, default=0.0025)
    ap.add_argument("--steps", type=int, default=200)
    args = ap.parse_args()
    from paper_1110_3711_gb300 import build
    build.build()
    from tests.test_gpu_northstar import split_precision_errors
    t0 = time.time()
    out = split_precision_errors(args.dp, args.steps)
    out["wall_s"] = time.time() - t0
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
