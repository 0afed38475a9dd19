"""Error of each field of the FP32 split-precision run against the FP64 oracle.

Runs the dam break at a given dp for a number of steps on the GPU
(SPH_FP32_SPLIT and SPH_FP64) and with the oracle on the host cores from the
same initial state, then prints one JSON line with the max and RMS error of
position (in units of dp), velocity (relative to max|v| + g t) and density
(relative), for both GPU forms.  Test infrastructure: not collected by pytest.

    python tests/report_split_precision.py --dp 0.0025 --steps 200
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
    from sphcases import dam_break
    from oracle import oracle as O
    from paper_1110_3711_gb300 import build
    build.build()
    from paper_1110_3711_gb300.sph import Simulation
    c = dam_break(args.dp)
    t0 = time.time()
    st = O.State(c)
    st.run(args.steps, nthreads=os.cpu_count() or 1)
    t_oracle = time.time() - t0
    vscale = np.abs(st.vel).max() + 9.81 * st.time
    out = {"dp": args.dp, "particles": c.n, "steps": args.steps, "sim_time_s": st.time,
           "oracle_s": t_oracle, "out_of_grid": st.n_out}
    for prec in ("fp32", "fp64"):
        sim = Simulation.from_case(c, precision=prec)
        sim.run(args.steps)
        pos, vel, rho = sim.get_state()
        ex = np.abs(pos - st.pos) / c.params.dp
        ev = np.abs(vel - st.vel) / vscale
        er = np.abs(rho / st.rho - 1.0)
        out[prec] = {"x_max_dp": float(ex.max()), "x_rms_dp": float(np.sqrt((ex ** 2).mean())),
                     "v_max_rel": float(ev.max()), "v_rms_rel": float(np.sqrt((ev ** 2).mean())),
                     "rho_max_rel": float(er.max()), "rho_rms_rel": float(np.sqrt((er ** 2).mean())),
                     "sim_time_s": sim.time()[0], "status": sim.status()}
        sim.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
