"""Time and memory of one differentiable dam-break run (forward with
checkpoints, backward by the hand-written adjoint with recomputation).
Prints one JSON line.  Test infrastructure: not collected by pytest.

    python tests/report_adjoint.py --dp 0.003 --steps 100 --every 20
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
    ap.add_argument("--dp", type=float, default=0.01)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--window", type=int, default=100)
    ap.add_argument("--dt", type=float, default=1e-4)
    args = ap.parse_args()
    import torch
    from sphcases import dam_break, wall_sensors
    from paper_1110_3711_gb300 import build
    build.build()
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    c = dam_break(args.dp, vel_sigma=0.05, seed=0, fixed_dt=args.dt)
    run = DamBreakRun(c, args.steps, args.dt, min(args.window, args.steps), wall_sensors(c),
                      checkpoint_every=args.every)
    v0 = torch.tensor(c.vel[:c.n_f], dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(c.params.alpha, dtype=torch.float64, device="cuda", requires_grad=True)
    torch.cuda.reset_peak_memory_stats()
    torch.cuda.synchronize()
    t0 = time.time()
    J = objective(v0, a, run)
    torch.cuda.synchronize()
    t1 = time.time()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.time()
    free, total = torch.cuda.mem_get_info()
    print(json.dumps({"dp": args.dp, "particles": c.n, "steps": args.steps, "every": args.every,
                      "J": float(J.detach()), "dJ_dalpha": float(a.grad),
                      "grad_v0_norm": float(v0.grad.norm()), "forward_s": t1 - t0,
                      "backward_s": t2 - t1, "peak_torch_gb": torch.cuda.max_memory_allocated() / 1e9,
                      "device_used_gb": (total - free) / 1e9,
                      "checkpoint_gb": run.stats["checkpoint_bytes"] / 1e9}), flush=True)


if __name__ == "__main__":
    main()
