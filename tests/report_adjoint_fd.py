"""Central differences of the differentiable dam break against its adjoint.

Configuration: dp = 0.01 dam break (80,400 fluid + 58,606 boundary), seeded
N(0, 0.05 m/s) initial velocity, fixed dt = 1e-4 s, 400 steps, mean over the
last 100 states; objective the wall pressure (64 sensors behind the column)
or the front position (tau = dp).  For each objective, prints one JSON line
with, for every eps:
  * 8 seeded random unit directions d of the initial velocities (N(0, 1) per
    component, normalised): the central difference (J(v0 + eps d) -
    J(v0 - eps d)) / (2 eps) against the adjoint's g . d, as the error relative
    to |g . d| and relative to |g|;
  * the 16 components of largest |g|, as the error relative to |g_k|;
  * alpha, as the error relative to |dJ/dalpha|.
Test infrastructure: not collected by pytest.

    python tests/report_adjoint_fd.py --eps 1e-3 1e-4 1e-5
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

STEPS, DT, WINDOW = 400, 1e-4, 100


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, nargs="+", default=[1e-3, 1e-4, 1e-5])
    ap.add_argument("--dirs", type=int, default=8)
    ap.add_argument("--comps", type=int, default=16)
    ap.add_argument("--objective", choices=["wall", "front", "both"], default="both")
    args = ap.parse_args()
    import torch
    from sphcases import dam_break, wall_sensors
    from paper_1110_3711_gb300 import build
    build.build()
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    c = dam_break(0.01, vel_sigma=0.05, seed=0, fixed_dt=DT)
    v0 = c.vel[:c.n_f].copy()
    objs = ["wall", "front"] if args.objective == "both" else [args.objective]
    for name in objs:
        kw = ({"sensors": wall_sensors(c, wall="back")} if name == "wall"
              else {"front_tau": c.params.dp})

        def run_j(v, al):
            r = DamBreakRun(c, STEPS, DT, WINDOW, checkpoint_every=STEPS, **kw)
            return float(r.forward(torch.tensor(v, dtype=torch.float64, device="cuda"), al))

        run = DamBreakRun(c, STEPS, DT, WINDOW, checkpoint_every=20, **kw)
        vt = torch.tensor(v0, dtype=torch.float64, device="cuda", requires_grad=True)
        at = torch.tensor(0.1, dtype=torch.float64, device="cuda", requires_grad=True)
        J = objective(vt, at, run)
        J.backward()
        g, ga = vt.grad.cpu().numpy(), float(at.grad)
        gn = float(np.linalg.norm(g))
        out = {"objective": name, "J": float(J.detach()), "grad_norm": gn, "dJ_dalpha": ga,
               "eps": {}}
        flat = np.argsort(-np.abs(g).ravel())[:args.comps]
        for eps in args.eps:
            rec = {"dirs": [], "comps": []}
            for s in range(args.dirs):
                d = np.random.default_rng(1000 + s).normal(size=v0.shape)
                d /= np.linalg.norm(d)
                fd = (run_j(v0 + eps * d, 0.1) - run_j(v0 - eps * d, 0.1)) / (2 * eps)
                gd = float((g * d).sum())
                rec["dirs"].append({"g_dot_d": gd, "fd": fd, "rel": abs(fd - gd) / abs(gd),
                                    "rel_to_norm": abs(fd - gd) / gn})
            for k in flat:
                d = np.zeros(v0.size)
                d[k] = 1.0
                d = d.reshape(v0.shape)
                fd = (run_j(v0 + eps * d, 0.1) - run_j(v0 - eps * d, 0.1)) / (2 * eps)
                gk = float(g.ravel()[k])
                rec["comps"].append({"k": int(k), "g": gk, "fd": fd, "rel": abs(fd - gk) / abs(gk)})
            fda = (run_j(v0, 0.1 + eps) - run_j(v0, 0.1 - eps)) / (2 * eps)
            rec["alpha"] = {"fd": fda, "rel": abs(fda - ga) / abs(ga)}
            rec["dirs_rel_max"] = max(r["rel"] for r in rec["dirs"])
            rec["dirs_rel_to_norm_max"] = max(r["rel_to_norm"] for r in rec["dirs"])
            rec["comps_rel_max"] = max(r["rel"] for r in rec["comps"])
            out["eps"][repr(eps)] = rec
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
