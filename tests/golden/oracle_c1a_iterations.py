"""Write c1a_oracle_iters.json: FP64 oracle solves of C1a images at full size.

For the first images of the 8 x RGB 256^2 motion-blur workload (C1a), runs the
oracle's inertial iteration from x0 = A^T y to ||x^{k+1}-x^k|| < 1e-4 ||x^k|| and
records the iteration count, the seconds per iteration on this host and the
PSNR.  The benchmark's CPU-baseline legs extrapolate the oracle's per-iteration
time to restorations/s with these counts.  Calls only oracle/ and synth/.

usage: python tests/golden/oracle_c1a_iterations.py [n_images]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import nets, operators, solver  # noqa: E402
from synth import get_config, workload  # noqa: E402


def main(n_img=1):
    cfg = get_config("C1a")
    wl = workload(cfg)
    net = nets.Net.from_config(cfg["net"], cfg["c"], wl["weights"])
    ops = operators.make_operators(cfg, wl)
    ys = operators.observe(ops, wl["x_true"], wl["noise"]).astype(np.float32).astype(np.float64)
    out = {"config": "C1a", "tol": cfg["tol"], "images": []}
    for i in range(n_img):
        x0 = ops[i].AT(ys[i])
        t0 = time.time()
        x, info = solver.solve_image(net, ops[i], ys[i], x0, cfg["lam"], cfg["tau"], cfg["beta"],
                                     cfg["B"], cfg["tol"], cfg["max_iter"])
        dt = time.time() - t0
        out["images"].append({"index": i, "iters": info["iters"], "status": info["status"],
                              "restarts": info["restarts"], "sec_per_iter": dt / info["iters"],
                              "psnr": solver.psnr(x, wl["x_true"][i])})
        print(out["images"][-1], flush=True)
    out["host_cores"] = os.cpu_count()
    with open(os.path.join(HERE, "c1a_oracle_iters.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1)
