"""Write c1a_oracle_samples.npz: sampled FP64 oracle iterates of full-size C1a solves.

For images 0 and 1 of the 8 x RGB 256^2 motion-blur workload (C1a), runs the
oracle's inertial iteration from x0 = A^T y without a stopping test for K_MAX
updates and records, for every update k in [K_LO, K_MAX], the values of x^k at a
fixed seeded set of 512 pixel positions, the relative step ||x^k - x^{k-1}|| /
||x^{k-1}|| and the PSNR of x^k.  Without restarts the trajectory up to the
stopping update is the one the stopping test would give, so `stop` (the first k
whose relative step is below tol) is the oracle's iteration count.  The GPU
parity test compares its full-size solve, element by element on the sampled
positions, with the oracle iterate at the GPU's own iteration count.  Calls only
oracle/ and synth/.

usage: python tests/golden/oracle_c1a_samples.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import nets, operators, solver  # noqa: E402
from synth import get_config, workload  # noqa: E402

N_IMG, K_LO, K_MAX, N_SAMPLES = 2, 30, 50, 512


def main():
    cfg = get_config("C1a", n=N_IMG)
    wl = workload(cfg)
    net = nets.Net.from_config(cfg["net"], cfg["c"], wl["weights"])
    ops = operators.make_operators(cfg, wl)
    ys = operators.observe(ops, wl["x_true"], wl["noise"]).astype(np.float32).astype(np.float64)
    per = cfg["c"] * cfg["h"] * cfg["w"]
    idx = np.sort(np.random.default_rng(12345).choice(per, N_SAMPLES, replace=False))
    nk = K_MAX - K_LO + 1
    samples = np.zeros((N_IMG, nk, N_SAMPLES), np.float64)
    rel = np.zeros((N_IMG, nk))
    psnr = np.zeros((N_IMG, nk))
    stop = np.zeros(N_IMG, np.int64)
    for i in range(N_IMG):
        first = [0]

        def rec(k, x, r, i=i, first=first):
            if r < cfg["tol"] and first[0] == 0:
                first[0] = k
            if k >= K_LO:
                samples[i, k - K_LO] = x.ravel()[idx]
                rel[i, k - K_LO] = r
                psnr[i, k - K_LO] = solver.psnr(x, wl["x_true"][i])
                print(i, k, r, psnr[i, k - K_LO], flush=True)

        x0 = ops[i].AT(ys[i])
        solver.solve_image(net, ops[i], ys[i], x0, cfg["lam"], cfg["tau"], cfg["beta"],
                           cfg["B"], 0.0, K_MAX, on_update=rec)
        stop[i] = first[0]
    np.savez_compressed(os.path.join(HERE, "c1a_oracle_samples.npz"), idx=idx,
                        k=np.arange(K_LO, K_MAX + 1), samples=samples, rel=rel, psnr=psnr,
                        stop=stop, tol=cfg["tol"])


if __name__ == "__main__":
    main()
