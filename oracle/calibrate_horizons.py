"""Pick each synthetic workload's time horizon T so that the mean number of
events per trajectory is close to the workload's target, by running the
oracle on a few replicas (T <- T * target / mean_events, three rounds).

Writes paper_1010_2438_gb300/workload_horizons.json, which the input
generators read.  The horizon is an input of both the oracle and the CUDA
path; it is not an expected value of any test.

    python -m oracle.calibrate_horizons
"""
import json
import os

import numpy as np

import oracle
from paper_1010_2438_gb300 import workloads as W

TARGETS = {  # workload -> (constructor, target mean events, replicas used)
    "flat8x12": (W.flat8x12, 1e4, 16),
    "flat32x64": (W.flat32x64, 1e5, 8),
    "flat16x24": (W.flat16x24, 1e4, 16),
    "cwc3x24": (W.cwc3x24, 1e4, 16),
}


def calibrate(name, ctor, target, reps, rounds=3):
    b = ctor(R=reps, use_calibrated=False)
    T = float(b.grid[-1])
    for _ in range(rounds):
        bb = W.Batch(b.model, b.rates, b.init, W.uniform_grid(T, 2), reps, b.seed)
        ev = oracle.simulate(bb, states=False, threads=os.cpu_count() or 1)["events"]
        T = T * target / float(np.mean(ev))
    return T


def main():
    out = {}
    for name, (ctor, target, reps) in TARGETS.items():
        out[name] = calibrate(name, ctor, target, reps)
        print(name, out[name])
    with open(W.HORIZONS_PATH, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
