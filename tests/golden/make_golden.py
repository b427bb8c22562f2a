"""Write the golden regression values of the oracle.

Calls only the oracle and the seeded input generators.  The values are the
oracle's own real-space pad update (Sec. 1, Eq. 1; Sec. 3.2, Eqs. 37-38) for
the tiny isotropic ring workload (N_I = 200, N_P = 300, L = 16, mu = 1,
nu = 0.3, seed 0) at 64 seeded pad atoms, with Richardson's (n, N) = (4, 6)
(Sec. 3.1, Eq. 36).  They guard the oracle against drift between hosts; they
are not the paper's numbers (the paper prints none for this quantity).

    python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2105_08798_gb300 import inputs  # noqa: E402


def main():
    w = inputs.WORKLOADS["ring200x300_L16_iso"]
    xy_i, xy_p = w.geometry()
    f = w.forces()
    rng = np.random.Generator(np.random.PCG64(12345))
    samples = np.stack([rng.integers(0, w.n_p, 64), rng.integers(0, w.L, 64)], axis=1)
    u = oracle.pad_update(xy_i, xy_p, w.L, w.c, w.material, f, samples=samples, n=4, N=6)
    out = {
        "workload": w.name,
        "what": "oracle pad update G f (neutral-projected forces) at sampled (pad column, repeat) pairs",
        "rich_n": 4,
        "rich_N": 6,
        "samples": samples.tolist(),
        "u": [[float("%.17g" % x) for x in row] for row in u[0]],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ring200x300_L16_iso_samples.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
