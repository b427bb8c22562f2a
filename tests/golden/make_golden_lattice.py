"""Write the golden regression values of the oracle's lattice Green function.

Calls only the oracle.  The values are the zone-grid lattice Green function (App.) of the synthetic
spring model (central springs k1 = 1 to the |n|_1 = 1 neighbours and k2 = 0.4 to the |n|_1 = 2 ones,
plane spacing c = 1) in the modes of the line-periodic lattice with L = 16, on a 64 x 64 zone
grid, at a few in-plane differences, in the six-real layout [Re g11, Re g12, Re g22, Re g33,
Im g13, Im g23].  They guard the oracle against drift between hosts; they are not the paper's
numbers (the paper prints none for this model).

    python tests/golden/make_golden_lattice.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import harmonic  # noqa: E402

D_LIST = [(0, 0), (1, 0), (0, 1), (1, 1), (2, -1), (3, 2), (-4, 1), (5, 0)]
K_LIST = [0, 1, 2, 5, 8]


def main():
    K = harmonic.spring_blocks(1.0, 0.4, 1.0)
    g = harmonic.lattice_mode_table(K, 16, D_LIST, K_LIST, 64)
    six = np.stack([g[..., 0, 0].real, g[..., 0, 1].real, g[..., 1, 1].real, g[..., 2, 2].real,
                    g[..., 0, 2].imag, g[..., 1, 2].imag], axis=-1)
    out = {
        "what": "zone-grid lattice Green function of the spring model, six-real layout",
        "k1": 1.0, "k2": 0.4, "c": 1.0, "L": 16, "n_zone": 64,
        "d": D_LIST, "k": K_LIST,
        "g": [[[float("%.17g" % x) for x in row] for row in blk] for blk in six],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spring_lattice_modes_L16_n64.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
