"""Write tests/golden/adjoint_channel_512_fd.json: FP64 central finite
differences of the outlet flux with respect to eps at 32 random cells of the
512x512 adjoint channel workload (2000 steps from rest), from the oracle only.

J(eps) = sum over the plane x = 511 of eps*rho*u_x (Eq. 1moment) after 2000
steps; dJ/deps(c) ~ (J(eps + h e_c) - J(eps - h e_c)) / (2h), h = 1e-4, with the
perturbation applied in double precision to the float32 eps value of cell c.

  python tests/golden/make_adjoint_fd.py [--threads N]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1406_6438_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "adjoint_channel_512_fd.json"))
    args = ap.parse_args()
    if args.threads:
        O.set_num_threads(args.threads)
    p, eps32, nsteps, every = W.adjoint_channel()
    cells = W.fd_cells(eps32.shape, 32, seed=5)
    po = O.Params(**p)
    x_out = p["nx"] - 1
    h = 1e-4

    def J(e):
        f = O.run(po, e, O.init(po, e), nsteps)
        return O.flux(po, e, f, x_out)

    base = eps32.astype(np.float64)
    t0 = time.time()
    J0 = J(base)
    fd = []
    for k, c in enumerate(cells):
        ep = base.copy()
        ep[c] += h
        em = base.copy()
        em[c] -= h
        fd.append((J(ep) - J(em)) / (2 * h))
        print(f"{k + 1}/{len(cells)} cell {c}: {fd[-1]:.9e}  ({time.time() - t0:.0f} s)", flush=True)
    out = {
        "workload": "adjoint_channel(): D2Q9 512x512, walls y, eps smoothed noise seed 5 in "
                    "[0.4,1.0], tau 0.8, Ergun drag d_p 21.33, g_x 2e-5",
        "nsteps": nsteps, "x_out": x_out, "h": h, "J": J0,
        "cells_zyx": [list(c) for c in cells], "dJdeps_fd": fd,
        "writer": "tests/golden/make_adjoint_fd.py (FP64 oracle only)",
    }
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
