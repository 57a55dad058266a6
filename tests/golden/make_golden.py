"""Write the oracle's expected outputs for the full-size parity tests.

Calls only ``oracle/`` (Algorithm 1, sp4, threshold 1000, FP64) on the seeded workloads of
``paper_2306_00271_gb300.workloads``; nothing here comes from the CUDA path.

    python tests/golden/make_golden.py            # writes tests/golden/trhepd_n61_sp4.npz
    python tests/golden/make_golden.py large      # writes tests/golden/large_n255_sp4_sampled.npz
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.curve import rocking_curve_parallel  # noqa: E402
from paper_2306_00271_gb300 import workloads as W  # noqa: E402


def main():
    wl = W.trhepd_n61()
    t = time.time()
    rho, eta, flux, n_rhst = rocking_curve_parallel(wl, "sp4", 1000.0)
    out = os.path.join(HERE, "trhepd_n61_sp4.npz")
    np.savez_compressed(out, theta0=wl.theta0, theta1=wl.theta1, rho=rho, eta=eta,
                        n_rhst=n_rhst, n_steps=wl.n_steps, z_e=wl.z_e)
    print(f"wrote {out} in {time.time() - t:.1f}s; rhst per angle {n_rhst.min()}..{n_rhst.max()}")


# sampled angles of the 255-beam recipe's first structure (of its 120 angles 0.2 .. 6.2 deg)
LARGE_ANGLES = (10, 40, 70, 100)


def large():
    """The 255-beam square-cell recipe (3000 slices of 0.01 A, sp4) of its first parameter set at
    LARGE_ANGLES."""
    wl = W.large_n255(1)[0]
    t = time.time()
    # two processes: the oracle expands U(tau) at every node, about 17 GB per process here
    rho, eta, flux, n_rhst = rocking_curve_parallel(wl, "sp4", 1000.0, angles=LARGE_ANGLES,
                                                    processes=2)
    out = os.path.join(HERE, "large_n255_sp4_sampled.npz")
    np.savez_compressed(out, angles=np.array(LARGE_ANGLES), theta0=wl.theta0[list(LARGE_ANGLES)],
                        theta1=wl.theta1[list(LARGE_ANGLES)], rho=rho, eta=eta, n_rhst=n_rhst,
                        n_steps=wl.n_steps, z_e=wl.z_e)
    print(f"wrote {out} in {time.time() - t:.1f}s; rhst per angle {n_rhst.min()}..{n_rhst.max()}")


if __name__ == "__main__":
    large() if sys.argv[1:] == ["large"] else main()
