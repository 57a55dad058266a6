"""Write the oracle's R-factor gradient for the full-size differentiation workload.

Calls only ``oracle/`` on the seeded fit problem of ``paper_2306_00271_gb300.workloads``
(N = 61 beams, 2000 slices, 60 angles; 12 free z coordinates and 6 Debye-Waller classes): the
target curve is O2's specular curve at the hidden true structure, and the gradient is O2's
central difference at the starting structure (h = 1e-5 A and 1e-5 A^2). Nothing here comes from
the CUDA path.

    python tests/golden/make_golden_grad.py       # writes tests/golden/rfactor_fit_n61.npz
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.gradient import fd_gradient, specular_curves  # noqa: E402
from paper_2306_00271_gb300 import workloads as W  # noqa: E402


def main():
    fp = W.rfactor_fit()
    t = time.time()
    target = specular_curves([W.fit_structure(fp, fp.z_true, fp.b_true)])[0]
    res = fd_gradient(fp.workload, fp.free_atoms, fp.dw_class, target)
    out = os.path.join(HERE, "rfactor_fit_n61.npz")
    np.savez_compressed(out, target=target, R=res["R"], eta1=res["eta1"], grad=res["grad"],
                        jac=res["jac"], hz=1e-5, hb=1e-5)
    print(f"wrote {out} in {time.time() - t:.1f}s; R = {res['R']:.6e}")


if __name__ == "__main__":
    main()
