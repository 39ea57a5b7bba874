"""Write the stored oracle results used by the GPU parity tests.

Calls only oracle/ (and the seeded input generators).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2111_11538_gb300 import inputs, workloads  # noqa: E402


def coreshell64():
    """64 x 64 core-shell, FP64, elastic, CG rtol 1e-10, 500 steps."""
    wl = workloads.WORKLOADS["coreshell64"]
    f = workloads.build_fields("coreshell64")
    s = oracle.Sim(f, wl["params"])
    iters = []
    for _ in range(wl["steps"]):
        iters.append(s.step(1))
    sums = s.sums()
    np.savez_compressed(os.path.join(HERE, "coreshell64_fp64_500.npz"),
                        phi_f=s.phi_f, phi_w=s.phi_w, xO=s.f["xO"], xH=s.f["xH"], xW=s.f["xW"],
                        sigma=s.f["sigma"], u=s.f["u"], Ebar=s.f["Ebar"],
                        removedW=s.removedW, suppliedH=s.suppliedH, sums=sums,
                        cg_iters=np.array(iters), dt=s.dt)


if __name__ == "__main__":
    coreshell64()
