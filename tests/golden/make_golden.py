"""Writes the stored expected values under tests/golden/ by running the CPU
oracle only (nothing here touches the CUDA path).

plain_pipe_24x24x96_wake.txt: longitudinal wake potential W(s) of Sec. 5,
W(s) = -(1/Q) * integral of E_z along the test-charge path, for the plain
rectangular PEC pipe 24 x 24 x 96 cells, dx = dy = sqrt(2) mm, dz = 1 mm,
c*dt = dz, vacuum, Gaussian bunch sigma = 4 mm, Q = 1 nC on the axis node
(12, 12), cold start, 400 steps of the explicit scheme (23).

Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from paper_0901_1053_gb300 import workloads as wl  # noqa: E402


def plain_pipe_wake():
    w = wl.plain_pipe()
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    o.step(w.steps)
    wk, s0, ds = o.wake()
    return wk, s0, ds, o.energy()


def main():
    wk, s0, ds, energy = plain_pipe_wake()
    path = os.path.join(HERE, "plain_pipe_24x24x96_wake.txt")
    with open(path, "w") as f:
        f.write("# Longitudinal wake W(s) [V/C] (Sec. 5 definition), FP64 CPU oracle of the\n")
        f.write("# explicit TE/TM scheme (Sec. 4.2, Eq. (23)); plain PEC pipe 24x24x96,\n")
        f.write("# dx=dy=sqrt(2) mm, dz=1 mm, c*dt=dz, sigma=4 mm, Q=1 nC on node (12,12), 400 steps.\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write("# s0_m %.17g ds_m %.17g field_energy_J %.17g\n" % (s0, ds, energy))
        for v in wk:
            f.write("%.17g\n" % v)
    print(path)


if __name__ == "__main__":
    main()
