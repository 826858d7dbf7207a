"""Writes the oracle regression fixtures of this folder (calls only oracle/ and tat_inputs/).

oracle_n16_forward.txt : A f, n=16, n_det=32, n_t=24, support radius 0.9, phantom seed 11
oracle_n16_adjoint.txt : A* g for g = random_sinogram(32, 24, seed 12), same plan
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tat_oracle as O  # noqa: E402
from tat_inputs import ellipse_phantom, random_sinogram  # noqa: E402

if __name__ == "__main__":
    P = O.OraclePlan(16, 32, 24, support_radius=0.9)
    np.savetxt(os.path.join(HERE, "oracle_n16_forward.txt"), O.forward(P, ellipse_phantom(16, 11)), fmt="%.17e")
    np.savetxt(os.path.join(HERE, "oracle_n16_adjoint.txt"), O.adjoint(P, random_sinogram(32, 24, 12)), fmt="%.17e")
