"""Surface tension gamma of the two-component Shan-Chen fluid at G = 3.6
(Sec. 3.2 parameters), measured with the FP64 oracle by Laplace's law on
cylinders of A in B: dp = gamma / R for R = 8, 11, 14 (periodic 1 x 48 x 48
slices, 4000 steps), bulk pressure p = c_s^2 (rho_A + rho_B) + c_s^2 G psi_A
psi_B.  gamma is the least-squares slope of dp against 1/R through the
origin.  The paper gives no value (reading c25); this script writes the one
the theory check uses: python tests/golden/make_gamma.py > tests/golden/gamma_G3.6.txt
Calls only the oracle."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle as O  # noqa: E402

CS2 = 1.0 / 3.0


def laplace_points(G=3.6, steps=4000, radii=(8.0, 11.0, 14.0), n=48):
    _, w, _ = O.tables()
    out = []
    for R in radii:
        o = O.Oracle(1, n, n, wall=0, G=G)
        y, z = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        r = np.sqrt((y - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.5) ** 2)
        inside = (r < R).T[:, :, None]  # [z, y, x]
        rA = np.where(inside, 0.7, 0.04)
        rB = np.where(inside, 0.04, 0.7)
        f = np.stack([w[:, None, None, None] * rA[None], w[:, None, None, None] * rB[None]])
        o.set_populations(f)
        o.step(steps)
        rho, _ = o.fields()
        psi = 1 - np.exp(-rho)
        p = CS2 * (rho[0] + rho[1]) + CS2 * G * psi[0] * psi[1]
        out.append((R, p[n // 2, n // 2, 0] - p[0, 0, 0]))
        o.close()
    return out


if __name__ == "__main__":
    pts = laplace_points()
    invR = np.array([1.0 / R for R, _ in pts])
    dp = np.array([d for _, d in pts])
    gamma = float(np.dot(invR, dp) / np.dot(invR, invR))
    for R, d in pts:
        print(f"# R = {R:g}: dp = {d:.10e}, dp R = {d * R:.10e}")
    print(f"{gamma:.10e}")
