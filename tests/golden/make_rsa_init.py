"""Write the seeded random-sequential-addition start of the 1024-pentagon system.

Calls only the oracle (oracle/): regular pentagons of circumradius 0.5 in a
square periodic box at area fraction 0.50, placed one at a time at uniform
random positions and orientations (Philox stream keyed by seed 42), each
kept only if it overlaps none placed before.  Output: one line per particle,
``x y c s`` as float.hex() so the values round-trip exactly.

Run from the repository root:  python tests/golden/make_rsa_init.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as orc  # noqa: E402

N, PHI, SEED = 1024, 0.50, 42


def main():
    # pentagon of circumradius 0.5, counter-clockwise, first vertex on +y
    k = np.arange(5)
    th = 0.5 * np.pi + 2.0 * np.pi * k / 5
    v = np.stack([0.5 * np.cos(th), 0.5 * np.sin(th)], axis=1)
    area = 0.5 * float(np.sum(v[:, 0] * np.roll(v[:, 1], -1) - np.roll(v[:, 0], -1) * v[:, 1]))
    L = (N * area / PHI) ** 0.5
    sysm = orc.OracleSystem(2, [L, L], v)
    pos, ori, used = sysm.rsa_2d(N, SEED, 100_000_000)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rsa_pentagons_N1024_phi050_seed42.txt")
    with open(out, "w") as f:
        f.write(f"# RSA start: N={N} regular pentagons R=0.5, phi={PHI}, L={L.hex()}, seed={SEED}, "
                f"attempts={used}\n")
        f.write("# written by tests/golden/make_rsa_init.py with the oracle's or_rsa_2d (random sequential "
                "addition; overlaps by the contract test of Sec. 2.3); columns x y cos sin as float.hex()\n")
        for i in range(N):
            f.write(" ".join(float(t).hex() for t in (pos[i, 0], pos[i, 1], ori[i, 0], ori[i, 1])) + "\n")
    print(out, used)


if __name__ == "__main__":
    main()
