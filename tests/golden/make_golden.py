"""Writes the golden fixtures of tests/golden/ from closed forms only.

gaussian_plane_integrals.json: plane integrals of a sampled Gaussian blob,
A 2 pi sigma^2 exp(-(s - d.c)^2 / (2 sigma^2)) at the integer offsets
s = -M/2..M/2-1 of a few directions.  By the Fourier Slice Theorem (Sec. 2.2.1)
the radial inverse DFT of the blob's Fourier samples on a line through the
origin equals these values up to the blob's aliasing and truncation (below
1e-10 for sigma = 2 voxels in a 32^3 box).  Only oracle/ closed forms are used.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nufft3d_oracle as O  # noqa: E402


def main():
    n, m, sig = 32, 64, 2.0
    c = [0.5, 0.25, -1.0]
    dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8], [0.48, -0.6, 0.64],
                     [-0.36, 0.48, 0.8]], dtype=np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = np.arange(m) - m // 2
    vals = [O.gaussian_plane_integral(d, s, c, sig).tolist() for d in dirs]
    out = {
        "citation": "Fourier Slice Theorem (Sec. 2.2.1); Gaussian plane integral closed form",
        "n": n, "m": m, "sigma_vox": sig, "center_vox": c,
        "dirs": dirs.tolist(), "plane_integrals": vals,
    }
    with open(os.path.join(os.path.dirname(__file__), "gaussian_plane_integrals.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
