"""Writes the small parity fixtures in this folder.

Inputs come from a seeded numpy generator; expected values come only from
the FP64 oracle (``oracle.rl_planes``).  Re-run after a change to the oracle
that a paper passage justifies:  python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [
    # name, boundary, V, P, H, W, K, iters, seed
    ("small_zero", "zero", 2, 2, 20, 13, 5, 3, 100),
    ("small_circular", "circular", 3, 1, 12, 17, 7, 2, 101),
]


def main():
    for name, boundary, V, P, H, W, K, iters, seed in CASES:
        rng = np.random.default_rng(seed)
        phi = rng.uniform(1.0, 200.0, size=(V, P, H, W)).astype(np.float32)
        psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
        psfs /= psfs.sum(axis=(1, 2), keepdims=True)
        psfs = psfs.astype(np.float32)
        out = oracle.rl_planes(phi.astype(np.float64), psfs.astype(np.float64), iters,
                               boundary=boundary, eps=1e-6)
        case = {
            "cite": "Supp. Note 1, multi-view RL update equation; expected values from the FP64 oracle",
            "boundary": boundary, "iters": iters, "eps": 1e-6,
            "phi": phi.tolist(), "psf": psfs.tolist(),
            "expected": out.tolist(),
        }
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(case, f)


if __name__ == "__main__":
    main()
