"""Tolerances of the GPU-vs-oracle comparisons.

FP32 results against the FP64 oracle on identical inputs:
  relative L2      ||g - o||_2 / ||o||_2                    <= 1e-4
  per pixel        |g - o| <= 1e-3 * max(|o|, tau)         with tau = 1e-3 * max|o|
The floor tau keeps pixels that the iterations drive towards zero from
turning a tiny absolute error into a huge relative one; the unfloored
maximum is returned as well.
"""

import numpy as np

REL_L2 = 1e-4
PIX = 1e-3


def metrics(got, ref):
    g = np.asarray(got, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    rel_l2 = float(np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300))
    tau = 1e-3 * float(np.max(np.abs(o))) if o.size else 0.0
    pix = np.abs(g - o) / np.maximum(np.abs(o), max(tau, 1e-300))
    raw = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
    return rel_l2, float(pix.max()) if o.size else 0.0, float(raw.max()) if o.size else 0.0


def assert_parity(got, ref, rel_l2=REL_L2, pix=PIX, what=""):
    r, p, raw = metrics(got, ref)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    assert r <= rel_l2, f"{what}: rel-L2 {r:.3e} > {rel_l2:.0e} (per-pixel {p:.3e}, raw {raw:.3e})"
    assert p <= pix, f"{what}: per-pixel {p:.3e} > {pix:.0e} (rel-L2 {r:.3e}, raw {raw:.3e})"
    return r, p, raw
