"""The seeded input generator: shapes, dtypes, determinism and recipe."""

import numpy as np

from paper_1503_07998_gb300 import synth


def test_plane_case_default_recipe():
    c = synth.plane_case(seed=0)
    assert c.phi.shape == (2, 1, 128, 128) and c.phi.dtype == np.float32
    assert c.psfs.shape == (2, 17, 17)
    assert c.truth.min() >= 10.0
    d = synth.plane_case(seed=0)
    np.testing.assert_array_equal(c.phi, d.phi)
    # the second view is the first one turned by 90 degrees
    np.testing.assert_allclose(c.psfs[1], c.psfs[0].T, rtol=1e-7)


def test_volume_stacks_small_cpu():
    stacks, psfs = synth.volume_stacks(12, 10, 16, 7, 3.0, 1.2, (0, 90), 2e-2, seed=3)
    assert tuple(stacks.shape) == (2, 12, 10, 16)
    assert str(stacks.dtype) == "torch.uint16"
    assert psfs.shape == (2, 7, 7)
    s2, _ = synth.volume_stacks(12, 10, 16, 7, 3.0, 1.2, (0, 90), 2e-2, seed=3)
    assert bool((stacks.int() == s2.int()).all())
    assert int(stacks.int().min()) >= 0


def test_uneven_volumes_subsets_match_the_full_list():
    """A rank that builds only its own volumes gets exactly those of the full
    list (each volume depends on seed + i alone)."""
    full = synth.uneven_volumes(5, seed=3, side=(16, 24), planes=(2, 3), views=(2, 3), psf=(3, 5), iters=(1, 2))
    part = synth.uneven_volumes(5, seed=3, side=(16, 24), planes=(2, 3), views=(2, 3), psf=(3, 5), iters=(1, 2),
                                only=[1, 4])
    shapes = synth.uneven_volumes(5, seed=3, side=(16, 24), planes=(2, 3), views=(2, 3), psf=(3, 5), iters=(1, 2),
                                  shapes_only=True)
    assert len(part) == 2 and len(shapes) == 5
    for a, b in zip(part, [full[1], full[4]]):
        np.testing.assert_array_equal(np.asarray(a["stacks"]), np.asarray(b["stacks"]))
        np.testing.assert_array_equal(a["psfs"], b["psfs"])
    for a, b in zip(shapes, full):
        assert a["stacks"] is None and all(a[k] == b[k] for k in ("H", "W", "P", "views", "K", "iters"))
