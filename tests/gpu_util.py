"""Helpers shared by the GPU tests: run the same lattice on the GPU (through
the C ABI) and on the oracle, and compare."""
import numpy as np

OBS_FIELDS = ("bond_sum", "mag", "nclusters", "nbonds", "spans_x", "spans_y", "threshold")


def assert_obs_equal(got, ref, fields=OBS_FIELDS):
    assert len(got) == len(ref), (len(got), len(ref))
    for f in fields:
        np.testing.assert_array_equal(np.asarray(got[f]), np.asarray(ref[f]), err_msg=f)
