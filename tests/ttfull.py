"""Test helper: the full tensor of a device train, contracted on the host from its
cores (eq. z_tt) for comparisons with the oracle."""
import numpy as np


def full(t):
    z1, z2, z3 = t.cores()
    return np.einsum("ia,ajb,bk->ijk", z1, z2, z3)
