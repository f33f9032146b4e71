"""Seeded synthetic 0-1 ILP instances.

This module only draws inputs: integer constraint matrices in CSR form, right-hand
sides, senses and objective vectors.  It holds none of the method's arithmetic (no BDDs,
no messages, no bounds), so both the oracle and the CUDA library may read what it
produces.
"""
from .generators import (  # noqa: F401
    Instance,
    SENSE_LE,
    SENSE_EQ,
    SENSE_GE,
    potts_mrf,
    potts_grid_2label,
    sparse_matching,
    tomography,
    tracking,
    potts_batch,
    potts_batch_member,
    potts_batch_shape,
    random_ilp,
    config,
    CONFIG_NAMES,
    CONFIG_ITERS,
)
