"""Seeded synthetic inputs for tensorial template matching.

This module only *makes inputs*: rotation sets, blob templates, binary ball
masks and tomograms with planted copies plus Gaussian noise.  It contains none
of the matching method's arithmetic (no normalisation, no correlation, no
tensor algebra), so that both the FP64 oracle and the CUDA path can be fed the
same seeded data without sharing any code of the method.

The paper has no dataset; these volumes stand in for cryo-electron tomograms
(the application named in Sec. 1 and Sec. 5 of the paper).
"""

from .volumes import (  # noqa: F401
    BATCH_CONFIGS,
    CONFIGS,
    BatchWorkload,
    Workload,
    ball_mask,
    batch_workload,
    blob_template,
    config_workload,
    default_mask_radius,
    make_batch,
    make_workload,
    plant_copies,
    shoemake_quaternions,
    soft_ball_mask,
    super_fibonacci_quaternions,
)
