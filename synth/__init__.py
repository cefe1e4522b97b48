"""Seeded synthetic inputs for the Gaussian Photon Field radiance query.

This module only draws random numbers and traces camera rays against an
analytic floor-plus-sphere scene. It holds none of the radiance method's
arithmetic (no Gaussian weight, falloff, normalisation or gradient), so both
the FP64 oracle tests and the CUDA path may consume what it produces.
"""

from .scenes import (  # noqa: F401
    Field,
    Queries,
    config1_random,
    caustic_photons,
    field_from_photons,
    merge_photon_pairs,
    pinhole_hitpoints,
    orbit_views,
    uneven_views,
    perturbed_copy,
    concat_queries,
    subset_field,
    subset_queries,
    knn_distance,
    random_quaternions,
)
from . import storage  # noqa: F401,E402
