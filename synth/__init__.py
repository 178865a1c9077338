"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This package only produces geometry and densities (mesh nodes, quadrature
rules and weights, normals, expansion centers and radii, targets, locally
bisected and adaptive meshes).  It contains none of the evaluation method's arithmetic: no
spherical-harmonic expansions, translations, trees or interaction lists.
"""
from .surfaces import (  # noqa: F401
    Surface,
    make_surface,
    surface_from_flat,
    collocation_surface,
    flat_mesh,
    bisect_flat,
    scaled_curvature,
    urchin_radius,
    adaptive_flat_mesh,
    map_tail,
    conical_rule,
    sphere_radius,
    star_radius,
    real_ylm,
    triangle_rule,
    greens_density,
    random_harmonic_density,
    danger_radius,
    volume_points,
    near_surface_points,
    config_surface,
    batched_specs,
)
