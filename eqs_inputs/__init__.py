"""Seeded synthetic inputs for the EQS workloads.

This module produces the *inputs* of the method only: node coordinates,
tetrahedral connectivity, per-tet material ids, per-node Dirichlet tags and
the material/drive parameters.  It holds none of the method's arithmetic
(no element operator, no solver, no time integrator), so both the CPU oracle
and the CUDA path may use it.

The paper's own workload (an insulator with a 1 mm microvaristor coating,
Section V) is not available; Kuhn-split cube meshes of the same size class
stand in for it (the 128^3 jittered cube has 2.15 M nodes / 31.8 M matrix
non-zeros against the paper's 2.1 M DoF / 30.4 M nnz).
"""

from .mesh import (  # noqa: F401
    L_CUBE,
    Material,
    Problem,
    splitmix64,
    uniform01,
    kuhn_cube,
    kuhn_cube_p2,
    P2_EDGES,
    dirichlet_tags_p2,
    make_problem_p2,
    tag_materials_block,
    tag_materials_spheres,
    dirichlet_tags,
    make_problem,
    config_problem,
    batch_instance_params,
    BACKGROUND,
    VARISTOR,
    MLP_SIZES,
    MLP_NPARAM,
    mlp_init,
)
