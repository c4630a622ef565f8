"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds input synthesis only: counter-based random numbers, the
structured-then-unstructured meshes of the paper's experiments (Kuhn-split
tetrahedral boxes and perturbed hexahedral boxes, Section 4.1), their
cell->vertex and cell->node maps, and smooth synthetic fields.  It contains
none of the finite element arithmetic (no basis, quadrature, geometry or
operator code), so both the oracle and the GPU library can take their inputs
from it without sharing any of the computation under test.
"""
from .rng import splitmix64, uniform, randint
from .mesh import (
    PlaneMesh,
    quad_mesh,
    tri_mesh,
    quad_node_map,
    tri_lattice,
    tri_node_map,
    pk_lattice,
    pk_node_map,
    TetMesh,
    HexMesh,
    kuhn_tet_mesh,
    hex_box_mesh,
    hex_slab_mesh,
    p2_node_map,
    hex_node_map,
    shuffle_mesh,
    p2_node_coords,
)
from .fields import sinusoid_displacement, uniform_vector, grf_fourier_features, grf_lattice

__all__ = [
    "splitmix64",
    "uniform",
    "randint",
    "TetMesh",
    "HexMesh",
    "kuhn_tet_mesh",
    "hex_box_mesh",
    "hex_slab_mesh",
    "p2_node_map",
    "hex_node_map",
    "shuffle_mesh",
    "p2_node_coords",
    "sinusoid_displacement",
    "uniform_vector",
    "grf_fourier_features",
    "grf_lattice",
]
