"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package produces *inputs only*: box meshes (node coordinates, hexahedra,
boundary quadrilaterals), material constants, motion parameters and seeded
random draws. It contains none of the time-stepping or finite-element
arithmetic of the method; both the library and the oracle receive the same
arrays from here and compute everything else on their own.
"""

from .machines import (  # noqa: F401
    BoxMesh,
    Machine,
    box_mesh,
    build_machine,
    machine_config,
    tiny_machine,
    CONFIGS,
)
