"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package generates *inputs only*: meshes (node coordinates, 10-node
tetrahedra, boundary faces), layer-interface random fields, input velocity
wavelets and receiver layouts.  It holds none of the method's arithmetic
(no element matrices, no time stepping, no solver, no misfit), so both the
CPU oracle and the GPU library can consume its output without sharing any
computation.
"""
from .mesh import layered_box, VTK_TET10_EDGES, TRI6_EDGES, FACE_TOP, FACE_BASE, FACE_SIDE
from .fields import grf2d
from .waves import ricker, random_phase, sin2_pulse
from . import configs

__all__ = ["layered_box", "VTK_TET10_EDGES", "TRI6_EDGES", "FACE_TOP", "FACE_BASE",
           "FACE_SIDE", "grf2d", "ricker", "random_phase", "sin2_pulse", "configs"]
