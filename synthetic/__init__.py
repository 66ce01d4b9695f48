"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates meshes (nodes + cells + boundary description) and the
initial / exact flow data as cell averages (exact solutions: translated waves,
the isentropic vortex, the exact 1D Riemann solution of the shock tubes).  It holds none of the WENO
method's arithmetic: no geometry tables, stencils, reconstruction, weights,
fluxes or time stepping.  Every random draw uses numpy's PCG64 with an
explicit seed, so the same call gives the same bytes on every machine.
"""
from .meshes import (MeshInput, quad_grid, perturbed_quads, split_quads, stretched_vortex_mesh,
                     mesh_for_config, batch_instances, instance_mesh, tube_mesh, periodic_mesh)
from .flows import (density_wave, isentropic_vortex, scalar_wave, four_quadrant_states,
                    cell_average, four_quadrant_average, euler_prim_to_cons, riemann_exact, shock_tube, shock_vortex,
                    moving_shock, double_mach)

__all__ = [
    "MeshInput", "quad_grid", "perturbed_quads", "split_quads", "stretched_vortex_mesh",
    "mesh_for_config", "batch_instances", "instance_mesh", "tube_mesh", "periodic_mesh", "density_wave", "isentropic_vortex", "scalar_wave",
    "four_quadrant_states", "cell_average", "four_quadrant_average", "euler_prim_to_cons", "riemann_exact",
    "shock_tube", "shock_vortex", "moving_shock", "double_mach",
]
