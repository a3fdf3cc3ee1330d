"""FP64 CPU oracle for the nonsmooth sphere DEM step of arXiv 2501.05300.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users; the library never imports this package.
It shares no code with the CUDA library.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  detection (sphere-sphere)   pinned: KD-tree pair query (scipy), brute force
  detection (sphere-geometry) pinned: dense surface sampling of the primitive
  normal law + SPOOK          pinned: Hertz head-on collision closed form,
                              static resting column, energy / momentum laws
  Coulomb friction            pinned: sphere on an inclined plane (stick/slip)
  rolling resistance          pinned: rolling sphere on an incline
  Jacobi sweep                pinned: converges to the MCP solution found by an
                              independent projected Gauss-Seidel on tiny cases
  step-size / iteration rules pinned: Table 3 of the paper
  coloured PGS (solver = 1)   pinned: reaches the Jacobi solution where the
                              problem has one (frictionless), converges faster,
                              meets the resting-column static limit; colour
                              count within the greedy-colouring bounds
  load-driven plate groups    pinned: free fall under load equals the discrete
                              sum of the step; a loaded plate on a sphere on a
                              floor reaches the Hertz static overlaps; particle
                              plus plate momentum changes by exactly F t
  gradient (torch_step.py)    pinned: its FP64 forward equals oracle.c step by
                              step; its autograd gradient with respect to
                              (k_n scale, mu_t, mu_r) equals central finite
                              differences of oracle.c
"""
from .binding import Oracle, OracleParams, Geom, detect, load, lib_path, build  # noqa: F401
