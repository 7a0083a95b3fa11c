"""FP64 CPU oracle for the mixed-variational plane-wave band problem and its adjoint.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA library.

It is the plain dense definition of the method, written from the paper:

* ``lattice``     -- cubic primitive cells, reciprocal basis T, plane-wave index set
                     (Results, eq. ``mixedvariation`` and the test-function definition
                     that follows it; Methods, "Study of cubic unit cells").
* ``mixed``       -- element-sum assembly of Omega, Phi and H by centroid quadrature
                     (Methods, eqs. ``loop`` and ``matrixofintegral``; Results,
                     eqs. ``intH``, ``intOmega``, ``intPhi``), material interpolation
                     (Methods, eq. ``combinematerial``), the condensed pencil
                     H Phi^-1 H^H U = lambda Omega U (Results, eq. ``matrixform``) and
                     its dense LAPACK solve.
* ``gap``         -- the normalized gap objective (Methods, eq. ``obj``; Results,
                     "A note on normalized band gaps") and its gradient weights.
* ``sensitivity`` -- eigenvalue sensitivities (Methods, eqs. ``normalev``,
                     ``sensitivityew``, ``diffOmega``, ``diffPhi``) in two forms: the
                     literal per-element matrices (tiny cases) and the voxel quadratic
                     forms they reduce to.
* ``mma``         -- one step of the method of moving asymptotes for the box-constrained
                     design problem (Methods, eq. ``topopt``; the paper names no optimizer).
* ``projection``  -- the design parametrisation: reduced design field, Heaviside projection
                     and the SC mirror symmetry, with their chain rule (Methods, "Topology
                     optimization formulation"; Results, "Topology optimized structures").

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms
(homogeneous media, Rytov laminates), invariants (Gamma zero modes, time
reversal, translation, point group, inversion), brute-force finite differences
and the numbers the paper prints (band edges of its optimized cells, sphere-inclusion
gaps, the 1-D laminate optimum).
"""
from . import lattice, mixed, gap, sensitivity, mma, projection  # noqa: F401
