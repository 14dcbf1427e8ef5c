"""FP64 CPU oracle of the MR-STAT signal model, its Jacobian products and the
inexact Gauss-Newton solve (van der Heide et al., arXiv 1904.13244).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, calls or links this package; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code, table or constant generator with the
CUDA path; both sides only share the seeded input generators in ``synth``.

Everything here is plain NumPy in float64 (complex128), written for clarity, not
speed: a loop over TRs vectorised over voxels, and the spatial encoding as the
explicit sum over voxels of rho * m * exp(-i k.r) per TR.

Modules
-------
bloch     Supporting Information S2: hard-pulse Bloch recursion (Rodrigues rotation,
          T1/T2 decay and regrowth) and its forward-mode derivatives.
encoding  Theory, Eqs. 1-2 and the s = M rho form: the volumetric signal sum with
          the Cartesian gradient-encoding phase, and its adjoint.
model     Residual/objective/gradient (Theory, "Computing the gradient g") and the
          Jacobian products J.v and Re(J^H w) (Algorithm 4, Eq. 4).
solver    CGLS initial proton density (Methods, "Reconstructions"), mask, Steihaug
          truncated CG and the trust-region inexact Gauss-Newton loop (Algorithm 6).
metrics   NRMSE (Results, "Numerical Brain Phantom").

Parity pins (tests/test_oracle_*.py) tie each function to something other than
itself: the Freeman-Hill bSSFP steady state, pure inversion recovery, free
induction decay, complex-step and central finite-difference derivatives,
numpy.fft on piecewise-constant time courses, exact linearity in rho, the
adjoint identity, brute-force double sums on tiny grids and noiseless recovery
of ground-truth maps.  The low-rank model (model.project_onto_basis,
model.time_basis) is pinned to the identity at full rank, numpy's least-squares
solver, the algebra of orthogonal projectors, Eckart-Young optimality and the
Freeman-Hill steady-state pattern; the bound reflections (solver.reflect_into_bounds,
solver.apply_bounds) to hand-computed values (tests/test_oracle_lowrank.py).
"""
from . import bloch, encoding, model, solver, metrics  # noqa: F401
