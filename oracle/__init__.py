"""FP64 CPU oracle for the electrostatic global-placement inner loop.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it.

Everything is plain numpy in float64 (integers in int64), written from the
definitions:

* ``wirelength`` -- HPWL (Eq. 1) and the weighted-average wirelength model with
  its gradient (Eq. 3).
* ``density`` -- fixed-point quantisation, exact cell/bin overlap-area density
  map, overflow, bin density and the density-gradient field gather.  The paper
  only cites the electrostatic density (ePlace); the reading is stated in each
  function.
* ``poisson`` -- the spectral (cosine-series) Poisson solve for potential and
  field, in a naive O(n^4) and a separable O(n^3) form.
* ``placer`` -- the Nesterov/Lipschitz iteration with its lambda and gamma
  schedules that minimises Eq. 2 (the global-placement step of Algorithm 1,
  run until it converges).
* ``perturb`` -- SplitMix64 and the Shuffle / Shuffle (all) operators
  (Algorithm 1; Section 4.2).
* ``wiremask`` -- the WireMask perturbation (Section 4.2): every movable macro
  in turn to the grid position of least HPWL.
* ``hybro`` -- the Hybro loop and best-solution selection (Algorithm 1).
"""
