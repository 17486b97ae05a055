"""FP64 CPU oracle for the laminographic operator L, its adjoint and ADMM-TV.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2511_01893_b300``): the only common module
is the seeded input generator ``paper_2511_01893_b300.inputs``, which holds
none of the method's arithmetic.

What it follows (paper: Ma et al., "mLR: Scalable Laminography Reconstruction
based on Memoization", SC'25):

* Eq. 1 (Section 2): the objective 1/2 ||L u - d||^2 + alpha ||u||_TV.
* Section 2, operator dimensionalities: F_u1D maps u[n1, n0, n2] to
  u1[n1, h, n2]; F_u2D maps u1 to u2[n_theta, h, w]; F*_2D is the per-angle
  inverse 2D FFT on the h x w grid.
* Algorithm 1 (LSP) and Algorithm 2 (Optimized LSP, the operation
  cancellation of Section 4.2 that uses F_2D F*_2D = I).
* Section 6.1, Eq. 4: the accuracy metric E = ||R_comp - R||_F / ||R_comp||_F.

The paper defers the mathematics of L (kernel, oversampling, geometry,
normalisation, CG rule, TV discretisation, penalty rule) to its references
(Dutt-Rokhlin / Beylkin unequally-spaced FFT; Boyd et al. ADMM).  The readings
taken here are listed in each module's docstring:

* ``usfft``  - Gaussian-kernel unequally-spaced FFT, type 2 and its exact
  transpose, 1D and 2D.  Pinned by direct NUDFT sums and error decay in m.
* ``lamino`` - laminographic geometry, L-hat, L, adjoints and the direct
  NUDFT of the Fourier-slice projection.  Pinned by the direct NUDFT, the
  adjoint identity, a closed-form Gaussian-blob projection and the phi = 0
  tomography limit.
* ``tv``     - forward-difference gradient, its negative transpose (div),
  isotropic TV and isotropic shrinkage.  Pinned by adjointness and closed forms.
* ``admm``   - Algorithm 1 / Algorithm 2 LSP with a Dai-Yuan CG step and an
  exact line search, RSP, dual and penalty updates.  Pinned by a dense normal
  equation solve, Alg 1 == Alg 2, and the minimum of the smoothed objective
  found by an independent quasi-Newton solver.
"""
