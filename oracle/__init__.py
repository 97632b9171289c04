"""FP64 CPU oracle for compressed-sensing SAR imaging with an approximated
observation (chirp-scaling focusing operator M, its inverse G = M^H, and the
iterative thresholding algorithm of Algorithm 1, Eq. (25)).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never calls it and shares no code with it: the oracle evaluates every
phase directly from its physical formula in float64 radians on full 2-D grids,
uses library FFTs (scipy.fft), and runs the algorithm steps in the paper's order
with no blocking, fusion or reordering.

Modules
  csa      grids, chirp-scaling phase functions H1/H2/H3, operators M and G
  rda      the range-Doppler operator pair with truncated-sinc RCMC C and D = C^T
           (the paper's own concrete example, Section III-C)
  ita      soft / half thresholding, the (K+1)-th largest magnitude, ITA with
           fixed or NIHT step, the autofocus loss and its gradients
  echo     exact point-target echo simulator (time domain, hyperbolic range)
  metrics  relative L2 error, point-response PSLR / IRW

Pins (tests under ``tests/test_oracle_*.py``) tie each function to something
other than itself: the dense Kronecker-matrix form of Theorem 1 (Eqs. (19)-(22)),
exact unitarity and the adjoint identity, point-target focusing with the textbook
resolution and sidelobe level, brute-force minimisation of the threshold
objectives, sorting, and the closed-form iterate at full sampling.
"""
