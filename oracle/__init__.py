"""FP64 CPU oracle for the free-space convolution of Jiang, Greengard & Bao (arXiv 1311.4120).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or execute
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path (no kernels, headers,
tables or helpers); the only common input is the seeded density from ``synth``.

Contents
--------
quadrature   nodes k_j and weights W_j of eq. 3.7 (Gauss-Legendre in r and theta,
             trapezoidal rule in phi) and the kernel symbols U_hat of eq. (int3dd).
direct       O1: the discrete operator written out as plain sums (eq. 3.2 into eq. 3.7,
             energy by the trapezoidal rule of Remark 3.3).  Exact up to rounding; tiny grids.
nufft        O2: the Gaussian-gridding NUFFT of Section 2 (periodic heat kernel, oversampled
             FFT, deconvolution by the heat kernel's Fourier coefficients), FP64, in C.
closed_forms O3: analytic potentials and energies of Section 4 and of the benchmark densities.
pipeline     Algorithm 1 assembled from the above: type-2 -> multiply -> type-1 -> energy.
alg2         Algorithm 2 (eq. 3.9): the partition of unity u = I_1 + I_2, I_1 by the
             2x zero-padded FFT with U_hat (1 - p_d), I_2 by Algorithm 1 with weights times p_d.

Every function is pinned in ``tests/test_oracle_*.py`` against something other than itself:
library special cases (the uniform DFT), brute force, closed forms, the paper's printed
energies (Example 7) and operator invariants.
"""
