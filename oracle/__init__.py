"""FP64 CPU oracle for the FKP multipole estimators (Scoccimarro 2015).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct statement of what the CUDA path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA
path (``paper_1506_02729_gb300``) and imports nothing from it; the only
module both sides use is ``mockgen`` (seeded catalogs, none of the method's
arithmetic).

Modules
-------
``power``      scalars (alpha, I22, N0, I33, S3, L^ab), gridding, moment
               fields, one 3-D FFT per field, Legendre recombination
               (eqs. delta2b, delta4b), shell binning and P_0, P_2, P_4, P_4b
               (eqs. P0_impl - P4_implb, I22def, N0true).
``bispectrum`` shell-filtered inverse FFTs (eq. F_k), real-space triangle
               sums (eq. Factorize), exact triangle counts by rounded FP64
               convolution, thin-shell shot noise (eq. SNbisp2thin) and B_l
               (eqs. BispMono, BispQuad).

Readings of the paper that the oracle fixes (the CUDA path follows the same):
Fourier sign e^{-ik.x}; weighted alpha = W_g/W_r; x^ at grid nodes; CIC/TSC
with nodes at origin + iH and periodic indices; compensation by prod sinc^p;
modes with any |n_a| = N/2 excluded; half-open FP64 bins; P_4b constant
35/2 with the 7/2 N_0 self-pair term; I_33 = alpha sum_r nbar^2 w^3; thin-shell
cosines from shell centres.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(brute-force DFT, direct Yamamoto sums, closed forms, plane-parallel Kaiser
and isotropy identities, brute-force triangle enumeration).  The window
compensation is pinned against the assignment kernel's own Fourier transform
(quadrature of the B-spline pieces) and by the compensated fields of an object
on a node; the monopole's shot-noise subtraction by one galaxy on a node with
randoms on every node (|F_0|^2 = w^2 on every mode, so P_0 = -alpha^2 sum_r
w_r^2 / I_22 in every bin).  The thin-shell
bispectrum shot noise is pinned for l = 0 by the single-object identity (one
galaxy on a node, randoms on every node: B_0 = -2 alpha^2/nbar^2 exactly for
every triangle) and for l = 0, 2, 4 against F_l and F^w_l summed directly over
objects placed on nodes (no grid, moments or FFT).
"""
from . import power, bispectrum  # noqa: F401
