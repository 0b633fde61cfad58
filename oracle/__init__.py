"""Plain FP64 CPU oracle for filter diagonalization (FD).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it.  The CUDA
library never calls it and shares no code with it: the two sides meet only in
the seeded input generators of ``fd_inputs`` (which hold none of the method's
arithmetic) and in the published definitions each side implements on its own
(the SplitMix64 counter generator, the Hubbard basis ordering).

Every function follows the paper (Alvermann, Hager, Fehske, "Orthogonal layers
of parallelism in large-scale eigenvalue computations", arXiv 2209.01974) in
the order its text states, in float64, with NumPy / SciPy primitives (matrix
products, Cholesky, triangular solves, dense symmetric eigensolvers) as steps
and no blocking, fusion or reordering beyond that.  Algorithms 1 and 2 of the
paper are printed as images; their steps are reconstructed from the prose of
Sec. 2 and the kappa = 5 memory-traffic count of Sec. 3.2 (Eq. EstimateT).

Modules
-------
splitmix     counter-based SplitMix64 streams (Steele, Lea, Flood 2014)
matrices     Hubbard chain/ring, 3D Anderson, tight-binding chain, diagonal test
             matrices, all as CSR (Sec. 3.2, Sec. 4.1)
chebyshev    Jackson kernel, window coefficients, Chebyshev filter (Sec. 2, Alg. 2)
lanczos      spectral inclusion interval from m Lanczos steps (Sec. 2)
ortho        Cholesky-QR 2 with shifted fallback (Sec. 2 orthogonalisation)
rayleigh_ritz  Ritz pairs and residual norms (Sec. 2)
fd           the FD outer loop (Sec. 2, Alg. 1) with the interval/degree heuristic
kpm          kernel-polynomial density-of-states moments (Sec. 4.1)
lehmann      Lehmann bounds of the eigenvalues nearest a shift (Sec. 2 intervals)
comm         communication metrics chi_1..3 and volumes of distributed SpMV (Sec. 3.1)
mlp          the filter-parameter perceptron: forward, gradient, Adam
"""
