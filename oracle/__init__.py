"""FP64 CPU oracle for the T^2S^2 hot path (arXiv 2506.04732).

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or runs
this package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg do.  It shares no code with the CUDA path: the only common
module is ``workloads`` (seeded problem parameters, no method arithmetic).

Everything here is plain, slow, FP64 numpy written from the paper:

* ``gll``          - Legendre polynomials, Gauss-Lobatto-Legendre representation
                     points (Overview (i)), Gauss points.
* ``collocation``  - superconsistent collocation points and the 1D Lagrange
                     matrices R, D, D2 evaluated on them (Overview (ii)).
* ``operator``     - the d-dimensional collocation operator as a sum of
                     Kronecker products / a rank-2 TT-matrix (eq. tt-matrix-format),
                     dense assembly for tiny grids, manufactured sources.
* ``tt``           - TT format (eq. TT-format:elementwise), TT-SVD, rounding,
                     add/scale/dot/norm, TT-matrix-by-TT product (Methods).
* ``solve``        - dense direct solve for tiny grids, an AMEn-style
                     alternating solver, Crank-Nicolson / backward-Euler steps
                     (eq. ttss-Crank-Nicolson, eq. ttss-backward-Euler).
* ``spacetime``    - the unified space-time formulation: time as one more
                     collocated dimension, the initial condition lifted into
                     the right-hand side.

Pinning status of each function is listed in its module header.  The
superconsistent node rule follows a reading of the paper (the formula itself
is not printed in it); see ``collocation.sc_nodes``.
"""
