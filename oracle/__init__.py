"""FP64 CPU oracle for the boundary-integral hot path (test infrastructure only).

This package is the slow, plain restatement of the method that the CUDA library is checked
against. Only the tests, the smoke check and the bench's CPU-baseline leg may import it; the
product path never calls it and shares no code with it. Every function cites the part of
the paper it follows (Sorgentone, Tornberg & Vlahovska, "A 3D boundary integral method for
the electrohydrodynamics of surfactant-covered drops").

Modules:
    sh         Gaussian grid, normalised Legendre functions, real harmonics, SHT (Section 2)
    geometry   surface position, tangents, normal, area element (Section 1, Section 2.1)
    quadrature regular rule (Eq. reg_quadrature), modified weights (Eq. mod_weights),
               rotated-pole singular self-integration (Section 2.1)
    operators  Laplace and Stokes layer operators and their Galerkin projections
               (Eqs. op_stokes, dl_op_laplace, BIM_galerkin, galerkin_En)
    gmres      restarted GMRES used to solve the Galerkin systems
    nearsing   nearly-singular correction by upsampling (Section 2.1)
    physics    forces, rates and the midpoint time step (Section 1, Algorithm 1)
    mlp        the warm-start network (forward, backward, Adam)
"""
