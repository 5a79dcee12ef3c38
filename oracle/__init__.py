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
    nearinterp the interpolation step of the nearly-singular method for the closest targets
               (Section 2.1, last paragraph)
    fastrot    band-limited fields on the rotated grids of all targets of a latitude by FFTs, and
               the singular rule built on them (Section 2.1, the fast all-target rotation)
    physics    forces, rates and the midpoint time step (Section 1, Algorithm 1)
    reparam    the reparametrisation of the surfaces (Section 2.2)
    upsampling adaptive upsampling from the mean curvature's spectrum (Section 2)
    spt        small-deformation theory (Section 3, Appendix)
    mlp        the warm-start network (forward, backward, Adam)
"""
