"""FP64 CPU oracle of the VarSim thermal solve (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow, independently written reference that the CUDA
path is checked against. Only the tests, the smoke check of the build entry
point and the CPU-baseline leg of the benchmark may import it; the product path
(the CUDA library and its Python binding) never does and shares no code with it.

Modules
-------
physics : layer-stack spectrum g^(k), the fast-decaying top-layer
          Green's function by its eigenfunction series, the disc-source
          half-space closed form, and the spectral kernel K~ of the imaged die.
solve   : the mirror-image convolution (direct summation and dense-cosine
          spectral form), the leakage/conductivity fixed point (plain Picard on
          the unsplit equation, the mean/variation split, and the engines'
          preconditioned iteration from the uniform start with the update and
          the error-estimate stopping rules), the fixed point
          with a piecewise-linear leakage and kappa(T) through the Kirchhoff
          transform, the paper's one-shot closed form, and the transient
          Duhamel superposition with its windowed and implicit-leakage variants.
cnn     : the warm-start network (forward and backward).

Every function cites the passage of the paper it follows (section / equation).
Where the paper is silent the reading used is stated in the docstring.
"""
