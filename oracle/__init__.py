"""FP64 CPU oracle for the SARA / SDMM imaging path.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
NumPy/SciPy statement of what the imaging path computes, written from the
paper ("Why CLEAN when you can PURIFY?", arXiv:1502.05037) and from the
published methods it relies on (Kaiser-Bessel gridding, Daubechies wavelets,
SDMM). Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import it. The CUDA library never calls into it and shares no code,
table or constant generator with it.

Modules:
  nufft       - measurement operator Phi = G F Z S, its adjoint, exact DFT model
  wavelets    - Daubechies filters, periodic 2-D DWT, SARA dictionary Psi
  sdmm        - prox, projections, CG, SDMM iteration (all blocks, or one
                group of blocks per iteration), reweighting, epsilon
  primal_dual - a Chambolle-Pock solver of problem (3): pins SDMM's fixed
                point and is the oracle of the library's primal-dual solver
  unet        - the learned warm start's network (not in the paper): forward,
                backward and Adam in FP64
"""
