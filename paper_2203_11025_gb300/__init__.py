"""GB300-native preconditioned Helmholtz solver (FGMRES + shifted-Laplacian
multigrid + U-Net preconditioners) behind the C ABI of libhelm.

Importing the package loads nothing; `paper_2203_11025_gb300.lib` opens the
CUDA library and fails loudly if it has not been built.
"""
__all__ = ["synth"]
