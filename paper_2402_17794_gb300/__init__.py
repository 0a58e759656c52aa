"""GB300-native randomized SVD (Algorithm 4 of X. Li's 2021 thesis on
randomized SVD algorithms, Section 3.3) behind a C ABI (include/rsvd.h).

``rsvd`` holds the Python binding (same names as the C entry points);
``synthetic`` builds seeded test matrices; ``_build`` compiles the CUDA
sources in ``csrc/`` for sm_103a.
"""
__all__ = ["rsvd", "synthetic", "build_library"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    from ._build import build
    return build(force=force, verbose=verbose)
