"""CPU oracle for the randomized SVD -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of the thesis' randomized SVD (Algorithm 4,
Section 3.3; Algorithm 2 when q = 0; Algorithm 3 and Algorithm 1 for the
analysis tests), with the analysis formulas it is checked against
(Eq. 3.1, Theorems 2, 3, 5 and 6, Eq. 3.5, Eq. 4.3); Algorithm 5
(``hermitian``); Algorithm 6 (``singlepass``); the toolbox's adaptive range finder (``adaptive``) and its
SRFT test matrix with FastRandRF (``srft``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything here.  The
library (``paper_2402_17794_gb300``) never does: it shares no code, no
helpers and no constants with this package, and the two are compared only
on the same seeded inputs.

Pinning (what ties the oracle to the thesis rather than to itself) lives in
``tests/test_oracle_*.py``: exact recovery of matrices of known rank and
spectrum, Eckart-Young (Eq. 3.1), orthonormality, interlacing, the expected
error bounds of Theorems 2, 3 and 6 averaged over seeds, the canonical-angle
bound of Theorem 5, distribution tests of the Gaussian generator, and planted
mistakes that each pin must catch.  The Philox bit stream is pinned to the
published Philox4x32-10 known-answer vectors (Salmon et al., SC'11), stored
in ``tests/golden/philox4x32_10_kat.txt``.
"""

from .philox import philox4x32_10, gaussian_matrix  # noqa: F401
from .randsvd import (  # noqa: F401
    RsvdResult, orth, range_finder, rsvd, sign_normalise,
)
from . import adaptive, analysis, hermitian, singlepass, srft  # noqa: F401
