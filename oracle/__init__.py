"""CPU oracle for the batched DC loadflow path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or call anything in this package.  The product path
(the CUDA library and its binding) never imports it, and it imports nothing
from the product path: the only code both sides share is the seeded input
generator module, which holds no loadflow arithmetic.

Everything is FP64 and follows the paper's definitions directly: each
topology is rebuilt as a graph and its reduced susceptance matrix is factored
from scratch, with no low-rank update of a base solution.

Parity pins (tests/test_oracle_*.py): the hand-worked 3-bus example, Kirchhoff
current law at every non-slack bus, the zero slack column, LODF[l,l] = -1,
reciprocity of the branch-to-branch factors, the bridge <=> Phi_cc = 1
equivalence, brute-force islanding against an independent graph library,
LODF-of-own-PTDF against refactorisation per contingency, the Moore-Penrose
pseudo-inverse of the full Laplacian, and the paper's BSDF/MODF forms.
"""
from .dcflow_ref import *  # noqa: F401,F403
