"""CPU FP64 oracle for the SPPC eigensolver (test infrastructure only).

This package is the plain, slow, obviously correct reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never does,
and it shares no code with the CUDA path (inputs come from ``workloads``).

Contents
--------
sppc.py      Algorithm 2 (SPPC for the k lowest eigenpairs) step by step, with
             the correction recursion of Sec. 4.1 (Eqs. exp_seq2, bl_diag,
             sm_first, sm_lin_proj), block Gram-Schmidt + QR (Eqs. blkGS, QR,
             Qp), the bordered projected matrix (Eq. proj) and the SpMV-saving
             identities of Sec. 4.3 (Eqs. avoid_SpMV2, HPsip).
minres.py    MINRES (Paige and Saunders, 1975) for the small shifted solves.
hybrid.py    SPPC followed by a block continuation (preconditioned residual
             expansion) once SPPC stagnates (Sec. 5, 6).
lanczos.py   Block Lanczos with full reorthogonalisation (eigenvalue truth for
             matrices too large for a dense eigendecomposition).
spmm.py      CSR x dense block product (plain C loop with OpenMP, or SciPy).
rmmdiis.py   SPPC followed by per-pair RMM-DIIS (the paper's hybrid, Sec. 6).
learned.py   Learned correction proposal (not in the paper): features, the
             per-row network, its gradient, Adam, the regression target built
             from exact eigenvectors, and the keep rule.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, special cases that reduce to textbook routines, invariants and brute
force (dense eigendecomposition of the whole matrix).
"""
from .sppc import sppc, small_eigenpairs, SPPCResult  # noqa: F401
from .minres import minres  # noqa: F401
from .lanczos import block_lanczos, dense_lowest  # noqa: F401
from .spmm import csr_spmm  # noqa: F401
from .hybrid import sppc_hybrid  # noqa: F401
