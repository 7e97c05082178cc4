"""CPU FP64 oracle for FS-1 (Liao, Chen, Wang, Bai, Jin, Wu: "Fast Sinkhorn I: an
O(N) algorithm for the Wasserstein-1 metric").

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path imports,
links or runs this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2202_10042_gb300/csrc``); the only module
both sides use is the seeded input generator
``paper_2202_10042_gb300/inputs.py``, which holds none of the method's
arithmetic.

Contents
  dense       the plain definitions: Gibbs kernel, ground cost, dense Sinkhorn
              (plain and log-domain twin) in the loop order of Algorithm 1 / 2,
              marginal error, transport cost, in 1D, 2D and 3D (the third axis
              of Section 4's closing remark).  FP64, O(N^2) per iteration.
  exact       closed forms that pin the above: exact 1D W1 from the CDFs,
              brute-force LP, entropy.
  recurrence  Algorithm 1 and Algorithm 2 with the Horner / Qin Jiushao
              recurrences of Section 3 (eq. "recursion") and Section 4
              (eq. "2d recursion") in pure Python loops, the log-domain
              recurrences, and the O(N) transport-cost recurrence.
  marginals   log-domain application of the (separable) Gibbs kernel and the
              row / column marginals of a returned iterate, vectorised for
              entry-by-entry checks of full-size workloads.
  cref        ctypes wrapper of fs1_ref.c: the same sequential recurrences in
              plain C99 FP64 (plain form and the stabilised form of the Remark
              in Section 3), in 1D, 2D and 3D, fast enough for N = 2^20 and
              512 x 512 grids.

Every function states the passage of the paper it follows, and where the
paper is silent or ambiguous, the reading it takes.
"""
