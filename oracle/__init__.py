"""Plain FP64 CPU oracle of the method of Vales & Giannakis (arXiv 2510.26574).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` use it.  It shares no code with the CUDA path.

Every function follows the paper's definitions or the steps of its algorithms
in order, in float64 with NumPy/SciPy/LAPACK as the only library primitives:

* kernel.py   -- Gaussian kernel entries (Eq. (data-kernel)), dense K.
* dense.py    -- dense D, Q, P = D^-1 K Q^-1 K D^-1 and L = D^-1/2 K D^-1/2
                 (Section 1.1) and their eigendecompositions.
* philox.py   -- Philox4x32-10 counter-based generator (Salmon et al. 2011),
                 the source of every random number the method draws.
* pchol.py    -- pivoted partial Cholesky: greedy, RPC/ARPC (Algorithm 2 with
                 the accept/reject check of Algorithm 3), residual diagonal.
* alg1.py     -- Algorithm 1: degree vectors, Householder QR of D~^-1 F,
                 r x r EVD, lift U = Q1 V; the symmetric variant (Section 2.1).
* lowmem.py   -- low-memory ARPC (Appendix A, Remark of Section 4.2): only the
                 pivots S and W = F(S,:) are kept, F = K(:,S) W^-T is rebuilt
                 in row panels; Algorithm 1's degrees, Grams and eigenpairs
                 from (S, W) without an N x r array.
* bounds.py   -- Theorem 1, Theorem 4 and Lemmas dbound/qbound evaluated densely.

Every function is pinned by tests under tests/test_oracle_*.py against values
and properties the paper or the mathematics fixes.  Parity unpinned: only the
paper's printed 8.91% trace error of its own KS run (Section 4.1), whose data,
initial condition and bandwidth rule differ from the synthetic inputs here.
"""
