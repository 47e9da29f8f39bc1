"""FP64 CPU oracle for the multilevel ELM-FBPINN hot path (arxiv 2409.01949).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2409_01949_gb300``) never imports it, and it never
imports the product path: the two share no code.  The only shared module is
``workloads`` (seeded problem data, no method arithmetic).

Everything here is plain numpy / scipy in float64, written from the paper's
definitions so that a reader can check it against the paper by eye:

* ``rng``            SplitMix64 counter stream for the fixed random parameters
* ``decomposition``  multilevel subdomain centres and half-widths (§4.1), and the
                     subdomains discarded outside an L-shaped domain (§4.1, §4.4)
* ``windows``        cos^2 windows, derivatives, partition-of-unity (Eq. window_func)
* ``features``       shallow tanh random features and derivatives (§3, h = 1)
* ``ansatz``         the hard-constraint ansatz factor and its derivatives (§4.3)
* ``system``         entries of M and h (§3 "Definition of vectors / matrices")
* ``lstsq``          least-squares minimiser of ||M a - h|| (Eq. multilevel_ls): own
                     column-pivoted Householder QR, SciPy LSQR, and the Golub-Kahan
                     bidiagonalisation behind the condition-number estimates
* ``evaluate``       u_hat (Eq. multilevel_solution), e_L1 (Eq. l1_error), rel. L2
* ``gnn``            the learned preconditioner's network (not in the paper)

Parity status of each function is stated in its module header.
"""
