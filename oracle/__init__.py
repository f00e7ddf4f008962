"""CPU oracle for graph-coloured H^1 peeling compression (Levitt & Martinsson).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute this package: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg use it.  It shares no code with the CUDA path (the only common
module is hm_workloads, which generates seeded input points and holds none of
the method's arithmetic).

Everything here is plain FP64 NumPy/Python, plus one small plain-C file
(graph.c) for the incompatibility-graph edges and DSatur so that the
200k-point workload finishes in seconds.  Each function cites the passage of
the paper it follows.

Modules
  tree     cluster tree, cuts, neighbour and interaction lists   (Section 3)
  graph    constraint sets, incompatibility graph, DSatur         (Sec. 2.6, 4.1.2, 4.1.3)
  philox   Philox4x32-10 counter-based generator + Box-Muller     (Gaussian test matrices)
  h1       the compression loop, black-box operators, apply, error (Alg. 2.1, Alg. 4.1, Sec. 5)

Parity status: every function is pinned by tests/test_oracle_*.py except the
tolerance-mode rank decisions at blocks whose singular values straddle the
threshold (parity unpinned by the paper: it does not say how k is chosen from a
tolerance).
"""
