"""Plain FP64 CPU oracle of the consistent neural message-passing (NMP) network.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.

It is written from the paper (arXiv 2410.01657) in numpy/scipy float64, with
no blocking, fusion or reordering beyond what the paper's definitions state:

* ``oracle.graph``   -- GLL-brick graph (Sec. II-A, Figs. 2-3), element
  partitioning, reduced sub-graphs, edge/node multiplicities and halo rows
  (Sec. II-A, Fig. 4).
* ``oracle.model``   -- MLP blocks (Sec. III, Table 1), the consistent NMP
  layer Eq. 5a-5e evaluated rank by rank with halo rows appended, the
  encode-process-decode network, the consistent loss Eq. 8a-8c, and a
  hand-written FP64 adjoint of all of it (Eq. 3).

Pins (tests/test_oracle_*.py): Table 1 parameter counts, Table 2's R=8 row,
the Fig. 4 two-element example, closed-form graph sizes and GLL points,
Eq. 8c (N_eff = N), the consistency property Eq. 2/Eq. 3 (partitioned ==
unpartitioned), permutation equivariance, closed-form special cases of the
layer, brute-force loops on tiny graphs with torch.nn reference modules, and
central finite differences of the adjoint. Absolute output values of the
paper's own runs are not printed in the paper: that part is parity unpinned.
"""
