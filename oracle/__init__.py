"""Independent CPU oracle for EBIC population fitness evaluation and the EBIC generation loop.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this package:
only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use
it.  It shares no code with the CUDA path (no kernels, headers, helpers or constant tables) and it
never imports the product package.

The oracle is written from the EBIC.jl paper (Renc et al., GECCO'21 Companion, arXiv 2105.01196):
the chromosome / trend definition of Sec. 2.3 ("EBIC" paragraph), the nine-step algorithm of
Sec. 2.4 ("EBIC.jl"), the evolutionary strategies of Sec. 2.3 (elitism, penalised tournament,
tabu list) and the parameters of Sec. 2.4 (negative trends, approximate-trend threshold, allowed
overlap, iterations, number of biclusters).  Where the paper is silent the module that implements
the step states the reading it takes.

Modules
  philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the word stream.
  fnv      64-bit FNV-1a hash of a column sequence (tabu-list identity).
  params   the parameter record and its validation.
  counts   per-(individual,row) trend counts, the approximate-trend threshold and fitness.
  bitmap   the column-pair comparison bitmap, from its plain definition.
  ebic     initialisation, tournament, crossover, mutation, tabu list, top rank list, the
           generation loop and bicluster extraction.
  quality  clustering error (CE, Eq. 1) with an optimal assignment.

Parity status: the counts, the threshold, Philox and FNV-1a are pinned by the tests in
``tests/test_oracle_*.py`` (hand example, brute force, invariants, published test vectors).  The
fitness formula, the top-list rule and the evolution operators follow readings the paper does not
fix: they are "parity unpinned" by the paper.  They are pinned to the text of those readings by
scripted-word and hand-worked cases (``tests/test_oracle_operators.py``,
``tests/test_oracle_toplist.py``, ``tests/test_oracle_tabu.py``) and by invariants of whole runs
(``tests/test_oracle_ebic.py``).
"""
