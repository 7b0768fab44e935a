"""CPU oracle for delta-temporal motif counting and the interval-sampling
estimator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import or run anything here.  The oracle shares no code with the CUDA
library in ``paper_1810_00980_gb300``, and neither imports the other.

Contents (Liu, Benson & Charikar, "A sampling framework for counting temporal
motifs", WSDM 2019):

* ``count_bruteforce``  -- Def. 2.2 / Def. 2.3 written out: every l-subset of
  edges, ordered by time, checked for strictly increasing times, span <= delta
  and a node map that is injective both ways.  Tiny graphs only.
* ``count_exact``       -- the same count by extending partial instances in
  time order (C, ``enum.c``); returns the count-duration histogram that the
  Section 4 subroutine A(T', M, delta) must output.
* ``estimate``          -- Algorithm 1 step by step (shift, windows of Eq. 1,
  Bernoulli(q_j) keeps, exact per-window counts, weights 1/p_{M'} of Eq. 2
  with p_{M'} = 1 - Delta/(c delta), division by q_j, mean over b shifts),
  with exact rational per-term arithmetic and a correctly rounded sum.
* ``ex23``              -- Algorithm 2 (EX23) for the two-node motif
  (u,v),(v,u),(u,v), an independent exact counter used as a pin.
* ``rng``               -- the random draws of Algorithm 1 (shift and keep
  decisions) from SplitMix64, implemented here from its published definition.

Pins (tests/test_oracle_pins.py) tie every function to something other than
itself: hand-counted graphs, exhaustive enumeration, the k-clique reduction of
Theorem 3.1, Eq. 2 by brute force over shifts, Lemma 4.1, Theorem 4.3 and
Lemma 4.4 exhaustively over keep sets, Lemma 4.2, and closed forms.
"""
from .core import (count_bruteforce, count_exact, count_exact_hist, windows_of_shift,
                   window_records, z_from_records, estimate, ex23, relabel_motif)
from . import rng

__all__ = ["count_bruteforce", "count_exact", "count_exact_hist", "windows_of_shift",
           "window_records", "z_from_records", "estimate", "ex23", "relabel_motif", "rng"]
