"""CPU oracle for the clean SLPF of a text under a regular expression.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package.  The product library never does.

What is here, and the passage of the paper each part follows
(arXiv 2503.06763, "A parallel parser for regular expressions"):

* ``re_front``  -- RE syntax (Sect. 2.1), numbered RE e_# (Sect. 2.2, Eq. 1),
  classic followers Fol (Eq. classicfollowers), the recursive segment
  computation (Fig. segmentalgo), FolSeg (Eq. folsegdef), initial / final
  segments, ε symbols and character sets (App. A).
* ``serial``    -- the serial two-way NFA parser written from Eq. matrixmul,
  Eq. reverseNFAdef and Fig. serialparser: C_0 = I, C_r = N_{x_r} C_{r-1};
  Ĉ_n = F, Ĉ_r = N_{x_{r+1}}^T Ĉ_{r+1}; output C_r ∩ Ĉ_r.  A pure-Python loop
  serves small texts; ``serial_parser.c`` runs the same matrix products for
  large ones.
* ``trees``     -- brute-force enumeration of all syntax trees of a text
  (Sect. 2.1, Example 1), their LSTs (Prop. 1) and their factoring into
  segments (Sect. 2.3.2): an independent definition of the clean SLPF.
* ``matches``   -- match extraction (Sect. 4.2, getMatches): the spans of a
  group, from enumerated trees and from a visit of the clean SLPF.
* ``parallel_equations`` -- the parallel algorithm's Eqs. reacher, joiner,
  builder and merger (Sect. 3.2) with DFA / ME-DFA transition functions
  computed on segment sets (Sect. 3.1), used for the Example 6 pins and
  chunk-invariance checks; ``parse_parallel_dfa_starts`` starts either
  direction from every DFA state instead (Sect. 5's comparison).
* ``speculation`` -- counts a chunk's speculative runs and transitions under
  ME-DFA starts, all-DFA-state starts, forward-restricted backward starts and
  shifted chunk edges (Sects. 3.1, 4.3), for the measured comparison of the
  speculation reductions.

Every function here is pinned by a ``-m "not gpu"`` test against values the
paper prints, closed forms, or brute force; none is "parity unpinned".
"""
