"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the accelerated path computes, in
float64 / int64 numpy, written from the paper (Expression Acceleration, arXiv 2211.00621)
and from the textbook definitions it leaves to the user.  It shares no code with the CUDA
path: it imports nothing from the library package, and the library imports nothing from
here.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it.

Modules
-------
patterns  -- flatten / marshaling (one and two levels, and back), map, map2, reduce,
             segmented reduce, loop (Sec. 3.3 "Marshaling"; appendix Fig.
             "pmexpr-extension", the Futhark and CUDA parallel keywords; Sec. "Dynamic
             Assumptions").
hmm       -- HMM forward recursion (log-space and scaled), forward-backward expected
             counts, and the re-estimation after them (softmax-parameterised gradient,
             Baum-Welch M-step).  The paper is silent on HMMs; these are the textbook
             definitions, instantiated as a map (over states j) of a reduce (over states i)
             inside a sequential loop over t (Listing 1's foldl/reduce pairing).
pairwise  -- the all-pairs softened-gravity map-of-reduce.
pairhist  -- the all-pairs angular histogram (tpacf shape: a map over pairs reduced into
             bins).
brute     -- enumeration over HMM state paths (pins hmm on tiny models).

Every function here is pinned by ``tests/test_oracle_*.py`` against things other than
itself: brute force, closed forms, invariants and worked examples from the paper.
"""
from . import patterns, hmm, pairwise, pairhist, brute  # noqa: F401
