"""FP64 CPU oracle for the sliced tensor-network contraction.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call, link or
execute anything in this package; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (``paper_2205_00393_gb300``) and never
imports it; both sides only share the seeded input generators in ``tnc_inputs``.

Contents, each written from the paper (Liu et al., "Lifetime-based
Optimization for Simulating Quantum Circuits on a New Sunway Supercomputer"):

* ``statevector``  - brute-force state-vector simulation (ground truth for the
  circuit -> network translation and for amplitudes of small circuits).
* ``tn``           - contraction of a tensor network along a contraction tree,
  with slicing (Sec. 2.1.1, Eq. 1, Eq. 2): the amplitude is the sum over all
  assignments of the sliced indices of the sliced contraction.
* ``planner``      - greedy contraction path, contraction-tree bookkeeping,
  Eq. 1/2/3 costs, lifetimes (Def. 1), the stem, the slice finder
  (Algorithm 1), the simulated-annealing refiner (Algorithm 2) with
  find_critical_tensors (Algorithm 3) and find_candidate_indices (Algorithm 4).
* ``gradient``     - derivatives of amplitudes with respect to fSim parameters
  (exact, by multilinearity; and central finite differences).

Precision: complex128 / float64 throughout; integer costs are exact Python ints.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
something other than itself (closed forms, brute force, invariants, the
paper's worked examples under ``tests/golden/``).
"""
