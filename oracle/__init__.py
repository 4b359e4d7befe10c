"""Plain FP64 CPU oracle for batched TNMC (arXiv 2509.19006).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` use it. It shares no code with
the CUDA path (``paper_2509_19006_b300/``); the only common input is the seeded
generator in ``workloads.py``, which holds none of the method's arithmetic.

What it computes is the method itself, step by step, in float64 numpy:

* ``ising``   - Eq. 1 energy, Eq. 7 Boltzmann matrix, coupling layout (Sec. 3.1).
* ``bmps``    - Sec. 2.2 / 3.2 boundary-MPS environments: bottom-row MPS, row MPO,
                MPO x MPS (bond doubles), then compression by a left-to-right QR
                sweep and a right-to-left truncating SVD sweep; log Z (Eq. 6).
* ``sampler`` - Sec. 3.3 row-by-row ancestral proposal (right environments,
                left sweep, Eq. 5 logits, Eq. 9 log q) and teacher-forced scoring.
* ``mh``      - Eq. 10 independence Metropolis-Hastings.
* ``philox``  - Philox4x64-10 (Salmon et al., SC'11), the counter-based generator
                both sides implement from its published definition.
* ``exact``   - brute-force enumeration (Eq. 2-4) and the exact row transfer
                matrix, the references the oracle is pinned against.
* ``potts``   - the q-state Potts extension (Sec. 5): energy, q-state copy-tensor
                MPOs through the same compression, q-way proposals and scores, and
                its exact references (enumeration, row transfer matrix).

Each function's docstring states how it reads the points the paper leaves open.
"""
