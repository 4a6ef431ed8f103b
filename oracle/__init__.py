"""CPU oracle for the negacyclic NTT path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call, link or execute
anything in this package.  The product path (``paper_2410_05934_gb300``) never
touches it and shares no code with it.

Contents:
  ntt_oracle.c  plain C, O(N^2) definitions of Sec. II-D / Eq. 1 with 128-bit
                products (forward NTT, inverse NTT, pointwise product,
                schoolbook negacyclic product, Miller-Rabin, psi).
  ntt_radix2.c  plain iterative radix-2 transforms, O(N log N): the second,
                fairer CPU timing baseline (pinned against ntt_oracle.c).
  oracle.py     ctypes binding returning numpy arrays.
  mlp_oracle.py float64 numpy forward/backward of the schedule cost model.
  build.py      compiles ntt_oracle.c with gcc.
"""
