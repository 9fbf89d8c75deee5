"""CPU oracle for the recursive Green's function (RGF) transport path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg use it.  It shares no code with the CUDA library;
the only common module is ``workloads`` (seeded random inputs, no method
arithmetic).

Everything here is plain, slow, complex128 numpy, written from the paper
(S. Ihnatsenka, "Computation of electron quantum transport in graphene
nanoribbons using GPU", Comput. Phys. Commun. 183 (2012) 543):

* ``lattice``  -- armchair ribbon tight-binding blocks built from atom
  coordinates (one p orbital per carbon atom, armchair edges).
* ``leads``    -- semi-infinite lead self-energies by Lopez Sancho-Rubio
  decimation (the paper says the lead self-energies must be included at the
  first and last slice; it solves an eigenproblem, we decimate).
* ``dense``    -- the plain definition: G = (E + i eta - H - Sigma_L - Sigma_R)^-1
  (Eq. 1) and the Landauer trace (Eq. 2), by dense inversion.
* ``rgf``      -- the recursion over unit-cell slices (Eqs. 4-5) and the
  trace (Eq. 2).
* ``gradient`` -- dT/d eps_i: the closed form from the dense G, the closed
  form with its blocks assembled slice by slice from left- and
  right-connected sweeps (accurate near E = 0), and the reverse (adjoint)
  sweep of the recursion.
* ``ldos``     -- the local density of states -Im G_ii / pi from the
  Dyson-assembled diagonal blocks of G.
* ``bands``    -- channel counts: closed-form armchair band edges and a
  brute-force band structure; the Bloch-state LDOS of the infinite ribbon.
* ``mp``       -- the same recursion in arbitrary precision (mpmath) for the
  ill-conditioned E = 0 point on small ribbons.
"""
