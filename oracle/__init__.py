"""CPU FP64 oracle for the RHEED/TRHEPD multi-slice forward model.

TEST INFRASTRUCTURE ONLY. ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import it; the CUDA path (the package
``paper_2306_00271_gb300``) never imports, links or calls anything here, and this package never
imports the CUDA path. Both sides only share the seeded input descriptions of
``paper_2306_00271_gb300.workloads`` (passed in as plain objects; not imported here).

Modules:
  model         physics of Section 2.1 (gamma, Gamma, U(z), intensities)
  conventional  O1: conventional multi-slice + recursive reflection (Section 2.2)
  integrator    O2: Algorithm 1 with SRKN splitting / RK4 and the RHST (Section 3)
  brute         mpmath references for tiny problems (Eq. ichimiya4 directly, O2 without RHST)
  curve         rocking curves over angles, eacc-style curve error (Section 4)
  closed_forms  one-beam slab reflection (derived from Eqs. vtau-bd1)
"""
