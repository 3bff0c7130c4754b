"""GB300-native per-particle push for high-order DG point-particle solvers.

The compute path is the C-ABI library ``libpt`` (CUDA, sm_103a) declared in
``include/pt.h``; :mod:`paper_2211_05458_gb300.pt` is its thin ctypes binding.
:mod:`paper_2211_05458_gb300.workloads` makes the seeded synthetic inputs.
"""
