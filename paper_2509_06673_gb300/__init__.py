"""GB300-native FETI interface solver for coupled poroelasticity/elasticity.

The compute path is the C-ABI CUDA library ``libfetipe.so`` (``csrc/``), reached through
``paper_2509_06673_gb300.fetipe`` (ctypes binding, argument marshalling only).
``workloads`` holds the seeded synthetic inputs.  Importing this package does not load the
library; importing ``fetipe`` does, and fails loudly if it has not been built.
"""
