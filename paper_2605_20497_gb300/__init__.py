"""GB300-native constrained multilevel hypergraph partitioner.

The compute path is the CUDA library ``libhp.so`` (sm_103a kernels behind a
C ABI, ``include/hp.h``); :mod:`.hp` is its thin ctypes binding and
:mod:`.inputs` holds the seeded synthetic workloads.  Importing the package
loads nothing; :func:`paper_2605_20497_gb300.hp.load` loads the library and
raises if it has not been built.
"""
