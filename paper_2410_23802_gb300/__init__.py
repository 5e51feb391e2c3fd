"""GB300 (sm_103a) implementation of the volumetric lattice Boltzmann method
for thermal particulate flows with conjugate heat transfer (arXiv 2410.23802).

The product is the CUDA library ``libvlb.so`` behind the C ABI of
``include/vlb.h``; :mod:`paper_2410_23802_gb300.vlb` is its thin ctypes
binding and :mod:`paper_2410_23802_gb300.workloads` builds the seeded
synthetic cases.
"""
