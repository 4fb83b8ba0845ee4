"""GB300-native two-site variational ground-state search (arXiv 1703.00387).

The compute lives in the CUDA shared library ``libosmps.so`` (sources in
``csrc/``, C ABI declared in ``include/osmps.h``). ``binding`` wraps it with
ctypes; it is loaded on first use and raises if it is missing. ``inputs``
draws seeded synthetic inputs and ``hamiltonians`` builds MPO tensors on the
host.
"""
