"""B300-native hot path of the NanoBTE steady phonon BTE solver.

``libnanobte.so`` (built from ``csrc/`` with ``python -m
paper_2607_03226_b300.build``) holds the C ABI declared in ``include/nbte.h``;
``nbte`` is its ctypes binding.  Importing this package loads nothing.
"""
