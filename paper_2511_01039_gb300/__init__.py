"""GB300-native boundary-MPS row absorption with rSVD / CBE compression.

The compute lives in the C-ABI library ``_lib/libfpeps.so`` (include/fpeps.h);
``fpeps`` is its thin ctypes binding. Importing this package loads nothing.
"""
