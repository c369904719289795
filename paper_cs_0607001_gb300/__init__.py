"""GB300-native multiresolution correlation of complex signals in the
shift-invariant DWT domain by lifting (Bhattacharya & Mahapatra).

The compute path is the CUDA library ``libsidwt`` (``csrc/``) behind a C ABI;
``sidwt`` is its thin ctypes binding.  Import ``paper_cs_0607001_gb300.sidwt``
to use it; this package root imports nothing heavy.
"""
