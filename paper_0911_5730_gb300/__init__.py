"""Adaptive-multilevel BDDC (Sousedik & Mandel) on one GB300.

The compute path is the C-ABI library ``libbddc.so`` built from ``csrc/``;
``paper_0911_5730_gb300.bddc`` is its thin ctypes binding.  Importing the
package itself loads nothing, so the input generators in ``inputs`` stay
usable on machines without the library.
"""
