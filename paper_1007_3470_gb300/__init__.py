"""GB300-native Hermite-Fourier split-step library (Bader & Blanes, arXiv 1007.3470).

``hfs`` is the ctypes binding of the C-ABI library ``libhfs.so`` built from
``csrc/``; ``workloads`` holds the seeded synthetic inputs.  Importing the
package does not load the CUDA library; ``hfs.lib()`` does, and fails loudly
when it is missing.
"""
