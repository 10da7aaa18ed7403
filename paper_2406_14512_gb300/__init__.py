"""GB300-native hybrid force-free / PIC time step for the aligned pulsar rotator
(Soudais, Cerutti & Contopoulos 2024).

The compute path is the CUDA library ``libhff.so`` (C ABI declared in
``include/hff.h``); :mod:`paper_2406_14512_gb300.hff` is its thin ctypes
binding.  The binding is imported lazily so that the input generators in
:mod:`paper_2406_14512_gb300.workloads` can be used without a GPU.
"""

__all__ = ["workloads", "hff"]
