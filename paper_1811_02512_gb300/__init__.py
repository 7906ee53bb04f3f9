"""GB300-native graph-based power flow (arxiv 1811.02512, Section III hot path).

The compute path is the CUDA library ``libgbpf.so`` behind the C ABI declared
in ``include/gbpf.h``; ``paper_1811_02512_gb300.gbpf`` is its thin ctypes
binding.  ``gridgen`` synthesises seeded grids and scenarios.
"""
__all__ = ["gbpf", "gridgen"]
