"""GB300-native per-cell uniform-patch radiation-hydrodynamics update.

Implements the data-parallel hot path of Wibking & Krumholz (arXiv:2110.01792):
the PPM + HLLC + RK2-SSP hydro stage with ghost fill (Sec. 2.2.1), the explicit
two-moment radiation stage with the Levermore closure and the reduced speed of
light (Sec. 2.2.2), and the per-cell implicit matter-radiation exchange
(Sec. 2.2.3), as hand-written sm_103a CUDA kernels behind the C ABI declared in
``include/qk.h``.  ``paper_2110_01792_gb300.qk`` is the Python binding (ctypes,
argument marshalling only); ``paper_2110_01792_gb300.inputs`` holds the seeded
synthetic workloads.
"""
__all__ = ["inputs", "qk"]
