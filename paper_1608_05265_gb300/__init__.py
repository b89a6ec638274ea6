"""GB300-native single-precision GEMM (BLAS sgemm convention) with a plain FP32
SIMT path and a tcgen05 tensor-core path that splits each FP32 operand into
high and low BF16 parts.

Submodules:
  gbgemm   -- ctypes binding over the C-ABI library libgbgemm.so (the product)
  build    -- compiles the CUDA sources for sm_103a
  synth    -- seeded synthetic inputs (no GEMM arithmetic)
  metrics  -- FLOP counting and roofline bookkeeping
The binding is imported on first use so that the generator and metrics work
on machines without the built library.
"""

__all__ = ["gbgemm", "build", "synth", "metrics"]
