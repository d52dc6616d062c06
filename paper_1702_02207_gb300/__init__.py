"""cho: batched fixed-step RK4 for coupled linear oscillators M x'' + K x = 0 on GB300.

The compute path is the C-ABI library ``libcho.so`` (CUDA kernels for sm_103a);
``paper_1702_02207_gb300.cho`` is its thin ctypes binding.  Importing this
package does not load the library; ``cho.load()`` does, and raises if the
library has not been built.
"""
__all__ = ["inputs", "cho"]
