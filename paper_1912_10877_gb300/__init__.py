"""GB300 (sm_103a) state-vector simulator hot path of Yao.jl (arXiv 1912.10877).

The compute runs in libqsim.so (CUDA kernels behind the C ABI of
include/qsim.h); this package is the thin binding.  Importing a submodule that
needs the library raises if it has not been built.
"""
from ._native import QsimError, lib  # noqa: F401
from .qsim import (BatchProgram, Circuit, Observable, State, apply_circuit_ckpt, backward,  # noqa: F401
                   backward_work, checkpoint_buffer)
