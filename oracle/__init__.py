"""Plain, slow CPU FP64 (complex128) oracle of the hybrid stabilizer-tensor-
network simulation of noisy surface-code syndrome extraction under coherent
crosstalk (Harper, Nakhl, Sevior, Usman, "Non-Clifford Crosstalk Noise in
Surface Codes Using Hybrid Stabilizer-Tensor Network Methods").

This package is TEST INFRASTRUCTURE.  Only the tests, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` may import it.  It shares no code with
the CUDA path: the library compiles its own circuit, keeps its own tableau and
MPS, and draws its own Philox uniforms.

Modules: philox (random draws), pauli (exact Pauli algebra, Clifford tables
from gate matrices), tableau (inverse tableau, Eq. 7), mps (complex128 MPS,
MPO apply, QR/SVD truncation, Eq. 8), circuit (layout, schedule, program,
detectors; Sec. II-III), shot (one shot, Sec. IV).
"""
