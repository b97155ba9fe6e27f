"""Independent pins for the oracle: exact integer arithmetic, a Fourier-space
closed form and the dense unitary built explicitly.  None of them calls the
oracle or the CUDA library."""
