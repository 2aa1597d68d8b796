"""GB300 implementation of the F.A.S.T. time step (binding added with the CUDA library)."""
