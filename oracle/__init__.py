"""FP64 CPU oracle (test infrastructure only; see nufft3d_oracle.py)."""
