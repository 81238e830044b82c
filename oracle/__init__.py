"""CPU FP64 oracle (test infrastructure only; see gp_oracle.py)."""
