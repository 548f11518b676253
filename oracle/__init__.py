"""CPU FP64 oracle (test infrastructure only; see swih_oracle.py)."""
