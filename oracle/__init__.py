"""CPU FP64 oracle (test infrastructure only; see h2oracle.py)."""
