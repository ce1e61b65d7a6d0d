"""FP64 CPU oracle (test infrastructure only; see qudit_oracle.py)."""
