"""FP64 CPU oracle (test infrastructure only; see rd3q81.py)."""
