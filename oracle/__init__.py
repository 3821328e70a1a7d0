"""CPU FP64 oracle (test infrastructure only; see heat.py's header)."""
