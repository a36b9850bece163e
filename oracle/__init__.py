"""FP64 CPU oracle for SupPCG (test infrastructure; see oracle.py)."""
