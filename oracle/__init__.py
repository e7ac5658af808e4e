"""CPU oracle for the WECT / ECF (test infrastructure only; see oracle.py)."""
