"""Plain CPU oracle for the local trace (test infrastructure only; see oracle.py)."""
