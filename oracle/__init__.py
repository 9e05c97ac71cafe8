"""CPU oracle of the HSS-ULV path (test infrastructure only; see ulv.py)."""
