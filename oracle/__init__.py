"""CPU oracle of ABEA -- test infrastructure only (see oracle/oracle.py)."""
