"""CPU oracle (test infrastructure only): see oracle.py and srbe_oracle.c."""
