"""CPU oracle (test infrastructure only): see sofa_oracle.py."""
