"""CPU oracle (test infrastructure only; see amg_oracle.py)."""
