"""CPU oracle (test infrastructure only): see ``oracle.pcsir_oracle``."""
