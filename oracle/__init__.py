"""FP64 CPU oracle for XM: test infrastructure only (see xm_oracle)."""
